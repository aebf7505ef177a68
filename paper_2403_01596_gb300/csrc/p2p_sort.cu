// Device-wide exclusive scan and stable LSD radix sort (plan-time building blocks
// of the leaf binning and of the work-item / packed-layout offsets).
#include "p2p_internal.cuh"

namespace p2p_detail {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096 elements per block

// Exclusive block-wide scan of one int per thread; returns the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* smem_warp, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(P2P_FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (kScanThreads / 32) ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(P2P_FULL_MASK, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kScanThreads / 32)) smem_warp[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    int warp_off = warp > 0 ? smem_warp[warp - 1] : 0;
    total = smem_warp[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* __restrict__ in, int64_t n,
                                                              int32_t* __restrict__ block_sums) {
    __shared__ int warp_sums[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    int total;
    block_exclusive_scan(s, warp_sums, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                            int64_t n, const int32_t* __restrict__ block_off,
                                                            int32_t* __restrict__ total_dev) {
    __shared__ int warp_sums[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int total;
    int pre = block_exclusive_scan(s, warp_sums, total);
    const int off = block_off ? block_off[blockIdx.x] : 0;
    pre += off;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = pre;
        pre += v[i];
    }
    if (total_dev && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_dev = off + total;
}

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortSub = 16;                           // sub-chunks of 256 keys per tile
constexpr int kSortTile = kSortThreads * kSortSub;     // 4096 keys per block

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                             uint32_t mask, int32_t* __restrict__ hist, int tiles) {
    __shared__ int cnt[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&cnt[(uint32_t)(keys[idx] >> shift) & mask], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[(int64_t)d * tiles + blockIdx.x] = cnt[d];
}

// Stable scatter: within a tile, keys are ranked in index order sub-chunk by
// sub-chunk; inside a sub-chunk the rank among equal digits comes from the
// warp match mask (lanes) and a per-digit prefix over warps.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t* __restrict__ keys_in,
                                                                const int32_t* __restrict__ vals_in,
                                                                uint64_t* __restrict__ keys_out,
                                                                int32_t* __restrict__ vals_out, int64_t n, int shift,
                                                                uint32_t mask, const int32_t* __restrict__ hist_off,
                                                                int tiles) {
    __shared__ int base[kRadix];
    __shared__ int warp_cnt[kSortWarps][kRadix];
    __shared__ int warp_base[kSortWarps][kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int d = tid; d < kRadix; d += kSortThreads) {
        base[d] = hist_off[(int64_t)d * tiles + blockIdx.x];
        for (int w = 0; w < kSortWarps; ++w) warp_cnt[w][d] = 0;
    }
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    for (int c = 0; c < kSortSub; ++c) {
        const int64_t idx = tile0 + (int64_t)c * kSortThreads + tid;
        const bool valid = idx < n;
        uint64_t key = valid ? keys_in[idx] : 0ull;
        int32_t val = valid ? vals_in[idx] : 0;
        const int d = valid ? (int)((uint32_t)(key >> shift) & mask) : kRadix;  // kRadix = sentinel
        const unsigned peers = __match_any_sync(P2P_FULL_MASK, d);
        const int rank = __popc(peers & lt_mask);
        const bool leader = (__ffs(peers) - 1) == lane;
        if (valid && leader) warp_cnt[warp][d] = __popc(peers);
        __syncthreads();
        for (int dd = tid; dd < kRadix; dd += kSortThreads) {
            int run = base[dd];
            for (int w = 0; w < kSortWarps; ++w) {
                int cnt = warp_cnt[w][dd];
                warp_base[w][dd] = run;
                warp_cnt[w][dd] = 0;
                run += cnt;
            }
            base[dd] = run;
        }
        __syncthreads();
        if (valid) {
            const int dst = warp_base[warp][d] + rank;
            keys_out[dst] = key;
            vals_out[dst] = val;
        }
    }
}

}  // namespace

size_t scan_workspace_bytes(int64_t n) {
    if (n <= kScanTile) return 0;
    int64_t nblk = (n + kScanTile - 1) / kScanTile;
    return align_up((size_t)nblk * 4, 256) * 2 + scan_workspace_bytes(nblk);
}

cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev, void* work,
                               cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(int32_t), s);
        return cudaSuccess;
    }
    int64_t nblk = (n + kScanTile - 1) / kScanTile;
    if (nblk == 1) {
        k_scan_down<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total_dev);
        return cudaGetLastError();
    }
    char* w = static_cast<char*>(work);
    int32_t* sums = reinterpret_cast<int32_t*>(w);
    int32_t* offs = reinterpret_cast<int32_t*>(w + align_up((size_t)nblk * 4, 256));
    void* rest = w + align_up((size_t)nblk * 4, 256) * 2;
    k_scan_reduce<<<(unsigned)nblk, kScanThreads, 0, s>>>(in, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive_i32(sums, offs, nblk, nullptr, rest, s);
    if (e != cudaSuccess) return e;
    k_scan_down<<<(unsigned)nblk, kScanThreads, 0, s>>>(in, out, n, offs, total_dev);
    return cudaGetLastError();
}

size_t radix_workspace_bytes(int64_t n) {
    int64_t tiles = (n + kSortTile - 1) / kSortTile;
    if (tiles < 1) tiles = 1;
    size_t h = align_up((size_t)tiles * kRadix * 4, 256);
    return 2 * h + scan_workspace_bytes(tiles * kRadix);
}

cudaError_t radix_sort_pairs(uint64_t* keys, int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, int64_t n,
                             int bits, void* work, cudaStream_t s, bool* result_in_alt) {
    *result_in_alt = false;
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int tiles = (int)((n + kSortTile - 1) / kSortTile);
    char* w = static_cast<char*>(work);
    const size_t h = align_up((size_t)tiles * kRadix * 4, 256);
    int32_t* hist = reinterpret_cast<int32_t*>(w);
    int32_t* hist_off = reinterpret_cast<int32_t*>(w + h);
    void* scan_work = w + 2 * h;
    uint64_t *kin = keys, *kout = keys_alt;
    int32_t *vin = vals, *vout = vals_alt;
    for (int shift = 0; shift < bits; shift += kRadixBits) {
        const int pass_bits = bits - shift < kRadixBits ? bits - shift : kRadixBits;
        const uint32_t mask = (1u << pass_bits) - 1u;
        k_radix_hist<<<tiles, kSortThreads, 0, s>>>(kin, n, shift, mask, hist, tiles);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = scan_exclusive_i32(hist, hist_off, (int64_t)tiles * kRadix, nullptr, scan_work, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<tiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, mask, hist_off, tiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint64_t* tk = kin;
        kin = kout;
        kout = tk;
        int32_t* tv = vin;
        vin = vout;
        vout = tv;
        *result_in_alt = !*result_in_alt;
    }
    return cudaSuccess;
}

}  // namespace p2p_detail
