// Leaf binning (Sec. 3.1, Morton order of Sec. 3.2), neighbour lists (Sec. 3.2,
// 27-box 3D neighbourhood) and plan construction including the redundant
// per-box packed layout (Sec. 3.3, eq. 6 - 8, collected on the device).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "p2p_internal.cuh"

namespace p2p_detail {

static thread_local char g_last_error[512] = "";

void set_cuda_error(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

void set_message(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

}  // namespace p2p_detail

using namespace p2p_detail;

// Box-group kernel tables (p2p_group.cu).
cudaError_t p2p_group_build(p2p_plan* p, const int32_t* nbr_ptr, const int32_t* nbr_idx, uint64_t* keys,
                            int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, void* radix_ws, int32_t* maxes,
                            cudaStream_t s, int32_t* cap);

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n, int per_block) { return (unsigned)((n + per_block - 1) / per_block); }

// ------------------------------------------------------------------ binning --

// cell = clamp(floor((double(x) - lo) / h), 0, ng - 1), with explicitly rounded
// double operations so no contraction can change the result.
__device__ __forceinline__ uint32_t cell_of(float x, double lo, double h, int ng) {
    double t = __ddiv_rn(__dsub_rn((double)x, lo), h);
    double f = floor(t);
    if (f < 0.0) f = 0.0;
    if (f > (double)(ng - 1)) f = (double)(ng - 1);
    return (uint32_t)f;
}

__global__ void k_keys(const float* __restrict__ pts, int64_t n, double lo0, double lo1, double lo2, double h, int ng,
                       uint64_t* __restrict__ keys, int32_t* __restrict__ vals, int32_t* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
        *bad = 1;
        x = y = z = 0.f;
    }
    keys[i] = p2p_morton(cell_of(x, lo0, h, ng), cell_of(y, lo1, h, ng), cell_of(z, lo2, h, ng));
    vals[i] = (int32_t)i;
}

__global__ void k_heads(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ head) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    head[s] = (s == 0 || keys[s] != keys[s - 1]) ? 1 : 0;
}

__global__ void k_rle(const uint64_t* __restrict__ keys, const int32_t* __restrict__ vals,
                      const int32_t* __restrict__ head, const int32_t* __restrict__ ex, int64_t n,
                      int32_t* __restrict__ perm, int32_t* __restrict__ point_box, int64_t* __restrict__ box_keys,
                      int32_t* __restrict__ box_ptr) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int32_t id = ex[s] + head[s] - 1;
    if (head[s]) {
        box_keys[id] = (int64_t)keys[s];
        box_ptr[id] = (int32_t)s;
    }
    const int32_t orig = vals[s];
    perm[s] = orig;
    point_box[orig] = id;
    if (s == n - 1) box_ptr[id + 1] = (int32_t)n;
}

// --------------------------------------------------------------- neighbours --

__device__ __forceinline__ int32_t find_key(const int64_t* __restrict__ keys, int32_t nb, int64_t key) {
    int32_t lo = 0, hi = nb - 1;
    while (lo <= hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        int64_t v = __ldg(keys + mid);
        if (v == key) return mid;
        if (v < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// Ascending bitonic sort of one int per lane across the warp.
__device__ __forceinline__ int32_t warp_sort_asc(int32_t v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            int32_t o = __shfl_xor_sync(P2P_FULL_MASK, v, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            v = (lower == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

// One warp per target box; lane l < 27 probes the offset (l%3-1, (l/3)%3-1, l/9-1)
// among the source boxes' keys (the same keys for a one-set structure, TWO = false).
template <bool FILL, bool TWO>
__global__ void k_neighbors(const int64_t* __restrict__ box_keys, int32_t nb, const int64_t* __restrict__ src_keys,
                            int32_t nbs, const int32_t* __restrict__ src_box_ptr, int ng, int32_t* __restrict__ cnt,
                            int32_t* __restrict__ src_cnt, const int32_t* __restrict__ nbr_ptr,
                            int32_t* __restrict__ nbr_idx, int32_t* __restrict__ nbr_self, int32_t* __restrict__ bad) {
    const int lane = threadIdx.x & 31;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const uint64_t key = (uint64_t)box_keys[b];
    const int cx = (int)p2p_compact3(key), cy = (int)p2p_compact3(key >> 1), cz = (int)p2p_compact3(key >> 2);
    int32_t id = -1;
    if (lane < 27) {
        int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
        if (x >= 0 && y >= 0 && z >= 0 && x < ng && y < ng && z < ng)
            id = find_key(src_keys, nbs, (int64_t)p2p_morton(x, y, z));
    }
    const unsigned found = __ballot_sync(P2P_FULL_MASK, id >= 0);
    if (!FILL) {
        int s = id >= 0 ? src_box_ptr[id + 1] - src_box_ptr[id] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(P2P_FULL_MASK, s, o);
        if (lane == 0) {
            cnt[b] = __popc(found);
            src_cnt[b] = s;
            if (b > 0 && box_keys[b - 1] >= box_keys[b]) *bad = 1;  // keys must strictly ascend
            if (!TWO && !((found >> 13) & 1u)) *bad = 1;             // a box must find itself
        }
    } else {
        int32_t v = warp_sort_asc(id >= 0 ? id : INT32_MAX, lane);
        if (lane < __popc(found)) nbr_idx[nbr_ptr[b] + lane] = v;
        if (TWO) {
            // position of the source box of the target box's own cell (probe 13) in the sorted list
            const int32_t self = __shfl_sync(P2P_FULL_MASK, id, 13);
            const unsigned at = __ballot_sync(P2P_FULL_MASK, self >= 0 && v == self);
            if (lane == 0) nbr_self[b] = at ? __ffs(at) - 1 : -1;
        }
    }
}

__global__ void k_keys_ascending(const int64_t* __restrict__ keys, int32_t n, int32_t* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > 0 && i < n && keys[i - 1] >= keys[i]) *bad = 1;
}

__global__ void k_sum_i32(const int32_t* __restrict__ v, int64_t n, unsigned long long* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long s = i < n ? (long long)v[i] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(P2P_FULL_MASK, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, (unsigned long long)s);
}

// -------------------------------------------------------------------- plans --

__global__ void k_gather_xyz(const float* __restrict__ pts, const int32_t* __restrict__ perm, int64_t n,
                             float4* __restrict__ xs) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t j = perm[s];
    xs[s] = make_float4(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], 0.f);
}

// Per target box: S_b, work-item count ceil(S_b / chunk) and the padded length
// of its source list, and the size of the source box of its own cell (the
// sources that can sit at r = 0 from one of its targets).  Validates the CSR
// (ascending ids in range; a one-set structure lists each box itself, a two-set
// structure's nbr_self must point into the list or be -1).
__global__ void k_box_info(const int32_t* __restrict__ box_ptr, const int32_t* __restrict__ src_box_ptr,
                           int32_t nbs, const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                           const int32_t* __restrict__ nbr_self, int32_t nb, int64_t nnz, int chunk, int upper,
                           int32_t* __restrict__ box_src, int32_t* __restrict__ list_len,
                           int32_t* __restrict__ n_chunks, int32_t* __restrict__ padded, int32_t* __restrict__ self_len,
                           int32_t* __restrict__ maxes, unsigned int* __restrict__ status) {
    int32_t b = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (b >= nb) return;
    int32_t e0 = nbr_ptr[b], e1 = nbr_ptr[b + 1];
    int64_t s = 0, s_up = 0;
    int32_t self = -1, self_n = 0;
    bool ok = e0 >= 0 && e1 >= e0 && e1 <= nnz && e1 - e0 <= 27;
    if (ok) {
        const int32_t want = nbr_self ? nbr_self[b] : -2;
        if (nbr_self && (want < -1 || want >= e1 - e0)) ok = false;
        for (int32_t e = e0; ok && e < e1; ++e) {
            int32_t c = nbr_idx[e];
            if (c < 0 || c >= nbs || (e > e0 && c <= nbr_idx[e - 1])) {
                ok = false;
                break;
            }
            const int32_t sz = src_box_ptr[c + 1] - src_box_ptr[c];
            if (nbr_self ? (e - e0 == want) : (c == b)) {
                self = e - e0;
                self_n = sz;
            }
            s += sz;
            if (c >= b) s_up += sz;
        }
    }
    int32_t own = box_ptr[b + 1] - box_ptr[b];
    if (!ok || (!nbr_self && self < 0) || own <= 0 || s > INT32_MAX - 4) {
        atomicOr(status, P2P_DEV_BAD_INPUT);
        s = 0;
        s_up = 0;
        self_n = 0;
    }
    box_src[b] = (int32_t)s;
    self_len[b] = self_n;
    const int64_t len = upper ? s_up : s;  // length of the box's source list
    list_len[b] = (int32_t)len;
    int32_t c = (int32_t)((len + chunk - 1) / chunk);
    n_chunks[b] = c;
    padded[b] = (int32_t)((len + 3) & ~3ll);
    atomicMax(&maxes[0], c);
    atomicMax(&maxes[1], own);
    // lists just over one chunk: a full item plus a short tail item (counted for the default-tuning choice)
    if (len > chunk && 3 * len <= 4ll * chunk) atomicAdd(&maxes[2], 1);
    atomicAdd(&maxes[3], c);  // work items in all
}

// Work-item records (unsorted) and their sort keys: larger cost (targets x
// sources) first.
__global__ void k_item_records(const int32_t* __restrict__ n_chunks, const int32_t* __restrict__ item_off,
                               const int32_t* __restrict__ box_ptr, const int32_t* __restrict__ list_len,
                               const int32_t* __restrict__ self_len, const int32_t* __restrict__ pk_off, int32_t nb,
                               int chunk, int tg, int two_sets, ItemRec* __restrict__ recs,
                               uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
    int32_t b = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (b >= nb) return;
    const int32_t c = n_chunks[b], o = item_off[b];
    const int32_t tb = box_ptr[b], nt = box_ptr[b + 1] - tb, S = list_len[b];
    const int32_t last = nt - ((nt - 1) / tg) * tg;  // targets of the last target group
    // the list in c near-equal items (multiples of 4 entries but the last, at most chunk each) rather than c - 1
    // full items and a short tail
    int32_t L = c > 1 ? (((S + c - 1) / c + 3) & ~3) : chunk;
    if ((c - 1) * L >= S) L = chunk;
    for (int32_t i = 0; i < c; ++i) {
        const int32_t s0 = i * L;
        ItemRec r;
        r.src_off = pk_off[b] + s0;
        r.ns = min(L, S - s0);
        r.tb = tb;
        r.nt = nt;
        // the own cell's sources lead the list; in a one-set plan they are the box's targets themselves
        r.m_end = max(0, min(r.ns, self_len[b] - s0)) | ((s0 == 0 && !two_sets) ? (1 << 16) : 0);
        r.map_full = p2p_lane_map(min(nt, tg), r.ns);
        r.map_last = p2p_lane_map(last, r.ns);
        r.b = b;
        recs[o + i] = r;
        keys[o + i] = 0xFFFFFFFFull - (uint64_t)min((int64_t)nt * r.ns, (int64_t)0xFFFFFFFF);
        vals[o + i] = o + i;
    }
}

__global__ void k_item_gather(const ItemRec* __restrict__ recs, const int32_t* __restrict__ order, int64_t n,
                              ItemRec* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = recs[order[i]];
}

// Direct-kernel items: one per target box, its whole source list, lane maps for
// `lanes` lanes (passes of up to 4 * lanes targets), sort keys by decreasing cost.
__global__ void k_direct_items(const int32_t* __restrict__ box_ptr, const int32_t* __restrict__ list_len,
                               const int32_t* __restrict__ self_len, const int32_t* __restrict__ pk_off, int32_t nb,
                               int lanes, ItemRec* __restrict__ recs, uint64_t* __restrict__ keys,
                               int32_t* __restrict__ vals) {
    const int32_t b = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (b >= nb) return;
    const int32_t tb = box_ptr[b], nt = box_ptr[b + 1] - tb, S = list_len[b];
    const int pass = 4 * lanes;
    const int32_t last = nt - ((nt - 1) / pass) * pass;
    ItemRec r;
    r.src_off = pk_off[b];
    r.ns = S;
    r.tb = tb;
    r.nt = nt;
    r.m_end = min(S, self_len[b]);
    r.map_full = p2p_lane_map(min(nt, pass), S, lanes, 8);
    r.map_last = p2p_lane_map(last, S, lanes, 8);
    r.b = b;
    recs[b] = r;
    keys[b] = 0xFFFFFFFFull - (uint64_t)min((int64_t)nt * S, (int64_t)0xFFFFFFFF);
    vals[b] = b;
}

// Source groups of the tensor-core path: ceil(n_b / 16) per box.
__global__ void k_tc_groups(const int32_t* __restrict__ box_ptr, int32_t nb, int32_t* __restrict__ groups) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) groups[b] = (box_ptr[b + 1] - box_ptr[b] + 15) / 16;
}

// Length of every box's group list: the groups of its neighbour boxes, and that
// count padded to a multiple of 4.
__global__ void k_tc_list_len(const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                              const int32_t* __restrict__ gstart, int32_t nb, int32_t* __restrict__ count,
                              int32_t* __restrict__ padded) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int g = 0;
    for (int e = nbr_ptr[b]; e < nbr_ptr[b + 1]; ++e) {
        const int c = nbr_idx[e];
        g += gstart[c + 1] - gstart[c];
    }
    count[b] = g;
    padded[b] = (g + 3) & ~3;
}

// Group lists: neighbour boxes in ascending id, each box's groups in order, -1 padding.
__global__ void k_tc_list_fill(const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                               const int32_t* __restrict__ gstart, const int32_t* __restrict__ off, int32_t nb,
                               int32_t* __restrict__ list) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int o = off[b];
    for (int e = nbr_ptr[b]; e < nbr_ptr[b + 1]; ++e) {
        const int c = nbr_idx[e];
        for (int g = gstart[c]; g < gstart[c + 1]; ++g) list[o++] = g;
    }
    while (o < off[b + 1]) list[o++] = -1;
}

// One warp per target box: writes the box's source list -- the sources of its
// own cell first (the box itself in a one-set plan, the source box of the same
// cell in a two-set plan), then the other neighbour boxes in ascending id (the
// order the pair kernel's r = 0 mask relies on) -- as box-sorted source indices
// (nb_src, the index arrays of the indexing method, Sec. 3.2) and, for the
// redundant layout, as a copy of the coordinates plus original indices (the
// repetition of Sec. 3.3).  xs, perm and box_ptr are the SOURCE side.
__global__ void k_pack(const float4* __restrict__ xs, const int32_t* __restrict__ perm,
                       const int32_t* __restrict__ box_ptr, const int32_t* __restrict__ nbr_ptr,
                       const int32_t* __restrict__ nbr_idx, const int32_t* __restrict__ nbr_self,
                       const int32_t* __restrict__ pk_off, int32_t nb, int upper, int32_t* __restrict__ nb_src,
                       float4* __restrict__ pk_xyz, int32_t* __restrict__ pk_src) {
    const int lane = threadIdx.x & 31;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const int32_t e0 = nbr_ptr[b];
    int32_t ne = nbr_ptr[b + 1] - e0;
    const int32_t c = lane < ne ? nbr_idx[e0 + lane] : -1;
    int sp;
    if (nbr_self) {
        sp = nbr_self[b];  // -1: no source box in the own cell, the list keeps ascending order
    } else {
        const unsigned selfm = __ballot_sync(P2P_FULL_MASK, c == (int32_t)b);
        sp = selfm ? __ffs(selfm) - 1 : 0;
    }
    // full list: slot 0 <- own cell, slots 1..sp <- entries 0..sp-1, later slots unchanged;
    // upper list (own box and higher ids only): slot i <- entry sp + i
    int from = sp < 0 ? lane : (lane == 0 ? sp : (lane <= sp ? lane - 1 : lane));
    if (upper) {
        from = min(sp + lane, 31);
        ne -= sp;
    }
    const int32_t cs = __shfl_sync(P2P_FULL_MASK, c, from);
    int32_t start = 0, len = 0;
    if (lane < ne) {
        start = box_ptr[cs];
        len = box_ptr[cs + 1] - start;
    }
    int32_t incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(P2P_FULL_MASK, incl, o);
        if (lane >= o) incl += y;
    }
    const int32_t excl = incl - len;
    const int32_t total = __shfl_sync(P2P_FULL_MASK, incl, 31);
    const int64_t base = pk_off[b];
    const int32_t padded = pk_off[b + 1] - pk_off[b];
    for (int32_t p0 = 0; p0 < padded; p0 += 32) {
        const int32_t p = p0 + lane;
        int32_t seg = 0;
        for (int e = 0; e < ne; ++e) {
            int32_t ex = __shfl_sync(P2P_FULL_MASK, excl, e);
            if (p >= ex) seg = e;
        }
        const int32_t s0 = __shfl_sync(P2P_FULL_MASK, start, seg);
        const int32_t x0 = __shfl_sync(P2P_FULL_MASK, excl, seg);
        if (p < total) {
            const int32_t j = s0 + (p - x0);
            nb_src[base + p] = j;
            if (pk_xyz) {
                pk_xyz[base + p] = xs[j];
                pk_src[base + p] = perm[j];
            }
        } else if (p < padded) {
            nb_src[base + p] = -1;
            if (pk_xyz) {
                pk_xyz[base + p] = make_float4(0.f, 0.f, 0.f, 0.f);
                pk_src[base + p] = -1;
            }
        }
    }
}

// Pairs of target box b: n_b * S_b minus the (target, source) pairs of its own
// cell with identical coordinates (xt / box_ptr: targets; xs / src_box_ptr:
// sources; self_len / nbr_self locate the own cell's source box).
__global__ void k_pair_count(const float4* __restrict__ xt, const int32_t* __restrict__ box_ptr,
                             const float4* __restrict__ xs, const int32_t* __restrict__ src_box_ptr,
                             const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                             const int32_t* __restrict__ nbr_self, const int32_t* __restrict__ box_src, int32_t nb,
                             unsigned long long* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const int32_t t0 = box_ptr[b], t1 = box_ptr[b + 1];
    int32_t c = (int32_t)b;
    if (nbr_self) c = nbr_self[b] >= 0 ? nbr_idx[nbr_ptr[b] + nbr_self[b]] : -1;
    long long dup = 0;
    if (c >= 0) {
        const int32_t s0 = src_box_ptr[c], s1 = src_box_ptr[c + 1];
        for (int32_t i = t0 + lane; i < t1; i += 32) {
            float4 a = xt[i];
            for (int32_t j = s0; j < s1; ++j) {
                float4 q = xs[j];
                dup += (a.x == q.x && a.y == q.y && a.z == q.z) ? 1 : 0;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dup += __shfl_xor_sync(P2P_FULL_MASK, dup, o);
    if (lane == 0) {
        long long p = (long long)(t1 - t0) * (long long)box_src[b] - dup;
        atomicAdd(out, (unsigned long long)p);
    }
}

// Points (sorted position s) whose new coordinates fall in another grid cell
// than the coordinates the plan holds (same cell rule as the binning), and
// non-finite new coordinates.
__global__ void k_moved(const float* __restrict__ pts, const int32_t* __restrict__ perm,
                        const float4* __restrict__ xs, int64_t n, double lo0, double lo1, double lo2, double h, int ng,
                        unsigned long long* __restrict__ moved, int32_t* __restrict__ bad) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t j = perm[s];
    const float x = pts[3 * j], y = pts[3 * j + 1], z = pts[3 * j + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
        *bad = 1;
        return;
    }
    const float4 o = xs[s];
    if (cell_of(x, lo0, h, ng) != cell_of(o.x, lo0, h, ng) || cell_of(y, lo1, h, ng) != cell_of(o.y, lo1, h, ng) ||
        cell_of(z, lo2, h, ng) != cell_of(o.z, lo2, h, ng))
        atomicAdd(moved, 1ull);
}

// Redundant layout: the per-box copies of the listed source coordinates from the box-sorted ones.
__global__ void k_repack_xyz(const float4* __restrict__ xs, const int32_t* __restrict__ nb_src, int64_t packed,
                             float4* __restrict__ pk_xyz) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= packed) return;
    const int32_t j = nb_src[p];
    pk_xyz[p] = j >= 0 ? xs[j] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Repetition layout: entries of the records of box b's targets, n_b (1 + S_b).
__global__ void k_rep_count(const int32_t* __restrict__ box_ptr, const int32_t* __restrict__ box_src, int32_t nb,
                            int32_t* __restrict__ cnt) {
    const int32_t b = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (b < nb) cnt[b] = (box_ptr[b + 1] - box_ptr[b]) * (1 + box_src[b]);
}

// One warp per box: the records of its targets -- entry 0 the target's coordinates, entries 1 .. S_b a copy of
// the box's source list (own box first, then the other neighbour boxes in ascending id) with the sources'
// original indices, for the per-apply strength repack (the collection of Sec. 3.3, eq. 6, on the device).
__global__ void k_rep_fill(const float4* __restrict__ xs, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ box_ptr, const int32_t* __restrict__ box_src,
                           const int32_t* __restrict__ pk_off, const int32_t* __restrict__ nb_src,
                           const int32_t* __restrict__ rec_boff, int32_t nb, int64_t n, int32_t* __restrict__ rec_off,
                           float4* __restrict__ rec_xyz, int32_t* __restrict__ rec_src) {
    const int lane = threadIdx.x & 31;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const int32_t tb = box_ptr[b], nt = box_ptr[b + 1] - tb, S = box_src[b], len = 1 + S;
    const int32_t* list = nb_src + pk_off[b];
    for (int32_t u = 0; u < nt; ++u) {
        const int64_t base = (int64_t)rec_boff[b] + (int64_t)u * len;
        if (lane == 0) {
            rec_off[tb + u] = (int32_t)base;
            rec_xyz[base] = xs[tb + u];
            rec_src[base] = -1;
        }
        for (int32_t p = lane; p < S; p += 32) {
            const int32_t j = list[p];
            rec_xyz[base + 1 + p] = xs[j];
            rec_src[base + 1 + p] = perm[j];
        }
    }
    if (b == nb - 1 && lane == 0) rec_off[n] = rec_boff[nb];
}

int ceil_log2(int v) {
    int b = 0;
    while ((1 << b) < v) ++b;
    return b;
}

struct BinLayout {
    uint64_t *keys, *keys_alt;
    int32_t *vals, *vals_alt, *head, *ex, *small;
    void *radix_ws, *scan_ws;
    size_t bytes;
};

BinLayout bin_layout(int64_t n, void* work) {
    Carver c{static_cast<char*>(work), 0, (size_t)-1};
    BinLayout L;
    size_t m = (size_t)(n > 0 ? n : 1);
    L.keys = c.take<uint64_t>(m);
    L.keys_alt = c.take<uint64_t>(m);
    L.vals = c.take<int32_t>(m);
    L.vals_alt = c.take<int32_t>(m);
    L.head = c.take<int32_t>(m);
    L.ex = c.take<int32_t>(m);
    L.small = c.take<int32_t>(4);
    L.radix_ws = c.take<char>(radix_workspace_bytes(n));
    L.scan_ws = c.take<char>(scan_workspace_bytes(n));
    L.bytes = align_up(c.off, 256);
    return L;
}

struct NbrLayout {
    int32_t *cnt, *src_cnt, *bad;
    unsigned long long* sum;
    void* scan_ws;
    size_t bytes;
};

NbrLayout nbr_layout(int32_t nb, void* work) {
    Carver c{static_cast<char*>(work), 0, (size_t)-1};
    NbrLayout L;
    size_t m = (size_t)(nb > 0 ? nb : 1);
    L.cnt = c.take<int32_t>(m);
    L.src_cnt = c.take<int32_t>(m);
    L.bad = c.take<int32_t>(2);
    L.sum = c.take<unsigned long long>(1);
    L.scan_ws = c.take<char>(scan_workspace_bytes(nb));
    L.bytes = align_up(c.off, 256);
    return L;
}

bool tuning_valid(const p2p_tuning& t) {
    return t.chunk >= 32 && t.chunk <= 1024 && t.chunk % 32 == 0 && t.warps_per_cta >= 1 && t.warps_per_cta <= 16 &&
           t.target_group >= 32 && t.target_group <= 128 && t.target_group % 32 == 0 &&
           (t.warp_boxes == -2 || t.warp_boxes == -1 || t.warp_boxes == 0 || t.warp_boxes == 1 ||
            t.warp_boxes == 2 || t.warp_boxes == 4 || t.warp_boxes == 8 || t.warp_boxes == 16 || t.warp_boxes == 32);
}

// Default launch tuning; a plan whose caller leaves chunk and warps at zero may switch to kWideTuning or
// kNarrowTuning (see p2p_plan_create).
constexpr p2p_tuning kDefaultTuning{192, 8, 32, 0};
constexpr p2p_tuning kWideTuning{256, 6, 32, 0};
constexpr p2p_tuning kNarrowTuning{128, 8, 32, 0};

bool tuning_is_auto(const p2p_tuning* t) { return !t || (t->chunk == 0 && t->warps_per_cta == 0); }

p2p_tuning resolve_tuning(const p2p_tuning* t) {
    p2p_tuning r = kDefaultTuning;
    if (t) {
        if (t->chunk) r.chunk = t->chunk;
        if (t->warps_per_cta) r.warps_per_cta = t->warps_per_cta;
        if (t->target_group) r.target_group = t->target_group;
        r.warp_boxes = t->warp_boxes;
    }
    return r;
}

// Boxes per warp of the direct kernel for a plan left to choose (warp_boxes = 0), from the mean number of
// targets per box D.  Measured on GB300: the 2^20-point sphere at D = 8 (185 us with four boxes per warp
// against 217 us staged) and D = 16 (staged 290 us, direct 293 - 340 us), and square plates of 2^10 - 2^20
// points at D = 1.0 - 4 (at 2^20 points: D = 4.1, eight boxes per warp 74 us, four 82 us, staged 258 us;
// D = 1.6, sixteen 64 us; D = 1.0 - 1.1, thirty-two 39 - 47 us).
// Largest union the box-group kernel stages (sources; 24 bytes each in shared memory; its positions are 16-bit).
constexpr int32_t kGroupCapMax = 8192;

//
// Above that, up to D = 24, the box-group kernel (-2; indexed layout only, other layouts keep the staged
// pipeline): the sphere at D = 16, 259 us against 292 us staged (groups of 16 boxes, 24 warps per SM); at D = 32
// it measured 571 us against 474 staged, at D = 8 222 us against the direct kernel's 185.  A uniform cube gives
// the same ranking (D = 16: 0.228 ms against 0.274 staged, D = 24: 0.470 against 0.512, D = 32: 0.137 against
// 0.122).
int32_t auto_warp_boxes(int64_t n, int32_t nb) {
    if (nb <= 0) return -1;
    const double d = (double)n / nb;
    if (d <= 1.3) return 32;
    if (d <= 2.5) return 16;
    if (d <= 6.0) return 8;
    if (d <= 12.0) return 4;
    if (d <= 24.0) return -2;
    return -1;
}

struct PlanLayout {
    p2p_plan p;  // pointers only
    int32_t *n_chunks, *item_off, *padded, *maxes, *small, *list_len, *self_len;
    void* scan_ws;
    // item-sort scratch (aliases the strength staging buffer when it is large enough)
    ItemRec* recs;
    uint64_t *keys, *keys_alt;
    int32_t *vals, *vals_alt;
    void* radix_ws;
    size_t bytes;
};

// Sizes of a plan: n targets in nb boxes, n_src sources in nbs boxes (two_sets), sources = sum of S_b.
PlanLayout plan_layout(int64_t n, int32_t nb, int64_t n_src, int32_t nbs, bool two_sets, int64_t sources, int64_t nnz,
                       p2p_layout layout, int32_t max_nrhs, const p2p_tuning& t, void* ws, int64_t records = 0) {
    Carver c{static_cast<char*>(ws), 0, (size_t)-1};
    PlanLayout L;
    memset(&L.p, 0, sizeof(L.p));
    size_t m = (size_t)(n > 0 ? n : 1), mb = (size_t)(nb > 0 ? nb : 1);
    size_t ms = (size_t)(n_src > 0 ? n_src : 1), mbs = (size_t)(nbs > 0 ? nbs : 1);
    // room for the items of the narrowest chunk a plan may switch to
    const int sizing_chunk = t.chunk < kNarrowTuning.chunk ? t.chunk : kNarrowTuning.chunk;
    const size_t max_items = (size_t)(sources / sizing_chunk) + mb + 1;
    const size_t list_bound = (size_t)sources + 3 * mb + 4;
    const bool red = layout == P2P_LAYOUT_REDUNDANT;
    L.p.status = c.take<unsigned int>(4);
    L.p.scratch64 = c.take<long long>(4);
    L.p.xs = c.take<float4>(m);
    L.p.xs_src = two_sets ? c.take<float4>(ms) : L.p.xs;
    L.p.box_src = c.take<int32_t>(mb);
    L.p.items = c.take<ItemRec>(max_items);
    L.p.ditems = c.take<ItemRec>(mb);
    if (layout == P2P_LAYOUT_INDEXED && (t.warp_boxes == -2 || (t.warp_boxes == 0 && auto_warp_boxes(n, nb) == -2))) {
        // box-group kernel tables (requested, or the plan's own choice)
        const size_t ngr = (mb + kGroupBoxes - 1) / kGroupBoxes;
        L.p.g_union = c.take<int32_t>(ngr * kGroupBoxes * 27);
        L.p.g_nunion = c.take<int32_t>(ngr);
        L.p.g_order = c.take<int32_t>(ngr);
        L.p.g_pos = c.take<int16_t>(list_bound);
        L.p.g_mend = c.take<int32_t>(mb);
        L.p.g_map = c.take<int32_t>(2 * mb);
        L.p.g_morder = c.take<int32_t>(ngr * kGroupBoxes);
        L.p.g_copy = c.take<int4>(ngr * kGroupBoxes * 27);
    }
    L.p.pk_off = c.take<int32_t>(mb + 1);
    L.p.nb_src = c.take<int32_t>(list_bound);
    L.p.pk_xyz = red ? c.take<float4>(list_bound) : nullptr;
    L.p.pk_src = red ? c.take<int32_t>(list_bound) : nullptr;
    const bool rep = layout == P2P_LAYOUT_REPETITION;
    const size_t mr = (size_t)(records > 0 ? records : 1);
    L.p.rec_off = rep ? c.take<int32_t>(m + 1) : nullptr;
    L.p.rec_boff = rep ? c.take<int32_t>(mb + 1) : nullptr;
    L.p.rec_xyz = rep ? c.take<float4>(mr) : nullptr;
    L.p.rec_src = rep ? c.take<int32_t>(mr) : nullptr;
    size_t lam_rows = red ? (ms > list_bound ? ms : list_bound) : ms;
    if (rep && mr > lam_rows) lam_rows = mr;
    const size_t lam_bytes = lam_rows * (size_t)max_nrhs * sizeof(float2);
    L.p.lam_buf = c.take<float2>(lam_rows * (size_t)max_nrhs);
    L.p.g_buf = two_sets ? nullptr : c.take<float2>(m * (size_t)max_nrhs);
    const size_t tc_bytes = p2p_tc_pack_bytes((int64_t)ms, (int32_t)mbs, max_nrhs);
    L.p.tc_gstart = tc_bytes ? c.take<int32_t>(mbs + 1) : nullptr;
    L.p.tc_glist_off = tc_bytes ? c.take<int32_t>(mb + 1) : nullptr;
    L.p.tc_gcount = tc_bytes ? c.take<int32_t>(mb) : nullptr;
    L.p.tc_glist = tc_bytes ? c.take<int32_t>(p2p_tc_list_bound(sources, nnz, (int32_t)mb)) : nullptr;
    L.p.tc_pack = tc_bytes ? c.take<unsigned char>(tc_bytes) : nullptr;
    const size_t mx = mb > mbs ? mb : mbs;
    L.n_chunks = c.take<int32_t>(mx);
    L.list_len = c.take<int32_t>(mb);
    L.self_len = c.take<int32_t>(mb);
    L.item_off = c.take<int32_t>(mb + 1);
    L.padded = c.take<int32_t>(mb);
    L.maxes = c.take<int32_t>(4);
    L.small = c.take<int32_t>(4);
    L.scan_ws = c.take<char>(scan_workspace_bytes((int64_t)mx));
    // sort scratch: inside lam_buf if it fits, else after everything else
    Carver sc{reinterpret_cast<char*>(L.p.lam_buf), 0, lam_bytes};
    sc.take<ItemRec>(max_items);
    sc.take<uint64_t>(max_items);
    sc.take<uint64_t>(max_items);
    sc.take<int32_t>(max_items);
    sc.take<int32_t>(max_items);
    sc.take<char>(radix_workspace_bytes((int64_t)max_items));
    Carver& cs = (sc.off <= lam_bytes) ? sc : c;
    if (&cs == &sc) sc.off = 0;
    L.recs = cs.take<ItemRec>(max_items);
    L.keys = cs.take<uint64_t>(max_items);
    L.keys_alt = cs.take<uint64_t>(max_items);
    L.vals = cs.take<int32_t>(max_items);
    L.vals_alt = cs.take<int32_t>(max_items);
    L.radix_ws = cs.take<char>(radix_workspace_bytes((int64_t)max_items));
    L.bytes = align_up(c.off, 256);
    return L;
}

// Everything a plan is made from: the target side (points, perm, boxes), the
// source side (the same arrays for a one-set plan) and the target-to-source
// neighbour CSR.
struct PlanInput {
    const float* pts;
    int64_t n;
    const int32_t* perm;
    const int32_t* box_ptr;
    int32_t nb;
    const float* src_pts;
    int64_t n_src;
    const int32_t* src_perm;
    const int32_t* src_box_ptr;
    int32_t nbs;
    const int32_t* nbr_ptr;
    const int32_t* nbr_idx;
    const int32_t* nbr_self;  // NULL for one-set plans
    int64_t nnz;
    int64_t sources;
    bool two_sets;
};

p2p_status check_sizes(int64_t n, int32_t nb, int64_t n_src, int32_t nbs, int64_t sources, p2p_layout layout,
                       int32_t max_nrhs, bool two_sets) {
    if (n < 0 || n >= INT32_MAX || nb < 0 || nb > n || n_src < 0 || n_src >= INT32_MAX || nbs < 0 || nbs > n_src ||
        sources < 0 || sources >= INT32_MAX || max_nrhs < 1 || max_nrhs > 256)
        return P2P_ERR_INVALID;
    if (layout != P2P_LAYOUT_INDEXED && layout != P2P_LAYOUT_REDUNDANT && layout != P2P_LAYOUT_SYMMETRIC &&
        layout != P2P_LAYOUT_REPETITION)
        return P2P_ERR_INVALID;
    if (two_sets && (layout == P2P_LAYOUT_SYMMETRIC || layout == P2P_LAYOUT_REPETITION)) return P2P_ERR_UNSUPPORTED;
    if (layout == P2P_LAYOUT_REPETITION && max_nrhs != 1) return P2P_ERR_UNSUPPORTED;
    return P2P_OK;
}

p2p_status plan_create(p2p_plan** plan, const PlanInput& in, p2p_kernel kernel, float k, p2p_layout layout,
                       int32_t max_nrhs, const p2p_tuning* tuning, void* workspace, size_t workspace_bytes,
                       cudaStream_t s);

}  // namespace

// ===================================================================== C ABI ==

extern "C" {

P2P_API int32_t p2p_version(void) { return 100; }

P2P_API const char* p2p_status_string(p2p_status s) {
    switch (s) {
        case P2P_OK: return "ok";
        case P2P_ERR_INVALID: return "invalid argument or input";
        case P2P_ERR_WORKSPACE: return "workspace too small";
        case P2P_ERR_CUDA: return "CUDA error";
        case P2P_ERR_TIMEOUT: return "device-side wait timed out";
        case P2P_ERR_UNSUPPORTED: return "unsupported";
        case P2P_ERR_ALLOC: return "host allocation failed";
        case P2P_ERR_STALE: return "a point left its leaf box: rebuild the plan";
    }
    return "unknown status";
}

P2P_API const char* p2p_last_error_string(void) { return g_last_error; }

P2P_API p2p_status p2p_bin_workspace_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 0 || n >= INT32_MAX) return P2P_ERR_INVALID;
    *bytes = bin_layout(n, nullptr).bytes;
    return P2P_OK;
}

P2P_API p2p_status p2p_bin_points(const float* pts, int64_t n, const double lo[3], double h, int32_t ng,
                                  int32_t* perm, int32_t* point_box, int64_t* box_keys, int32_t* box_ptr,
                                  int32_t* num_boxes, void* work, size_t work_bytes, p2p_stream_t stream) {
    if (n < 0 || n >= INT32_MAX || !lo || !num_boxes || !box_ptr || !(h > 0.0) || !isfinite(h) || ng < 1 ||
        ng > (1 << 21))
        return P2P_ERR_INVALID;
    if (!isfinite(lo[0]) || !isfinite(lo[1]) || !isfinite(lo[2])) return P2P_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    *num_boxes = 0;
    if (n == 0) {
        P2P_TRY_CUDA(cudaMemsetAsync(box_ptr, 0, sizeof(int32_t), s), "p2p_bin_points");
        P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_bin_points");
        return P2P_OK;
    }
    if (!pts || !perm || !point_box || !box_keys || !work) return P2P_ERR_INVALID;
    if (((uintptr_t)pts & 3) || ((uintptr_t)work & 255)) return P2P_ERR_INVALID;
    BinLayout L = bin_layout(n, work);
    if (work_bytes < L.bytes) return P2P_ERR_WORKSPACE;

    P2P_TRY_CUDA(cudaMemsetAsync(L.small, 0, 4 * sizeof(int32_t), s), "p2p_bin_points");
    k_keys<<<blocks_for(n, kThreads), kThreads, 0, s>>>(pts, n, lo[0], lo[1], lo[2], h, ng, L.keys, L.vals, L.small);
    P2P_CHECK_LAUNCH("p2p_bin_points/keys");
    bool in_alt = false;
    P2P_TRY_CUDA(radix_sort_pairs(L.keys, L.vals, L.keys_alt, L.vals_alt, n, 3 * ceil_log2(ng), L.radix_ws, s, &in_alt),
                 "p2p_bin_points/sort");
    const uint64_t* ks = in_alt ? L.keys_alt : L.keys;
    const int32_t* vs = in_alt ? L.vals_alt : L.vals;
    k_heads<<<blocks_for(n, kThreads), kThreads, 0, s>>>(ks, n, L.head);
    P2P_CHECK_LAUNCH("p2p_bin_points/heads");
    P2P_TRY_CUDA(scan_exclusive_i32(L.head, L.ex, n, L.small + 1, L.scan_ws, s), "p2p_bin_points/scan");
    k_rle<<<blocks_for(n, kThreads), kThreads, 0, s>>>(ks, vs, L.head, L.ex, n, perm, point_box, box_keys, box_ptr);
    P2P_CHECK_LAUNCH("p2p_bin_points/rle");
    int32_t host[2] = {0, 0};
    P2P_TRY_CUDA(cudaMemcpyAsync(host, L.small, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s), "p2p_bin_points");
    P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_bin_points");
    if (host[0]) return P2P_ERR_INVALID;
    *num_boxes = host[1];  // total of the head flags = number of non-empty boxes
    return P2P_OK;
}

P2P_API p2p_status p2p_neighbors_workspace_size(int32_t num_boxes, size_t* bytes) {
    if (!bytes || num_boxes < 0) return P2P_ERR_INVALID;
    *bytes = nbr_layout(num_boxes, nullptr).bytes;
    return P2P_OK;
}

}  // extern "C"

namespace {

// Neighbour CSR of nb target boxes over nbs source boxes (the same boxes for a one-set structure).
p2p_status build_neighbors(const int64_t* box_keys, int32_t num_boxes, const int64_t* src_keys,
                           const int32_t* src_box_ptr, int32_t num_src, int32_t ng, int32_t* nbr_ptr,
                           int32_t* nbr_idx, int32_t* nbr_self, int64_t* nnz, int64_t* sources, void* work,
                           size_t work_bytes, cudaStream_t s, bool two) {
    if (num_boxes < 0 || num_src < 0 || ng < 1 || ng > (1 << 21) || !nbr_ptr || !nnz || !sources)
        return P2P_ERR_INVALID;
    *nnz = 0;
    *sources = 0;
    if (num_boxes == 0) {
        P2P_TRY_CUDA(cudaMemsetAsync(nbr_ptr, 0, sizeof(int32_t), s), "p2p_build_neighbors");
        P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_build_neighbors");
        return P2P_OK;
    }
    if (!box_keys || !src_keys || !src_box_ptr || !nbr_idx || !work || ((uintptr_t)work & 255)) return P2P_ERR_INVALID;
    if (two && !nbr_self) return P2P_ERR_INVALID;
    if ((int64_t)num_boxes * 27 >= INT32_MAX) return P2P_ERR_UNSUPPORTED;
    NbrLayout L = nbr_layout(num_boxes, work);
    if (work_bytes < L.bytes) return P2P_ERR_WORKSPACE;
    P2P_TRY_CUDA(cudaMemsetAsync(L.bad, 0, 2 * sizeof(int32_t), s), "p2p_build_neighbors");
    P2P_TRY_CUDA(cudaMemsetAsync(L.sum, 0, sizeof(unsigned long long), s), "p2p_build_neighbors");
    const unsigned wblocks = blocks_for((int64_t)num_boxes * 32, kThreads);
    if (two) {
        if (num_src > 1) {
            k_keys_ascending<<<blocks_for(num_src, kThreads), kThreads, 0, s>>>(src_keys, num_src, L.bad);
            P2P_CHECK_LAUNCH("p2p_build_neighbors_st/keys");
        }
        k_neighbors<false, true><<<wblocks, kThreads, 0, s>>>(box_keys, num_boxes, src_keys, num_src, src_box_ptr, ng,
                                                              L.cnt, L.src_cnt, nullptr, nullptr, nullptr, L.bad);
    } else {
        k_neighbors<false, false><<<wblocks, kThreads, 0, s>>>(box_keys, num_boxes, src_keys, num_src, src_box_ptr, ng,
                                                               L.cnt, L.src_cnt, nullptr, nullptr, nullptr, L.bad);
    }
    P2P_CHECK_LAUNCH("p2p_build_neighbors/count");
    P2P_TRY_CUDA(scan_exclusive_i32(L.cnt, nbr_ptr, num_boxes, nbr_ptr + num_boxes, L.scan_ws, s),
                 "p2p_build_neighbors/scan");
    if (two)
        k_neighbors<true, true><<<wblocks, kThreads, 0, s>>>(box_keys, num_boxes, src_keys, num_src, src_box_ptr, ng,
                                                             nullptr, nullptr, nbr_ptr, nbr_idx, nbr_self, L.bad);
    else
        k_neighbors<true, false><<<wblocks, kThreads, 0, s>>>(box_keys, num_boxes, src_keys, num_src, src_box_ptr, ng,
                                                              nullptr, nullptr, nbr_ptr, nbr_idx, nullptr, L.bad);
    P2P_CHECK_LAUNCH("p2p_build_neighbors/fill");
    k_sum_i32<<<blocks_for(num_boxes, kThreads), kThreads, 0, s>>>(L.src_cnt, num_boxes, L.sum);
    P2P_CHECK_LAUNCH("p2p_build_neighbors/sum");
    int32_t bad = 0, total = 0;
    unsigned long long src = 0;
    P2P_TRY_CUDA(cudaMemcpyAsync(&bad, L.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "p2p_build_neighbors");
    P2P_TRY_CUDA(cudaMemcpyAsync(&total, nbr_ptr + num_boxes, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                 "p2p_build_neighbors");
    P2P_TRY_CUDA(cudaMemcpyAsync(&src, L.sum, sizeof(src), cudaMemcpyDeviceToHost, s), "p2p_build_neighbors");
    P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_build_neighbors");
    if (bad) return P2P_ERR_INVALID;
    *nnz = total;
    *sources = (int64_t)src;
    return P2P_OK;
}

// Entries of the repetition layout's records, sum over boxes of n_b (1 + S_b), from the box pointers and the
// neighbour lists copied to the host.
p2p_status repetition_records(const int32_t* box_ptr, int32_t nb, const int32_t* nbr_ptr, const int32_t* nbr_idx,
                              int64_t* records, cudaStream_t s) {
    *records = 0;
    if (nb <= 0) return P2P_OK;
    int32_t* hb = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nb + 1) * 2);
    if (!hb) return P2P_ERR_ALLOC;
    int32_t* hp = hb + nb + 1;
    cudaError_t e = cudaMemcpyAsync(hb, box_ptr, sizeof(int32_t) * ((size_t)nb + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hp, nbr_ptr, sizeof(int32_t) * ((size_t)nb + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int32_t* hi = nullptr;
    const int64_t nnz = e == cudaSuccess ? hp[nb] : 0;
    if (e == cudaSuccess && (nnz < 0 || nnz > 27ll * nb || hp[0] != 0)) {
        free(hb);
        return P2P_ERR_INVALID;
    }
    if (e == cudaSuccess && nnz > 0) {
        hi = (int32_t*)malloc(sizeof(int32_t) * (size_t)nnz);
        if (!hi) {
            free(hb);
            return P2P_ERR_ALLOC;
        }
        e = cudaMemcpyAsync(hi, nbr_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        free(hb);
        free(hi);
        set_cuda_error(e, "p2p_repetition_records");
        return P2P_ERR_CUDA;
    }
    int64_t total = 0;
    p2p_status st = P2P_OK;
    for (int32_t b = 0; b < nb && st == P2P_OK; ++b) {
        int64_t sb = 0;
        for (int32_t q = hp[b]; q < hp[b + 1]; ++q) {
            const int32_t c = hi[q];
            if (c < 0 || c >= nb) {
                st = P2P_ERR_INVALID;
                break;
            }
            sb += hb[c + 1] - hb[c];
        }
        total += (int64_t)(hb[b + 1] - hb[b]) * (1 + sb);
    }
    free(hb);
    free(hi);
    if (st != P2P_OK) return st;
    *records = total;
    return P2P_OK;
}

p2p_status plan_create(p2p_plan** plan, const PlanInput& in, p2p_kernel kernel, float k, p2p_layout layout,
                       int32_t max_nrhs, const p2p_tuning* tuning, void* workspace, size_t workspace_bytes,
                       cudaStream_t s) {
    if (!plan) return P2P_ERR_INVALID;
    *plan = nullptr;
    p2p_status st = check_sizes(in.n, in.nb, in.n_src, in.nbs, in.sources, layout, max_nrhs, in.two_sets);
    if (st != P2P_OK) return st;
    p2p_tuning t = resolve_tuning(tuning);
    if (!tuning_valid(t)) return P2P_ERR_INVALID;
    const int32_t nb = in.nb;
    const int64_t n = in.n;
    if (kernel != P2P_HELMHOLTZ && kernel != P2P_LAPLACE) return P2P_ERR_INVALID;
    if (!isfinite(k)) return P2P_ERR_INVALID;
    if ((n > 0 && nb < 1) || (n == 0 && nb != 0)) return P2P_ERR_INVALID;
    if ((in.n_src > 0 && in.nbs < 1) || (in.n_src == 0 && in.nbs != 0)) return P2P_ERR_INVALID;
    if (in.two_sets ? (in.nnz < 0 || in.nnz > 27ll * nb) : (in.nnz < nb || in.nnz > 27ll * nb))
        return P2P_ERR_INVALID;
    if (n > 0 && (!in.pts || !in.perm || !in.box_ptr || !in.nbr_ptr || (in.nnz > 0 && !in.nbr_idx)))
        return P2P_ERR_INVALID;
    if (in.two_sets && n > 0 && (!in.nbr_self || (in.n_src > 0 && (!in.src_pts || !in.src_perm || !in.src_box_ptr))))
        return P2P_ERR_INVALID;
    if (!workspace || ((uintptr_t)workspace & 255) || ((uintptr_t)in.pts & 3) || ((uintptr_t)in.src_pts & 3))
        return P2P_ERR_INVALID;
    int64_t records = 0;
    if (layout == P2P_LAYOUT_REPETITION) {
        const p2p_status rs = repetition_records(in.box_ptr, nb, in.nbr_ptr, in.nbr_idx, &records, s);
        if (rs != P2P_OK) return rs;
        if (records >= INT32_MAX) return P2P_ERR_UNSUPPORTED;
    }
    PlanLayout L = plan_layout(n, nb, in.n_src, in.nbs, in.two_sets, in.sources, in.nnz, layout, max_nrhs, t,
                               workspace, records);
    if (workspace_bytes < L.bytes) return P2P_ERR_WORKSPACE;
    p2p_plan* p = (p2p_plan*)malloc(sizeof(p2p_plan));
    if (!p) return P2P_ERR_ALLOC;
    *p = L.p;
    p->n = n;
    p->nb = nb;
    p->two_sets = in.two_sets ? 1 : 0;
    p->n_src = in.n_src;
    p->nbs = in.nbs;
    p->nnz = in.nnz;
    p->sources = in.sources;
    p->kernel = kernel;
    p->k = kernel == P2P_LAPLACE ? 0.f : k;
    p->layout = layout;
    p->max_nrhs = max_nrhs;
    p->tune = t;
    p->pts = in.pts;
    p->perm = in.perm;
    p->box_ptr = in.box_ptr;
    p->nbr_ptr = in.nbr_ptr;
    p->nbr_idx = in.nbr_idx;
    p->src_pts = in.src_pts;
    p->src_perm = in.src_perm;
    p->src_box_ptr = in.src_box_ptr;
    p->nbr_self = in.two_sets ? in.nbr_self : nullptr;
    p->n_items = 0;
    p->max_chunks = 0;
    p->max_box = 0;
    p->packed = 0;
    p->tc_wait_polls = -1;
    p->records = records;
#define FAIL_CUDA(expr, where)                 \
    do {                                       \
        cudaError_t e_ = (expr);               \
        if (e_ != cudaSuccess) {               \
            set_cuda_error(e_, where);         \
            free(p);                           \
            return P2P_ERR_CUDA;               \
        }                                      \
    } while (0)
    FAIL_CUDA(cudaMemsetAsync(p->status, 0, 4 * sizeof(unsigned int), s), "p2p_plan_create");
    if (n == 0) {
        FAIL_CUDA(cudaStreamSynchronize(s), "p2p_plan_create");
        *plan = p;
        return P2P_OK;
    }
    FAIL_CUDA(cudaMemsetAsync(L.maxes, 0, 4 * sizeof(int32_t), s), "p2p_plan_create");
    k_gather_xyz<<<blocks_for(n, kThreads), kThreads, 0, s>>>(in.pts, in.perm, n, p->xs);
    FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/gather");
    if (in.two_sets && in.n_src > 0) {
        k_gather_xyz<<<blocks_for(in.n_src, kThreads), kThreads, 0, s>>>(in.src_pts, in.src_perm, in.n_src, p->xs_src);
        FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/gather_sources");
    }
    const int upper = layout == P2P_LAYOUT_SYMMETRIC;
    auto box_info = [&]() {
        k_box_info<<<blocks_for(nb, kThreads), kThreads, 0, s>>>(in.box_ptr, p->src_box_ptr, p->nbs, in.nbr_ptr,
                                                                 in.nbr_idx, p->nbr_self, nb, in.nnz, t.chunk, upper,
                                                                 p->box_src, L.list_len, L.n_chunks, L.padded,
                                                                 L.self_len, L.maxes, p->status);
        return cudaGetLastError();
    };
    FAIL_CUDA(box_info(), "p2p_plan_create/box_info");
    if (tuning_is_auto(tuning)) {
        // When most source lists hold just over one default chunk (193 .. 256 sources), every box would get a
        // full item and a short tail item with the same fixed cost; 256-source items (6 warps per block, so two
        // blocks still fit an SM) give those boxes one item each.  When the whole plan has fewer than 2.5 items
        // per resident warp (16 per SM), the last items of the heaviest-first list leave most warps idle;
        // 128-source items spread it (measured on the 32 768-point cube, 8^3 boxes: 3 584 items of 192
        // sources 60.4 us, 5 400 of 128 51.2 us, of 96 52.2 us, of 64 59.4 us).  The workspace is sized for
        // the narrow chunk.
        int32_t counts[2] = {0, 0};  // tails, items
        int sms = 0, dev = 0;
        FAIL_CUDA(cudaGetDevice(&dev), "p2p_plan_create");
        FAIL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "p2p_plan_create");
        FAIL_CUDA(cudaMemcpyAsync(counts, L.maxes + 2, sizeof(counts), cudaMemcpyDeviceToHost, s), "p2p_plan_create");
        FAIL_CUDA(cudaStreamSynchronize(s), "p2p_plan_create");
        const p2p_tuning* sw = nullptr;
        if (2ll * counts[0] > nb) sw = &kWideTuning;
        else if (2ll * counts[1] < 5ll * 16 * sms) sw = &kNarrowTuning;
        if (sw) {
            t.chunk = sw->chunk;
            t.warps_per_cta = sw->warps_per_cta;
            p->tune = t;
            FAIL_CUDA(cudaMemsetAsync(L.maxes, 0, 4 * sizeof(int32_t), s), "p2p_plan_create");
            FAIL_CUDA(box_info(), "p2p_plan_create/box_info");
        }
    }
    FAIL_CUDA(scan_exclusive_i32(L.n_chunks, L.item_off, nb, L.small, L.scan_ws, s), "p2p_plan_create/scan");
    FAIL_CUDA(scan_exclusive_i32(L.padded, p->pk_off, nb, p->pk_off + nb, L.scan_ws, s),
              "p2p_plan_create/scan_lists");
    k_pack<<<blocks_for((int64_t)nb * 32, kThreads), kThreads, 0, s>>>(p->xs_src, p->src_perm, p->src_box_ptr,
                                                                      in.nbr_ptr, in.nbr_idx, p->nbr_self, p->pk_off,
                                                                      nb, upper, p->nb_src, p->pk_xyz, p->pk_src);
    FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/pack");
    if (layout == P2P_LAYOUT_REPETITION) {
        // per-target records (L.padded is free once the list offsets are scanned)
        k_rep_count<<<blocks_for(nb, kThreads), kThreads, 0, s>>>(in.box_ptr, p->box_src, nb, L.padded);
        FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/rep_count");
        FAIL_CUDA(scan_exclusive_i32(L.padded, p->rec_boff, nb, p->rec_boff + nb, L.scan_ws, s),
                  "p2p_plan_create/rep_scan");
        k_rep_fill<<<blocks_for((int64_t)nb * 32, kThreads), kThreads, 0, s>>>(
            p->xs, in.perm, in.box_ptr, p->box_src, p->pk_off, p->nb_src, p->rec_boff, nb, n, p->rec_off, p->rec_xyz,
            p->rec_src);
        FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/rep_fill");
    }
    k_item_records<<<blocks_for(nb, kThreads), kThreads, 0, s>>>(L.n_chunks, L.item_off, in.box_ptr, L.list_len,
                                                                 L.self_len, p->pk_off, nb, t.chunk, t.target_group,
                                                                 p->two_sets, L.recs, L.keys, L.vals);
    FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/items");
    if (p->tc_gstart && p->nbs > 0) {
        // 16-source groups of the tensor-core path over the source boxes (n_chunks is free once the items are
        // built), then every target box's list of its neighbourhood's groups
        k_tc_groups<<<blocks_for(p->nbs, kThreads), kThreads, 0, s>>>(p->src_box_ptr, p->nbs, L.n_chunks);
        FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/tc_groups");
        FAIL_CUDA(scan_exclusive_i32(L.n_chunks, p->tc_gstart, p->nbs, p->tc_gstart + p->nbs, L.scan_ws, s),
                  "p2p_plan_create/tc_scan");
        k_tc_list_len<<<blocks_for(nb, kThreads), kThreads, 0, s>>>(in.nbr_ptr, in.nbr_idx, p->tc_gstart, nb,
                                                                    p->tc_gcount, L.n_chunks);
        FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/tc_lists");
        FAIL_CUDA(scan_exclusive_i32(L.n_chunks, p->tc_glist_off, nb, p->tc_glist_off + nb, L.scan_ws, s),
                  "p2p_plan_create/tc_scan");
        k_tc_list_fill<<<blocks_for(nb, kThreads), kThreads, 0, s>>>(in.nbr_ptr, in.nbr_idx, p->tc_gstart,
                                                                     p->tc_glist_off, nb, p->tc_glist);
        FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/tc_lists");
    }
    int32_t host[4] = {0, 0, 0, 0};
    unsigned int status = 0;
    int32_t packed = 0;
    int32_t tc_groups = 0;
    FAIL_CUDA(cudaMemcpyAsync(host, L.maxes, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s), "p2p_plan_create");
    FAIL_CUDA(cudaMemcpyAsync(host + 2, L.small, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "p2p_plan_create");
    FAIL_CUDA(cudaMemcpyAsync(&status, p->status, sizeof(status), cudaMemcpyDeviceToHost, s), "p2p_plan_create");
    FAIL_CUDA(cudaMemcpyAsync(&packed, p->pk_off + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
              "p2p_plan_create");
    if (p->tc_gstart && p->nbs > 0)
        FAIL_CUDA(cudaMemcpyAsync(&tc_groups, p->tc_gstart + p->nbs, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                  "p2p_plan_create");
    FAIL_CUDA(cudaStreamSynchronize(s), "p2p_plan_create");
    if (!status) {
        const int64_t items = host[2];
        bool in_alt = false;
        FAIL_CUDA(radix_sort_pairs(L.keys, L.vals, L.keys_alt, L.vals_alt, items, 32, L.radix_ws, s, &in_alt),
                  "p2p_plan_create/sort");
        if (items > 0) {
            k_item_gather<<<blocks_for(items, kThreads), kThreads, 0, s>>>(L.recs, in_alt ? L.vals_alt : L.vals,
                                                                           items, p->items);
            FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/order");
        }
        FAIL_CUDA(cudaStreamSynchronize(s), "p2p_plan_create");
    }
    if (status) {
        free(p);
        return P2P_ERR_INVALID;
    }
    // direct kernel: one item per target box (the item-sort scratch is free again)
    p->direct_k = 0;
    if (layout != P2P_LAYOUT_SYMMETRIC && layout != P2P_LAYOUT_REPETITION) {
        const int32_t wb = t.warp_boxes == 0 ? auto_warp_boxes(n, nb) : t.warp_boxes;
        p->tune.warp_boxes = wb;
        if (wb > 0) {
            p->direct_k = wb;
            k_direct_items<<<blocks_for(nb, kThreads), kThreads, 0, s>>>(in.box_ptr, L.list_len, L.self_len, p->pk_off,
                                                                         nb, 32 / wb, L.recs, L.keys, L.vals);
            FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/direct_items");
            bool in_alt = false;
            FAIL_CUDA(radix_sort_pairs(L.keys, L.vals, L.keys_alt, L.vals_alt, nb, 32, L.radix_ws, s, &in_alt),
                      "p2p_plan_create/direct_sort");
            k_item_gather<<<blocks_for(nb, kThreads), kThreads, 0, s>>>(L.recs, in_alt ? L.vals_alt : L.vals, nb,
                                                                        p->ditems);
            FAIL_CUDA(cudaGetLastError(), "p2p_plan_create/direct_order");
            FAIL_CUDA(cudaStreamSynchronize(s), "p2p_plan_create");
        }
    } else {
        p->tune.warp_boxes = -1;
    }
    // box-group kernel (indexed layout): groups of consecutive target boxes staging the union of their
    // neighbourhoods; a plan whose largest union does not fit the kernel's buffer keeps the staged pipeline
    p->group_k = 0;
    p->n_groups = 0;
    p->group_cap = 0;
    p->group_pos_cap = 0;
    if (p->tune.warp_boxes == -2 && (layout != P2P_LAYOUT_INDEXED || nb == 0)) p->tune.warp_boxes = -1;
    if (p->tune.warp_boxes == -2) {
        p->n_groups = (nb + kGroupBoxes - 1) / kGroupBoxes;
        int32_t cap[2] = {0, 0};
        FAIL_CUDA(p2p_group_build(p, in.nbr_ptr, in.nbr_idx, L.keys, L.vals, L.keys_alt, L.vals_alt, L.radix_ws,
                                  L.maxes, s, cap),
                  "p2p_plan_create/groups");
        if (cap[0] > 0 && cap[0] <= kGroupCapMax) {
            p->group_k = 1;
            p->group_cap = (cap[0] + 3) & ~3;
            p->group_pos_cap = cap[1];
        } else {
            p->tune.warp_boxes = -1;
        }
    }
    p->max_chunks = host[0];
    p->max_box = host[1];
    p->n_items = host[2];
    p->packed = packed;
    p->tc_groups = tc_groups;
    FAIL_CUDA(p2p_pair_configure(p), "p2p_plan_create/occupancy");
#undef FAIL_CUDA
    *plan = p;
    return P2P_OK;
}

}  // namespace

extern "C" {

P2P_API p2p_status p2p_build_neighbors(const int64_t* box_keys, const int32_t* box_ptr, int32_t num_boxes,
                                       int32_t ng, int32_t* nbr_ptr, int32_t* nbr_idx, int64_t* nnz,
                                       int64_t* sources, void* work, size_t work_bytes, p2p_stream_t stream) {
    return build_neighbors(box_keys, num_boxes, box_keys, box_ptr, num_boxes, ng, nbr_ptr, nbr_idx, nullptr, nnz,
                           sources, work, work_bytes, (cudaStream_t)stream, false);
}

P2P_API p2p_status p2p_build_neighbors_st(const int64_t* tgt_keys, int32_t num_tgt_boxes, const int64_t* src_keys,
                                          const int32_t* src_box_ptr, int32_t num_src_boxes, int32_t ng,
                                          int32_t* nbr_ptr, int32_t* nbr_idx, int32_t* nbr_self, int64_t* nnz,
                                          int64_t* sources, void* work, size_t work_bytes, p2p_stream_t stream) {
    if (num_src_boxes == 0 && num_tgt_boxes > 0) {
        // no sources: every list is empty
        if (!nbr_ptr || !nbr_self || !nnz || !sources) return P2P_ERR_INVALID;
        cudaStream_t s = (cudaStream_t)stream;
        *nnz = 0;
        *sources = 0;
        P2P_TRY_CUDA(cudaMemsetAsync(nbr_ptr, 0, sizeof(int32_t) * ((size_t)num_tgt_boxes + 1), s),
                     "p2p_build_neighbors_st");
        P2P_TRY_CUDA(cudaMemsetAsync(nbr_self, 0xff, sizeof(int32_t) * (size_t)num_tgt_boxes, s),
                     "p2p_build_neighbors_st");
        P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_build_neighbors_st");
        return P2P_OK;
    }
    return build_neighbors(tgt_keys, num_tgt_boxes, src_keys, src_box_ptr, num_src_boxes, ng, nbr_ptr, nbr_idx,
                           nbr_self, nnz, sources, work, work_bytes, (cudaStream_t)stream, true);
}

P2P_API p2p_status p2p_plan_workspace_size(int64_t n, int32_t num_boxes, int64_t nnz, int64_t sources,
                                           p2p_layout layout, int32_t max_nrhs, const p2p_tuning* tuning,
                                           size_t* bytes) {
    if (!bytes) return P2P_ERR_INVALID;
    if (layout == P2P_LAYOUT_REPETITION) return P2P_ERR_INVALID;  // its records: p2p_plan_workspace_size_rep
    p2p_status st = check_sizes(n, num_boxes, n, num_boxes, sources, layout, max_nrhs, false);
    if (st != P2P_OK) return st;
    p2p_tuning t = resolve_tuning(tuning);
    if (!tuning_valid(t)) return P2P_ERR_INVALID;
    *bytes = plan_layout(n, num_boxes, n, num_boxes, false, sources, nnz, layout, max_nrhs, t, nullptr).bytes;
    return P2P_OK;
}

P2P_API p2p_status p2p_repetition_records(const int32_t* box_ptr, int32_t num_boxes, const int32_t* nbr_ptr,
                                          const int32_t* nbr_idx, int64_t* records, p2p_stream_t stream) {
    if (!records || num_boxes < 0 || (num_boxes > 0 && (!box_ptr || !nbr_ptr || !nbr_idx))) return P2P_ERR_INVALID;
    return repetition_records(box_ptr, num_boxes, nbr_ptr, nbr_idx, records, (cudaStream_t)stream);
}

P2P_API p2p_status p2p_plan_workspace_size_rep(int64_t n, int32_t num_boxes, int64_t nnz, int64_t sources,
                                               int64_t records, const p2p_tuning* tuning, size_t* bytes) {
    if (!bytes || records < 0 || records >= INT32_MAX) return P2P_ERR_INVALID;
    p2p_status st = check_sizes(n, num_boxes, n, num_boxes, sources, P2P_LAYOUT_REPETITION, 1, false);
    if (st != P2P_OK) return st;
    p2p_tuning t = resolve_tuning(tuning);
    if (!tuning_valid(t)) return P2P_ERR_INVALID;
    *bytes = plan_layout(n, num_boxes, n, num_boxes, false, sources, nnz, P2P_LAYOUT_REPETITION, 1, t, nullptr, records)
                 .bytes;
    return P2P_OK;
}

P2P_API p2p_status p2p_plan_workspace_size_st(int64_t n_tgt, int32_t num_tgt_boxes, int64_t n_src,
                                              int32_t num_src_boxes, int64_t nnz, int64_t sources, p2p_layout layout,
                                              int32_t max_nrhs, const p2p_tuning* tuning, size_t* bytes) {
    if (!bytes) return P2P_ERR_INVALID;
    p2p_status st = check_sizes(n_tgt, num_tgt_boxes, n_src, num_src_boxes, sources, layout, max_nrhs, true);
    if (st != P2P_OK) return st;
    p2p_tuning t = resolve_tuning(tuning);
    if (!tuning_valid(t)) return P2P_ERR_INVALID;
    *bytes = plan_layout(n_tgt, num_tgt_boxes, n_src, num_src_boxes, true, sources, nnz, layout, max_nrhs, t, nullptr)
                 .bytes;
    return P2P_OK;
}

P2P_API p2p_status p2p_plan_create(p2p_plan** plan, const float* pts, int64_t n, const int32_t* perm,
                                   const int32_t* box_ptr, int32_t num_boxes, const int32_t* nbr_ptr,
                                   const int32_t* nbr_idx, int64_t nnz, int64_t sources, p2p_kernel kernel, float k,
                                   p2p_layout layout, int32_t max_nrhs, const p2p_tuning* tuning, void* workspace,
                                   size_t workspace_bytes, p2p_stream_t stream) {
    PlanInput in{pts, n, perm, box_ptr, num_boxes, pts, n, perm, box_ptr, num_boxes, nbr_ptr, nbr_idx, nullptr,
                 nnz, sources, false};
    return plan_create(plan, in, kernel, k, layout, max_nrhs, tuning, workspace, workspace_bytes,
                       (cudaStream_t)stream);
}

P2P_API p2p_status p2p_plan_create_st(p2p_plan** plan, const float* tgt_pts, int64_t n_tgt, const int32_t* tgt_perm,
                                      const int32_t* tgt_box_ptr, int32_t num_tgt_boxes, const float* src_pts,
                                      int64_t n_src, const int32_t* src_perm, const int32_t* src_box_ptr,
                                      int32_t num_src_boxes, const int32_t* nbr_ptr, const int32_t* nbr_idx,
                                      const int32_t* nbr_self, int64_t nnz, int64_t sources, p2p_kernel kernel,
                                      float k, p2p_layout layout, int32_t max_nrhs, const p2p_tuning* tuning,
                                      void* workspace, size_t workspace_bytes, p2p_stream_t stream) {
    PlanInput in{tgt_pts, n_tgt, tgt_perm, tgt_box_ptr, num_tgt_boxes, src_pts, n_src, src_perm, src_box_ptr,
                 num_src_boxes, nbr_ptr, nbr_idx, nbr_self, nnz, sources, true};
    return plan_create(plan, in, kernel, k, layout, max_nrhs, tuning, workspace, workspace_bytes,
                       (cudaStream_t)stream);
}

P2P_API p2p_status p2p_plan_destroy(p2p_plan* plan) {
    free(plan);
    return P2P_OK;
}

P2P_API p2p_status p2p_plan_info(const p2p_plan* plan, int64_t* n, int32_t* num_boxes, int64_t* sources,
                                 int64_t* work_items, p2p_layout* layout, p2p_tuning* tuning) {
    if (!plan) return P2P_ERR_INVALID;
    if (n) *n = plan->n;
    if (num_boxes) *num_boxes = plan->nb;
    if (sources) *sources = plan->sources;
    if (work_items) *work_items = plan->n_items;
    if (layout) *layout = plan->layout;
    if (tuning) *tuning = plan->tune;
    return P2P_OK;
}

P2P_API p2p_status p2p_plan_pair_count(const p2p_plan* plan, int64_t* pairs, p2p_stream_t stream) {
    if (!plan || !pairs) return P2P_ERR_INVALID;
    *pairs = 0;
    if (plan->n == 0) return P2P_OK;
    cudaStream_t s = (cudaStream_t)stream;
    P2P_TRY_CUDA(cudaMemsetAsync(plan->scratch64, 0, sizeof(long long), s), "p2p_plan_pair_count");
    k_pair_count<<<blocks_for((int64_t)plan->nb * 32, kThreads), kThreads, 0, s>>>(
        plan->xs, plan->box_ptr, plan->xs_src, plan->src_box_ptr, plan->nbr_ptr, plan->nbr_idx, plan->nbr_self,
        plan->box_src, plan->nb, (unsigned long long*)plan->scratch64);
    P2P_CHECK_LAUNCH("p2p_plan_pair_count");
    long long v = 0;
    P2P_TRY_CUDA(cudaMemcpyAsync(&v, plan->scratch64, sizeof(v), cudaMemcpyDeviceToHost, s), "p2p_plan_pair_count");
    P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_plan_pair_count");
    *pairs = v;
    return P2P_OK;
}

P2P_API p2p_status p2p_plan_update_points(p2p_plan* plan, const float* pts, const double lo[3], double h, int32_t ng,
                                          int64_t* moved, p2p_stream_t stream) {
    if (moved) *moved = 0;
    if (!plan || !lo || !(h > 0.0) || !isfinite(h) || ng < 1 || ng > (1 << 21)) return P2P_ERR_INVALID;
    if (!isfinite(lo[0]) || !isfinite(lo[1]) || !isfinite(lo[2])) return P2P_ERR_INVALID;
    if (plan->two_sets) return P2P_ERR_UNSUPPORTED;
    if (plan->n == 0) return P2P_OK;
    if (!pts || ((uintptr_t)pts & 3)) return P2P_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    // scratch64[0]: moved count, scratch64[1]: non-finite flag (the pair count's slot, free between calls)
    P2P_TRY_CUDA(cudaMemsetAsync(plan->scratch64, 0, 2 * sizeof(long long), s), "p2p_plan_update_points");
    k_moved<<<blocks_for(plan->n, kThreads), kThreads, 0, s>>>(pts, plan->perm, plan->xs, plan->n, lo[0], lo[1], lo[2],
                                                               h, ng, (unsigned long long*)plan->scratch64,
                                                               (int32_t*)(plan->scratch64 + 1));
    P2P_CHECK_LAUNCH("p2p_plan_update_points/check");
    long long host[2] = {0, 0};
    P2P_TRY_CUDA(cudaMemcpyAsync(host, plan->scratch64, sizeof(host), cudaMemcpyDeviceToHost, s),
                 "p2p_plan_update_points");
    P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_plan_update_points");
    if (host[1]) return P2P_ERR_INVALID;
    if (moved) *moved = host[0];
    if (host[0]) return P2P_ERR_STALE;
    k_gather_xyz<<<blocks_for(plan->n, kThreads), kThreads, 0, s>>>(pts, plan->perm, plan->n, plan->xs);
    P2P_CHECK_LAUNCH("p2p_plan_update_points/gather");
    if (plan->pk_xyz && plan->packed > 0) {
        k_repack_xyz<<<blocks_for(plan->packed, kThreads), kThreads, 0, s>>>(plan->xs, plan->nb_src, plan->packed,
                                                                             plan->pk_xyz);
        P2P_CHECK_LAUNCH("p2p_plan_update_points/repack");
    }
    plan->pts = pts;
    plan->src_pts = pts;
    P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_plan_update_points");
    return P2P_OK;
}

P2P_API p2p_status p2p_last_async_status(const p2p_plan* plan, p2p_stream_t stream) {
    if (!plan) return P2P_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int v = 0;
    P2P_TRY_CUDA(cudaMemcpyAsync(&v, plan->status, sizeof(v), cudaMemcpyDeviceToHost, s), "p2p_last_async_status");
    P2P_TRY_CUDA(cudaMemsetAsync(plan->status, 0, sizeof(unsigned int), s), "p2p_last_async_status");
    P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_last_async_status");
    if (v & P2P_DEV_TIMEOUT) return P2P_ERR_TIMEOUT;
    if (v & P2P_DEV_BAD_INPUT) return P2P_ERR_INVALID;
    if (v & P2P_DEV_TC_FAULTED) return P2P_ERR_UNSUPPORTED;
    return P2P_OK;
}

}  // extern "C"
