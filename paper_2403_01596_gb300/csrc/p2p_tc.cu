// Multi-RHS P2P on the 5th-generation tensor cores (tcgen05, TMEM accumulator).
//
// For one target box b and a group of at most 64 of its targets, the complex
// product out[t, r] = sum_s G(x_t, y_s) lambda[s, r] over the box's
// neighbourhood is computed as one real GEMM per 32-source stage,
//
//     D[128 x N] += A[128 x 64] . B[64 x N],
//     A[2t, 2s] = Re G, A[2t, 2s+1] = -Im G, A[2t+1, 2s] = Im G, A[2t+1, 2s+1] = Re G,
//     B[2s, r] = Re lambda[s, r],  B[2s+1, r] = Im lambda[s, r],
//
// so that D[2t, r] = Re out[t, r] and D[2t+1, r] = Im out[t, r].  The G tile is
// formed on the CUDA cores (rsqrt, sincos in FP32), both operands are split
// x = hi + lo into BF16, and three MMAs per K = 16 slice (hi.hi + hi.lo + lo.hi,
// kind::f16, FP32 accumulate in TMEM) keep the product error near 2^-17.  Two
// shared-memory stages alternate: CUDA cores fill one while the tensor core
// reads the other; tcgen05.commit on an mbarrier releases a stage.  Every wait
// is bounded: a wait that runs out sets the plan's status word and the CTA
// drains its MMAs (again bounded), frees its TMEM and returns.
//
// Operands use the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices, K-adjacent cores 128 bytes apart (leading byte offset) and
// 8-row groups kCoreStride bytes apart (stride byte offset; 1024 + 16 so that
// the 16-byte stores of eight consecutive rows hit distinct bank groups).
#include <cuda_bf16.h>
#include <math.h>

#include "p2p_internal.cuh"

using namespace p2p_detail;

namespace {

constexpr float kInv4Pi = 0.0795774715459476679f;
constexpr int kTcThreads = 128;
constexpr int kTcTargets = 64;        // targets per CTA (128 accumulator rows)
constexpr int kTcStageSrc = 32;       // sources per stage (K = 64)
constexpr int kCoreStride = 1040;     // bytes between 8-row core groups
constexpr int kATile = 16 * kCoreStride;
constexpr uint32_t kWaitLimit = 1u << 24;

__host__ __device__ inline int b_tile_bytes(int np) { return (np / 8) * kCoreStride; }
__host__ __device__ inline int stage_bytes(int np) { return 2 * kATile + 2 * b_tile_bytes(np); }
constexpr int kExtraBytes = 64 * 16 + 32 * 16 + 32 * 4 + 64 * 4 + 2 * 8 + 16;
__host__ __device__ inline int tc_smem_bytes(int np) { return 2 * stage_bytes(np) + kExtraBytes; }

// --------------------------------------------------------------- PTX helpers --

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading and stride byte offsets (>> 4),
// descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N, M = 128.
__host__ __device__ inline uint32_t idesc_bf16_f32(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 16 consecutive 32-bit columns of TMEM into registers.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo with hi, lo BF16 (round to nearest).
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    float2 hf = __bfloat1622float2(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

// Splits 8 floats (one 16-byte core-matrix row) and stores hi and lo rows.
__device__ __forceinline__ void store_split8(unsigned char* hi_base, unsigned char* lo_base, int off,
                                             const float (&v)[8]) {
    uint4 h, l;
    split2(v[0], v[1], h.x, l.x);
    split2(v[2], v[3], h.y, l.y);
    split2(v[4], v[5], h.z, l.z);
    split2(v[6], v[7], h.w, l.w);
    *reinterpret_cast<uint4*>(hi_base + off) = h;
    *reinterpret_cast<uint4*>(lo_base + off) = l;
}

__device__ __forceinline__ int core_off(int row, int kc) { return (row >> 3) * kCoreStride + kc * 128 + (row & 7) * 16; }

// Issues the three MMAs of every K = 16 slice of one stage (single thread).
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                            uint32_t idesc, bool first) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ah = smem_desc(a_hi + kk * 256, 128, kCoreStride);
        const uint64_t al = smem_desc(a_lo + kk * 256, 128, kCoreStride);
        const uint64_t bh = smem_desc(b_hi + kk * 256, 128, kCoreStride);
        const uint64_t bl = smem_desc(b_lo + kk * 256, 128, kCoreStride);
        mma_bf16(tmem, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
        mma_bf16(tmem, ah, bl, idesc, 1u);
        mma_bf16(tmem, al, bh, idesc, 1u);
    }
}

struct TcArgs {
    const float4* xs;
    const float2* lam;     // box-sorted strengths, row stride nrhs
    const int32_t* box_ptr;
    const int32_t* nbr_ptr;
    const int32_t* nbr_idx;
    const int32_t* box_src;
    const int32_t* perm;
    float2* out;
    int64_t ld;
    int32_t nrhs;
    int32_t np;            // nrhs rounded up to a multiple of 16 (MMA N)
    int32_t nacc;          // TMEM accumulators the stages rotate over (1, 2 or 4)
    int32_t tmem_cols;
    int32_t laplace;
    float k;
    unsigned int* status;
};

struct TcSmem {
    unsigned char* stage[2];
    float4* tx;
    float4* sx;
    int* sj;
    int* seg;
    uint64_t* bars;
    uint32_t* tmem_slot;
    int* flag;
};

__device__ __forceinline__ TcSmem carve(unsigned char* smem, int np) {
    TcSmem s;
    const int sb = stage_bytes(np);
    s.stage[0] = smem;
    s.stage[1] = smem + sb;
    unsigned char* e = smem + 2 * sb;
    s.tx = reinterpret_cast<float4*>(e);
    s.sx = s.tx + 64;
    s.sj = reinterpret_cast<int*>(s.sx + 32);
    s.seg = s.sj + 32;
    s.bars = reinterpret_cast<uint64_t*>(s.seg + 64);
    s.tmem_slot = reinterpret_cast<uint32_t*>(s.bars + 2);
    s.flag = reinterpret_cast<int*>(s.tmem_slot + 1);
    return s;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_p2p_tc(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x;
    const int tb = a.box_ptr[b];
    const int nt_all = a.box_ptr[b + 1] - tb;
    const int t0 = blockIdx.y * kTcTargets;
    if (t0 >= nt_all) return;  // uniform over the CTA
    const int nt = min(kTcTargets, nt_all - t0);
    const int S = a.box_src[b];
    const int nstages = (S + kTcStageSrc - 1) / kTcStageSrc;
    const int np = a.np;
    TcSmem sm = carve(smem, np);
    const int e0 = a.nbr_ptr[b];
    const int ne = a.nbr_ptr[b + 1] - e0;

    if (warp == 0) tmem_alloc(sm.tmem_slot, (uint32_t)a.tmem_cols);
    if (tid == 0) {
        mbar_init(&sm.bars[0], 1);
        mbar_init(&sm.bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *sm.flag = 0;
    }
    if (warp == 1) {
        int start = 0, len = 0;
        if (lane < ne) {
            const int c = a.nbr_idx[e0 + lane];
            start = a.box_ptr[c];
            len = a.box_ptr[c + 1] - start;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(P2P_FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        sm.seg[lane] = incl - len;
        sm.seg[32 + lane] = start;
    }
    if (tid < kTcTargets) sm.tx[tid] = tid < nt ? a.xs[tb + t0 + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_slot;
    const uint32_t idesc = idesc_bf16_f32(np);
    const float k = a.k;

    bool failed = false;
    int committed = 0;  // stages whose MMAs were issued and committed
    for (int st = 0; st < nstages; ++st) {
        const int bi = st & 1;
        unsigned char* A_hi = sm.stage[bi];
        unsigned char* A_lo = A_hi + kATile;
        unsigned char* B_hi = A_lo + kATile;
        unsigned char* B_lo = B_hi + b_tile_bytes(np);
        if (st >= 2 && !mbar_wait(&sm.bars[bi], (uint32_t)(((st >> 1) - 1) & 1))) *sm.flag = 1;
        const int p0 = st * kTcStageSrc;
        const int ns = min(kTcStageSrc, S - p0);
        if (tid < kTcStageSrc) {
            if (tid < ns) {
                const int pp = p0 + tid;
                int lo = 0, hi = ne - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sm.seg[mid] <= pp) lo = mid;
                    else hi = mid - 1;
                }
                const int j = sm.seg[32 + lo] + (pp - sm.seg[lo]);
                sm.sj[tid] = j;
                sm.sx[tid] = a.xs[j];
            } else {
                sm.sj[tid] = -1;
                sm.sx[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        if (*sm.flag) {
            failed = true;
            break;
        }
        // B: warp w fills source quads w and w + 4; lanes run over right-hand sides
#pragma unroll
        for (int qi = 0; qi < 2; ++qi) {
            const int kc = warp + 4 * qi;
            int js[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) js[u] = sm.sj[4 * kc + u];
            for (int r = lane; r < np; r += 32) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float2 l = make_float2(0.f, 0.f);
                    if (js[u] >= 0 && r < a.nrhs) l = a.lam[(int64_t)js[u] * a.nrhs + r];
                    v[2 * u] = l.x;
                    v[2 * u + 1] = l.y;
                }
                store_split8(B_hi, B_lo, core_off(r, kc), v);
            }
        }
        // A: thread -> target t, half of the stage's sources (4 quads)
        {
            const int t = tid & 63, half = tid >> 6;
            const float4 x = sm.tx[t];
            const bool tvalid = t < nt;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kc = 4 * half + q;
                float re_row[8], im_row[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int s = 4 * kc + u;
                    const float4 p = sm.sx[s];
                    const float dx = p.x - x.x, dy = p.y - x.y, dz = p.z - x.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    float inv = rsqrtf(r2);
                    inv = (r2 > 0.f && tvalid && s < ns) ? inv : 0.f;
                    float gr, gi;
                    if (a.laplace) {
                        gr = inv;
                        gi = 0.f;
                    } else {
                        float sn, cs;
                        __sincosf(k * (r2 * inv), &sn, &cs);
                        gr = cs * inv;
                        gi = sn * inv;
                    }
                    re_row[2 * u] = gr;
                    re_row[2 * u + 1] = -gi;
                    im_row[2 * u] = gi;
                    im_row[2 * u + 1] = gr;
                }
                const int off = core_off(2 * t, kc);
                store_split8(A_hi, A_lo, off, re_row);
                store_split8(A_hi, A_lo, off + 16, im_row);
            }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            // stage st accumulates into accumulator st % nacc: shorter accumulation chains
            const uint32_t acc = tmem + (uint32_t)((st % a.nacc) * np);
            issue_stage(acc, smem_u32(A_hi), smem_u32(A_lo), smem_u32(B_hi), smem_u32(B_lo), idesc, st < a.nacc);
            mma_commit(&sm.bars[bi]);
        }
        committed = st + 1;
    }

    // wait for the last stage (all earlier MMAs complete before it)
    if (!failed && nstages > 0) {
        const int last = nstages - 1;
        if (!mbar_wait(&sm.bars[last & 1], (uint32_t)((last >> 1) & 1))) *sm.flag = 1;
    }
    __syncthreads();
    failed = failed || (*sm.flag != 0);
    if (failed) {
        if (tid == 0) atomicOr(a.status, P2P_DEV_TIMEOUT | P2P_DEV_TC_FAULTED);
        // drain: bounded waits for the last committed stage of each barrier
        if (tid == 0) {
            for (int st = committed - 2; st < committed; ++st)
                if (st >= 0) mbar_wait(&sm.bars[st & 1], (uint32_t)((st >> 1) & 1));
        }
    } else {
        tc_fence_after();
        const int m = warp * 32 + lane;  // accumulator row of this lane
        const int t = m >> 1;
        const bool odd = (m & 1) != 0;
        const bool write = t < nt;
        const int64_t row = write ? (int64_t)a.perm[tb + t0 + t] * a.ld : 0;
        const int used = min(a.nacc, nstages);
        for (int c0 = 0; c0 < np; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            for (int q = 1; q < used; ++q) {
                float w[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * np + c0), w);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += w[i];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float x = __shfl_xor_sync(P2P_FULL_MASK, odd ? v[i] : v[8 + i], 1);
                const int r = c0 + (odd ? 8 : 0) + i;
                if (write && r < a.nrhs) {
                    const float2 o = odd ? make_float2(x * kInv4Pi, v[8 + i] * kInv4Pi)
                                         : make_float2(v[i] * kInv4Pi, x * kInv4Pi);
                    a.out[row + r] = o;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// ------------------------------------------------- operand-layout self-check --

// D[128 x N] = A[128 x K] . B[N x K]^T with A, B split into BF16 hi + lo (3 MMAs
// per K = 16 slice), through the same descriptors and stage layout as k_p2p_tc.
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_gemm_check(const float* __restrict__ A,
                                                                 const float* __restrict__ B, float* __restrict__ D,
                                                                 int K, int np, int tmem_cols,
                                                                 unsigned int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    TcSmem sm = carve(smem, np);
    if (warp == 0) tmem_alloc(sm.tmem_slot, (uint32_t)tmem_cols);
    if (tid == 0) {
        mbar_init(&sm.bars[0], 1);
        mbar_init(&sm.bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_slot;
    const uint32_t idesc = idesc_bf16_f32(np);
    const int nstages = K / 64;
    bool ok = true;
    int committed = 0;
    for (int st = 0; st < nstages && ok; ++st) {
        const int bi = st & 1;
        unsigned char* A_hi = sm.stage[bi];
        unsigned char* A_lo = A_hi + kATile;
        unsigned char* B_hi = A_lo + kATile;
        unsigned char* B_lo = B_hi + b_tile_bytes(np);
        if (st >= 2) ok = mbar_wait(&sm.bars[bi], (uint32_t)(((st >> 1) - 1) & 1));
        ok = __syncthreads_and(ok);
        if (!ok) break;
        for (int c = tid; c < 128 * 8; c += kTcThreads) {
            const int row = c >> 3, kc = c & 7;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = A[(int64_t)row * K + st * 64 + kc * 8 + i];
            store_split8(A_hi, A_lo, core_off(row, kc), v);
        }
        for (int c = tid; c < np * 8; c += kTcThreads) {
            const int row = c >> 3, kc = c & 7;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = B[(int64_t)row * K + st * 64 + kc * 8 + i];
            store_split8(B_hi, B_lo, core_off(row, kc), v);
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue_stage(tmem, smem_u32(A_hi), smem_u32(A_lo), smem_u32(B_hi), smem_u32(B_lo), idesc, st == 0);
            mma_commit(&sm.bars[bi]);
        }
        committed = st + 1;
    }
    if (ok && nstages > 0) ok = mbar_wait(&sm.bars[(nstages - 1) & 1], (uint32_t)(((nstages - 1) >> 1) & 1));
    ok = __syncthreads_and(ok);
    if (ok) {
        tc_fence_after();
        for (int c0 = 0; c0 < np; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(int64_t)(warp * 32 + lane) * np + c0 + i] = v[i];
        }
    } else if (tid == 0) {
        atomicOr(status, P2P_DEV_TIMEOUT);
        for (int st = committed - 2; st < committed; ++st)
            if (st >= 0) mbar_wait(&sm.bars[st & 1], (uint32_t)((st >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)tmem_cols);
}

int tmem_cols_for(int np) {
    int c = 32;
    while (c < np) c <<= 1;
    return c;
}

}  // namespace

bool p2p_tc_supported(const p2p_plan* plan, int32_t nrhs) {
    if (!plan || nrhs < 1 || nrhs > 256) return false;
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return false;
    return major == 10 && minor == 3;
}

p2p_status p2p_apply_tc(const p2p_plan* plan, const float2* lam_sorted, float2* out, int32_t nrhs, int64_t ld,
                        int32_t adjoint, cudaStream_t s) {
    if (plan->n == 0) return P2P_OK;
    TcArgs a;
    a.xs = plan->xs;
    a.lam = lam_sorted;
    a.box_ptr = plan->box_ptr;
    a.nbr_ptr = plan->nbr_ptr;
    a.nbr_idx = plan->nbr_idx;
    a.box_src = plan->box_src;
    a.perm = plan->perm;
    a.out = out;
    a.ld = ld;
    a.nrhs = nrhs;
    a.np = (nrhs + 15) / 16 * 16;
    const int smem_needed = tc_smem_bytes(a.np);
    int max_smem = 0, dev = 0;
    P2P_TRY_CUDA(cudaGetDevice(&dev), "p2p_apply_tc");
    P2P_TRY_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev), "p2p_apply_tc");
    const int ctas_per_sm = max(1, max_smem / (smem_needed + 1024));
    // up to four accumulators while the co-resident CTAs' TMEM fits in 512 columns
    a.nacc = 4;
    while (a.nacc > 1 && ctas_per_sm * tmem_cols_for(a.nacc * a.np) > 512) a.nacc >>= 1;
    a.tmem_cols = tmem_cols_for(a.nacc * a.np);
    a.laplace = plan->kernel == P2P_LAPLACE;
    a.k = adjoint ? -plan->k : plan->k;
    a.status = plan->status;
    const int smem = smem_needed;
    P2P_TRY_CUDA(cudaFuncSetAttribute(k_p2p_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem), "p2p_apply_tc");
    const int groups = (plan->max_box + kTcTargets - 1) / kTcTargets;
    dim3 grid((unsigned)plan->nb, (unsigned)groups);
    k_p2p_tc<<<grid, kTcThreads, smem, s>>>(a);
    P2P_CHECK_LAUNCH("p2p_apply_tc");
    return P2P_OK;
}

extern "C" P2P_API p2p_status p2p_diag_tc_gemm(const float* A, const float* B, float* D, int32_t K, int32_t n,
                                               unsigned int* status, p2p_stream_t stream) {
    if (!A || !B || !D || !status || K < 64 || K % 64 != 0 || n < 16 || n > 256 || n % 16 != 0)
        return P2P_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const int smem = tc_smem_bytes(n);
    P2P_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm_check, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                 "p2p_diag_tc_gemm");
    k_tc_gemm_check<<<1, kTcThreads, smem, s>>>(A, B, D, K, n, tmem_cols_for(n), status);
    P2P_CHECK_LAUNCH("p2p_diag_tc_gemm");
    return P2P_OK;
}
