// Apply path of the P2P operator: strength staging (sorted gather for the
// indexed layout of Sec. 3.2, repack into the per-box redundant tiles of Sec.
// 3.3), the FP32 pair kernel, its adjoint and the coordinate gradient.
//
// The pair kernel's device code (work items, staging, lane mapping) lives in
// p2p_pair.cuh, shared with the persistent batched launch.
#include <math.h>

#include <algorithm>

#include "p2p_direct.cuh"
#include "p2p_pair.cuh"

using namespace p2p_detail;
using namespace p2p_pair;
using p2p_direct::DirectArgs;
using p2p_direct::kDirectWarps;

namespace {

// Persistent pair kernel: warp w of the grid takes items w, w + W, w + 2W, ...
// of the plan's heaviest-first item list (W = warps in the grid).
template <int R>
__global__ void __launch_bounds__(P2P_PAIR_MAX_THREADS, R == 1 ? P2P_PAIR_MIN_BLOCKS : 1)
    k_pair(const __grid_constant__ PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    unsigned char* ws = smem_raw + (size_t)warp * warp_smem_bytes(a.chunk, R, a.sym);
    run_pipeline<R>(ws, a.chunk, a.sym != 0, lane, a.items, a.n_items, (int64_t)blockIdx.x * warps + warp,
                    (int64_t)gridDim.x * warps, a.status, [&](const ItemRec&) -> const PairArgs* { return &a; });
}

// Direct kernel (sparse boxes, one right-hand side): warp w of the persistent
// grid serves K boxes at a time, sources read through the L1 (p2p_direct.cuh).
#ifndef P2P_DIRECT_MIN_BLOCKS
#define P2P_DIRECT_MIN_BLOCKS 4
#endif
template <int KERN, bool RED, int K>
__global__ void __launch_bounds__(kDirectWarps * 32, P2P_DIRECT_MIN_BLOCKS)
    k_pair_direct(const __grid_constant__ DirectArgs a) {
    __shared__ float2 red[kDirectWarps][4 * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    p2p_direct::run_direct<KERN, RED, K>(a, red[warp], (int)blockIdx.x * kDirectWarps + warp,
                                         (int64_t)gridDim.x * kDirectWarps, lane);
}

using DirectKernel = void (*)(DirectArgs);

// Repetition layout (Sec. 3.3, eq. 9): one thread per target, reading its own record front to back -- entry 0
// its coordinates, entries 1 .. S_b its neighbourhood's sources with the strengths repacked at this apply.  The
// record holds the target itself among its own box's sources: the r = 0 mask applies to every entry.
template <int KERN>
__global__ void __launch_bounds__(256) k_pair_rep(const int32_t* __restrict__ rec_off,
                                                  const float4* __restrict__ rec_xyz,
                                                  const float2* __restrict__ rec_lam, const int32_t* __restrict__ perm,
                                                  int64_t n, float k, float2* __restrict__ out, int64_t ld) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t off = rec_off[t], end = rec_off[t + 1];
    const float4 x = rec_xyz[off];
    const float4 tx[1] = {x};
    float2 acc[1][1] = {{make_float2(0.f, 0.f)}};
    for (int32_t e = off + 1; e < end; ++e) {
        const float2 l[1] = {rec_lam[e]};
        pair_core<KERN, 1, 1, true>(rec_xyz[e], l, tx, acc, k);
    }
    out[(int64_t)perm[t] * ld] = make_float2(acc[0][0].x * kInv4Pi, acc[0][0].y * kInv4Pi);
}

template <int KERN, bool RED>
DirectKernel direct_kernel_k(int k) {
    switch (k) {
        case 1: return k_pair_direct<KERN, RED, 1>;
        case 2: return k_pair_direct<KERN, RED, 2>;
        case 4: return k_pair_direct<KERN, RED, 4>;
        case 8: return k_pair_direct<KERN, RED, 8>;
        case 16: return k_pair_direct<KERN, RED, 16>;
        default: return k_pair_direct<KERN, RED, 32>;
    }
}

DirectKernel direct_kernel(const p2p_plan* p) {
    const bool red = p->layout == P2P_LAYOUT_REDUNDANT;
    if (p->kernel == P2P_HELMHOLTZ)
        return red ? direct_kernel_k<P2P_HELMHOLTZ, true>(p->direct_k) : direct_kernel_k<P2P_HELMHOLTZ, false>(p->direct_k);
    return red ? direct_kernel_k<P2P_LAPLACE, true>(p->direct_k) : direct_kernel_k<P2P_LAPLACE, false>(p->direct_k);
}

// ------------------------------------------------------ coordinate gradient --

__host__ __device__ inline int grad_smem_bytes(int chunk) { return chunk * 16 + chunk * 16 + 32 * kMaxTT * 16; }

template <int KERN, int TT>
__device__ __forceinline__ void grad_targets(const PairArgs& a, const float4* __restrict__ sx,
                                             const float4* __restrict__ slg, float4* red, int ns, int tbase, int nt,
                                             int32_t map, int rhs, int lane) {
    const int G = map_g(map), Q = map_q(map);
    const int q = map_div(map, lane);
    const int g = lane - q * G;
    float4 tx[TT];
    float2 tl[TT], tgv[TT];
    float acc[TT][3];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const int t = g + u * G;
        const bool ok = t < nt;
        tx[u] = ok ? a.xt[tbase + t] : make_float4(0.f, 0.f, 0.f, 0.f);
        tl[u] = ok ? a.lam[(int64_t)(tbase + t) * a.nrhs + rhs] : make_float2(0.f, 0.f);
        tgv[u] = ok ? a.gsrc[(int64_t)(tbase + t) * a.nrhs + rhs] : make_float2(0.f, 0.f);
        acc[u][0] = acc[u][1] = acc[u][2] = 0.f;
    }
    if (q < Q && TT % 2 == 0) {
        // targets in pairs on the packed two-lane FP32 instructions (rsqrt, sincos per pair)
        constexpr int V = TT / 2 > 0 ? TT / 2 : 1;
        float2 px2[V], py2[V], pz2[V], lx2[V], ly2[V], gx2[V], gy2[V], ax[V], ay[V], az[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int u0 = 2 * v, u1 = (2 * v + 1) % TT;
            px2[v] = make_float2(tx[u0].x, tx[u1].x);
            py2[v] = make_float2(tx[u0].y, tx[u1].y);
            pz2[v] = make_float2(tx[u0].z, tx[u1].z);
            lx2[v] = make_float2(tl[u0].x, tl[u1].x);
            ly2[v] = make_float2(tl[u0].y, tl[u1].y);
            gx2[v] = make_float2(tgv[u0].x, tgv[u1].x);
            gy2[v] = make_float2(tgv[u0].y, tgv[u1].y);
            ax[v] = ay[v] = az[v] = make_float2(0.f, 0.f);
        }
        const float2 k2 = make_float2(a.k, a.k);
        for (int s = q; s < ns; s += Q) {
            const float4 p = sx[s];
            const float4 lg = slg[s];  // (lambda_s.re, lambda_s.im, g_s.re, g_s.im)
            const float2 npx = make_float2(-p.x, -p.x), npy = make_float2(-p.y, -p.y), npz = make_float2(-p.z, -p.z);
            const float2 sl_x = make_float2(lg.x, lg.x), sl_y = make_float2(lg.y, lg.y);
            const float2 sg_x = make_float2(lg.z, lg.z), sg_y = make_float2(lg.w, lg.w);
            const float2 nsl_x = make_float2(-lg.x, -lg.x), nsg_y = make_float2(-lg.w, -lg.w);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 dx = __fadd2_rn(px2[v], npx), dy = __fadd2_rn(py2[v], npy), dz = __fadd2_rn(pz2[v], npz);
                const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                inv.x = r2.x > 0.f ? inv.x : 0.f;
                inv.y = r2.y > 0.f ? inv.y : 0.f;
                const float2 inv2 = __fmul2_rn(inv, inv);
                // C = conj(g_t) lambda_s + conj(g_s) lambda_t
                const float2 cr = __ffma2_rn(gx2[v], sl_x, __ffma2_rn(gy2[v], sl_y,
                                  __ffma2_rn(sg_x, lx2[v], __fmul2_rn(sg_y, ly2[v]))));
                const float2 ci = __ffma2_rn(gx2[v], sl_y, __ffma2_rn(gy2[v], nsl_x,
                                  __ffma2_rn(sg_x, ly2[v], __fmul2_rn(nsg_y, lx2[v]))));
                float2 w;
                if (KERN == P2P_HELMHOLTZ) {
                    const float2 kr = __fmul2_rn(k2, __fmul2_rn(r2, inv));
                    float2 sn, cs;
                    __sincosf(kr.x, &sn.x, &cs.x);
                    __sincosf(kr.y, &sn.y, &cs.y);
                    const float2 ncs = make_float2(-cs.x, -cs.y), nsn = make_float2(-sn.x, -sn.y);
                    const float2 dgr = __fmul2_rn(__ffma2_rn(nsn, kr, ncs), inv2);
                    const float2 dgi = __fmul2_rn(__ffma2_rn(cs, kr, nsn), inv2);
                    w = __ffma2_rn(dgr, cr, __fmul2_rn(make_float2(-dgi.x, -dgi.y), ci));
                } else {
                    w = __fmul2_rn(make_float2(-inv2.x, -inv2.y), cr);
                }
                w = __fmul2_rn(w, inv);
                ax[v] = __ffma2_rn(w, dx, ax[v]);
                ay[v] = __ffma2_rn(w, dy, ay[v]);
                az[v] = __ffma2_rn(w, dz, az[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            acc[2 * v][0] = ax[v].x;
            acc[2 * v][1] = ay[v].x;
            acc[2 * v][2] = az[v].x;
            acc[(2 * v + 1) % TT][0] = ax[v].y;
            acc[(2 * v + 1) % TT][1] = ay[v].y;
            acc[(2 * v + 1) % TT][2] = az[v].y;
        }
    } else if (q < Q) {
        const float k = a.k;
        for (int s = q; s < ns; s += Q) {
            const float4 p = sx[s];
            const float4 lg = slg[s];  // (lambda_s.re, lambda_s.im, g_s.re, g_s.im)
#pragma unroll
            for (int u = 0; u < TT; ++u) {
                const float dx = tx[u].x - p.x, dy = tx[u].y - p.y, dz = tx[u].z - p.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                float inv = rsqrtf(r2);
                inv = r2 > 0.f ? inv : 0.f;
                const float inv2 = inv * inv;
                // C = conj(g_t) lambda_s + conj(g_s) lambda_t
                const float cr = tgv[u].x * lg.x + tgv[u].y * lg.y + lg.z * tl[u].x + lg.w * tl[u].y;
                const float ci = tgv[u].x * lg.y - tgv[u].y * lg.x + lg.z * tl[u].y - lg.w * tl[u].x;
                float w;
                if (KERN == P2P_HELMHOLTZ) {
                    const float kr = k * (r2 * inv);
                    float sn, cs;
                    __sincosf(kr, &sn, &cs);
                    const float dgr = (-cs - sn * kr) * inv2;
                    const float dgi = (cs * kr - sn) * inv2;
                    w = dgr * cr - dgi * ci;
                } else {
                    w = -inv2 * cr;
                }
                w *= inv;
                acc[u][0] = fmaf(w, dx, acc[u][0]);
                acc[u][1] = fmaf(w, dy, acc[u][1]);
                acc[u][2] = fmaf(w, dz, acc[u][2]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < TT; ++u) red[lane * TT + u] = make_float4(acc[u][0], acc[u][1], acc[u][2], 0.f);
    __syncwarp();
    for (int t = lane; t < nt; t += 32) {
        const int u = map_div(map, t);
        const int gg = t - u * G;
        float v0 = 0.f, v1 = 0.f, v2 = 0.f;
        for (int qq = 0; qq < Q; ++qq) {
            const float4 w = red[(qq * G + gg) * TT + u];
            v0 += w.x;
            v1 += w.y;
            v2 += w.z;
        }
        float* dst = a.grad + (int64_t)a.perm[tbase + t] * 3;
        atomicAdd(dst, v0 * kInv4Pi);
        atomicAdd(dst + 1, v1 * kInv4Pi);
        atomicAdd(dst + 2, v2 * kInv4Pi);
    }
    __syncwarp();
}

// One warp per work item; sources gathered through the box's source list.
template <int KERN>
__global__ void __launch_bounds__(512) k_grad(const __grid_constant__ PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (item >= a.n_items) return;
    const int chunk = a.chunk;
    unsigned char* ws = smem_raw + (size_t)warp * grad_smem_bytes(chunk);
    float4* sx = reinterpret_cast<float4*>(ws);
    float4* slg = reinterpret_cast<float4*>(ws + chunk * 16);
    float4* red = reinterpret_cast<float4*>(ws + chunk * 32);
    const ItemRec r = a.items[item];
    for (int p = lane; p < r.ns; p += 32) sx[p] = a.xs[a.nb_src[r.src_off + p]];
    for (int rhs = 0; rhs < a.nrhs; ++rhs) {
        __syncwarp();
        for (int p = lane; p < r.ns; p += 32) {
            const int64_t row = (int64_t)a.nb_src[r.src_off + p] * a.nrhs + rhs;
            const float2 l = a.lam[row], gg = a.gsrc[row];
            slg[p] = make_float4(l.x, l.y, gg.x, gg.y);
        }
        __syncwarp();
        for (int t0 = 0; t0 < r.nt; t0 += a.tg) {
            const int nt = min(a.tg, r.nt - t0);
            const int32_t map = (t0 + a.tg >= r.nt) ? r.map_last : r.map_full;
            const int tt = map_tt(map);
            if (tt == 1) grad_targets<KERN, 1>(a, sx, slg, red, r.ns, r.tb + t0, nt, map, rhs, lane);
            else if (tt == 2) grad_targets<KERN, 2>(a, sx, slg, red, r.ns, r.tb + t0, nt, map, rhs, lane);
            else grad_targets<KERN, 4>(a, sx, slg, red, r.ns, r.tb + t0, nt, map, rhs, lane);
        }
    }
}

// ----------------------------------------------------------------- staging --

// dst[s * nrhs + q] = src[rows[s] * ld + q]  (rows[s] < 0: zero)
__global__ void k_gather_rows(const float2* __restrict__ src, int64_t ld, const int32_t* __restrict__ rows, int64_t n,
                              int32_t nrhs, float2* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    const int64_t s = i / nrhs;
    const int q = (int)(i - s * nrhs);
    const int32_t r = rows[s];
    dst[i] = r >= 0 ? src[(int64_t)r * ld + q] : make_float2(0.f, 0.f);
}

// One right-hand side, four rows per thread: dst[s] = src[rows[s] * ld]
// (rows[s] < 0: zero) with a 16-byte index load, four independent gathers
// and two 16-byte stores.  rows and dst are 16-byte aligned.
__global__ void k_gather_rows4(const float2* __restrict__ src, int64_t ld, const int32_t* __restrict__ rows, int64_t n,
                               float2* __restrict__ dst) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s0 = q * 4;
    if (s0 >= n) return;
    if (s0 + 4 <= n) {
        const int4 r = *reinterpret_cast<const int4*>(rows + s0);
        const float2 z = make_float2(0.f, 0.f);
        const float2 v0 = r.x >= 0 ? src[(int64_t)r.x * ld] : z;
        const float2 v1 = r.y >= 0 ? src[(int64_t)r.y * ld] : z;
        const float2 v2 = r.z >= 0 ? src[(int64_t)r.z * ld] : z;
        const float2 v3 = r.w >= 0 ? src[(int64_t)r.w * ld] : z;
        reinterpret_cast<float4*>(dst + s0)[0] = make_float4(v0.x, v0.y, v1.x, v1.y);
        reinterpret_cast<float4*>(dst + s0)[1] = make_float4(v2.x, v2.y, v3.x, v3.y);
    } else {
        for (int64_t s = s0; s < n; ++s) dst[s] = rows[s] >= 0 ? src[(int64_t)rows[s] * ld] : make_float2(0.f, 0.f);
    }
}

cudaError_t stage_rows(const float2* src, int64_t ld, const int32_t* rows, int64_t nrows, int32_t nrhs, float2* dst,
                       cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    if (nrhs == 1) {
        const int64_t threads = (nrows + 3) / 4;
        k_gather_rows4<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(src, ld, rows, nrows, dst);
    } else {
        const int64_t total = nrows * nrhs;
        k_gather_rows<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(src, ld, rows, nrows, nrhs, dst);
    }
    return cudaGetLastError();
}

// dst[s * nrhs + q] = (|src[rows[s] * ld + q]|, 0)  (rows[s] < 0: zero): the strengths' magnitudes, for the sums
// of the terms' magnitudes of a guarded apply.
__global__ void k_gather_abs(const float2* __restrict__ src, int64_t ld, const int32_t* __restrict__ rows, int64_t n,
                             int32_t nrhs, float2* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    const int64_t s = i / nrhs;
    const int q = (int)(i - s * nrhs);
    const int32_t r = rows[s];
    float m = 0.f;
    if (r >= 0) {
        const float2 v = src[(int64_t)r * ld + q];
        m = hypotf(v.x, v.y);
    }
    dst[i] = make_float2(m, 0.f);
}

int r_index(int R) { return R == 1 ? 0 : (R == 2 ? 1 : 2); }

// The dynamic shared-memory limit is an attribute of the kernel function,
// shared by every plan: it only ever grows (to the largest launch seen), so no
// plan's configuration can lower it below another plan's launch.
int g_smem_attr[3] = {0, 0, 0};

template <int R>
cudaError_t raise_smem_limit(int smem) {
    int& cur = g_smem_attr[r_index(R)];
    if (smem <= __atomic_load_n(&cur, __ATOMIC_ACQUIRE)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_pair<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        int seen = __atomic_load_n(&cur, __ATOMIC_ACQUIRE);
        while (seen < smem && !__atomic_compare_exchange_n(&cur, &seen, smem, false, __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE)) {
        }
    }
    return e;
}

template <int R>
cudaError_t configure_r(p2p_plan* p) {
    const int ri = r_index(R);
    p->grid[ri] = 0;
    p->grid_warps[ri] = 0;
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_pair<R>);
    if (e != cudaSuccess) return e;
    const bool sym = p->layout == P2P_LAYOUT_SYMMETRIC;
    // the tuning's warps per block, halved until one block fits (threads, shared memory)
    for (int warps = p->tune.warps_per_cta; warps >= 1; warps >>= 1) {
        const int smem = warps * warp_smem_bytes(p->tune.chunk, R, sym);
        if (smem > optin || warps * 32 > fa.maxThreadsPerBlock) continue;
        e = raise_smem_limit<R>(smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair<R>, warps * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm > 0) {
            p->grid[ri] = per_sm * sms;
            p->grid_warps[ri] = warps;
            return cudaSuccess;
        }
    }
    return cudaSuccess;  // no block fits: the launch reports P2P_ERR_UNSUPPORTED
}

template <int R>
p2p_status launch_pair(const p2p_plan* p, const PairArgs& a, cudaStream_t s) {
    const int warps = p->grid_warps[r_index(R)];
    const int smem = warps * warp_smem_bytes(a.chunk, R, a.sym != 0);
    int grid = p->grid[r_index(R)];
    if (grid <= 0) {
        set_message("p2p_apply: the pair kernel does not fit on this device with this tuning (shared memory)");
        return P2P_ERR_UNSUPPORTED;
    }
    if ((int64_t)grid * warps > a.n_items) grid = (int)((a.n_items + warps - 1) / warps);
    P2P_TRY_CUDA(raise_smem_limit<R>(smem), "p2p_apply/attribute");
    k_pair<R><<<grid, warps * 32, smem, s>>>(a);
    P2P_CHECK_LAUNCH("p2p_apply/pair");
    return P2P_OK;
}

// lam: strengths (one row per source, may be NULL when there are none); out: results (one row per target).
p2p_status check_apply_args(const p2p_plan* plan, const void* lam, const void* out, int32_t nrhs, int64_t ld) {
    if (!plan || nrhs < 1 || nrhs > plan->max_nrhs || ld < nrhs) return P2P_ERR_INVALID;
    if ((plan->n_src > 0 && !lam) || (plan->n > 0 && !out)) return P2P_ERR_INVALID;
    if (((uintptr_t)lam & 7) || ((uintptr_t)out & 7)) return P2P_ERR_INVALID;
    return P2P_OK;
}

}  // namespace

// S[perm[t] * nrhs + q] = sum over the sources s of target t's neighbourhood (r > 0) of |lambda_sq| / (4 pi r),
// i.e. sum_s |G(r) lambda_sq| for both kernels (|exp(ikr)| = 1), through the staged pipeline with the Laplace
// kernel on the strengths' magnitudes (lambda: leading dimension ld; S: nrhs).  Uses the plan's staging buffer.
p2p_status p2p_abs_sums(const p2p_plan* plan, const float2* lam, int64_t ld, int32_t nrhs, float2* S, cudaStream_t s) {
    const bool red = plan->layout == P2P_LAYOUT_REDUNDANT;
    const int32_t* rows = red ? plan->pk_src : plan->src_perm;
    const int64_t nrows = red ? plan->packed : plan->n_src;
    if (nrows > 0) {
        const int64_t total = nrows * nrhs;
        k_gather_abs<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(lam, ld, rows, nrows, nrhs, plan->lam_buf);
        P2P_CHECK_LAUNCH("p2p_apply_guarded/abs");
    }
    P2P_TRY_CUDA(cudaMemsetAsync(S, 0, (size_t)plan->n * nrhs * 8, s), "p2p_apply_guarded");
    if (plan->n_items == 0 || nrows == 0) return P2P_OK;
    PairArgs a = base_args(plan);
    a.out = S;
    a.ld = nrhs;
    a.nrhs = nrhs;
    a.kernel = P2P_LAPLACE;
    a.k = 0.f;
    a.atomic_out = 1;  // the buffer is zeroed above
    const int R = nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1);
    return R == 1 ? launch_pair<1>(plan, a, s) : (R == 2 ? launch_pair<2>(plan, a, s) : launch_pair<4>(plan, a, s));
}

cudaError_t p2p_group_configure(p2p_plan* p);
p2p_status p2p_group_launch(const p2p_plan* p, float2* out, int64_t ld, float k, cudaStream_t s);

cudaError_t p2p_pair_configure(p2p_plan* plan) {
    cudaError_t e = p2p_group_configure(plan);
    if (e == cudaSuccess) e = configure_r<1>(plan);
    if (e == cudaSuccess) e = configure_r<2>(plan);
    if (e == cudaSuccess) e = configure_r<4>(plan);
    plan->direct_grid = 0;
    if (e == cudaSuccess && plan->direct_k > 0) {
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct_kernel(plan), kDirectWarps * 32, 0);
        if (e == cudaSuccess) plan->direct_grid = per_sm * sms;
    }
    return e;
}

// Entries shared with the tensor-core translation unit.
p2p_status p2p_tc_stage(const p2p_plan* plan, const float2* lam, int32_t nrhs, int64_t ld, int np,
                        cudaStream_t s);
p2p_status p2p_apply_tc(const p2p_plan* plan, float2* out, int32_t nrhs, int64_t ld, int32_t adjoint, int np,
                        cudaStream_t s);
bool p2p_tc_supported(const p2p_plan* plan, int32_t nrhs);

extern "C" {

static p2p_path resolve_path(const p2p_plan* plan, int32_t nrhs, p2p_path path) {
    if (path == P2P_PATH_AUTO)
        return (nrhs >= 16 && p2p_tc_supported(plan, nrhs)) ? P2P_PATH_TC_BF16X3 : P2P_PATH_FP32_SHARED;
    return path;
}

static bool is_tc(p2p_path path) { return path == P2P_PATH_TC_BF16X3 || path == P2P_PATH_TC_BF16X6; }
static int tc_parts(p2p_path path) { return path == P2P_PATH_TC_BF16X6 ? 3 : 2; }

P2P_API p2p_status p2p_apply_stage(const p2p_plan* plan, const void* lambda, int32_t nrhs, int64_t ld, p2p_path path,
                                   p2p_stream_t stream) {
    if (!plan) return P2P_ERR_INVALID;
    p2p_status st = check_apply_args(plan, lambda, plan->n > 0 ? plan : nullptr, nrhs, ld);
    if (st != P2P_OK) return st;
    if (path < P2P_PATH_AUTO || path > P2P_PATH_TC_BF16X6) return P2P_ERR_INVALID;
    if (plan->n == 0 || plan->n_src == 0) return P2P_OK;
    path = resolve_path(plan, nrhs, path);
    if (is_tc(path) && !p2p_tc_supported(plan, nrhs)) return P2P_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (is_tc(path)) return p2p_tc_stage(plan, (const float2*)lambda, nrhs, ld, tc_parts(path), s);
    if (plan->layout == P2P_LAYOUT_REPETITION) {
        // every target's record gets its own copy of its sources' strengths (the record head: 0)
        P2P_TRY_CUDA(stage_rows((const float2*)lambda, ld, plan->rec_src, plan->records, 1, plan->lam_buf, s),
                     "p2p_apply_stage");
        return P2P_OK;
    }
    const bool red = plan->layout == P2P_LAYOUT_REDUNDANT;
    const int32_t* rows = red ? plan->pk_src : plan->src_perm;  // strengths live on the sources
    const int64_t nrows = red ? plan->packed : plan->n_src;
    P2P_TRY_CUDA(stage_rows((const float2*)lambda, ld, rows, nrows, nrhs, plan->lam_buf, s), "p2p_apply_stage");
    return P2P_OK;
}

P2P_API p2p_status p2p_apply_staged(const p2p_plan* plan, void* out, int32_t nrhs, int64_t ld, int32_t adjoint,
                                    p2p_path path, p2p_stream_t stream) {
    if (!plan) return P2P_ERR_INVALID;
    p2p_status st = check_apply_args(plan, plan->n_src > 0 ? plan : nullptr, out, nrhs, ld);
    if (st != P2P_OK) return st;
    if (path < P2P_PATH_AUTO || path > P2P_PATH_TC_BF16X6) return P2P_ERR_INVALID;
    if (plan->n == 0) return P2P_OK;
    path = resolve_path(plan, nrhs, path);
    if (is_tc(path) && !p2p_tc_supported(plan, nrhs)) return P2P_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    // a two-set plan may have target boxes without any source nearby: no item or unit writes their rows
    if (plan->two_sets)
        P2P_TRY_CUDA(cudaMemset2DAsync(out, (size_t)ld * 8, 0, (size_t)nrhs * 8, (size_t)plan->n, s), "p2p_apply/zero");
    if (plan->n_src == 0) return P2P_OK;
    if (is_tc(path)) return p2p_apply_tc(plan, (float2*)out, nrhs, ld, adjoint, tc_parts(path), s);
    if (plan->layout == P2P_LAYOUT_REPETITION) {
        const float k = adjoint ? -plan->k : plan->k;
        const unsigned blocks = (unsigned)((plan->n + 255) / 256);
        if (plan->kernel == P2P_HELMHOLTZ)
            k_pair_rep<P2P_HELMHOLTZ><<<blocks, 256, 0, s>>>(plan->rec_off, plan->rec_xyz, plan->lam_buf, plan->perm,
                                                              plan->n, k, (float2*)out, ld);
        else
            k_pair_rep<P2P_LAPLACE><<<blocks, 256, 0, s>>>(plan->rec_off, plan->rec_xyz, plan->lam_buf, plan->perm,
                                                            plan->n, k, (float2*)out, ld);
        P2P_CHECK_LAUNCH("p2p_apply/repetition");
        return P2P_OK;
    }
    PairArgs a = base_args(plan);
    a.out = (float2*)out;
    a.ld = ld;
    a.nrhs = nrhs;
    if (adjoint) a.k = -a.k;
    if (nrhs == 1 && plan->group_k && plan->group_grid > 0) {
        // one right-hand side, groups of boxes staging the union of their neighbourhoods once
        return p2p_group_launch(plan, (float2*)out, ld, a.k, s);
    }
    if (nrhs == 1 && plan->direct_k > 0 && plan->direct_grid > 0) {
        // one right-hand side on sparse boxes: the direct kernel, one item per box, every row stored once
        DirectArgs d;
        d.items = plan->ditems;
        d.n_items = plan->nb;
        d.xs = plan->xs_src;
        d.xt = plan->xs;
        d.pk_xyz = plan->pk_xyz;
        d.nb_src = plan->nb_src;
        d.lam = plan->lam_buf;
        d.perm = plan->perm;
        d.out = (float2*)out;
        d.ld = ld;
        d.k = a.k;
        const int64_t blocks_needed = (plan->nb + (int64_t)kDirectWarps * plan->direct_k - 1) /
                                      ((int64_t)kDirectWarps * plan->direct_k);
        const int grid = (int)std::min<int64_t>(plan->direct_grid, blocks_needed);
        direct_kernel(plan)<<<grid, kDirectWarps * 32, 0, s>>>(d);
        P2P_CHECK_LAUNCH("p2p_apply/direct");
        return P2P_OK;
    }
    if (a.atomic_out && !plan->two_sets)
        P2P_TRY_CUDA(cudaMemset2DAsync(out, (size_t)ld * 8, 0, (size_t)nrhs * 8, (size_t)plan->n, s), "p2p_apply/zero");
    if (plan->n_items == 0) return P2P_OK;
    const int R = path == P2P_PATH_FP32_PER_RHS ? 1 : (nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1));
    return R == 1 ? launch_pair<1>(plan, a, s) : (R == 2 ? launch_pair<2>(plan, a, s) : launch_pair<4>(plan, a, s));
}

P2P_API p2p_status p2p_apply_path(const p2p_plan* plan, const void* lambda, void* out, int32_t nrhs, int64_t ld,
                                  int32_t adjoint, p2p_path path, p2p_stream_t stream) {
    p2p_status st = check_apply_args(plan, lambda, out, nrhs, ld);
    if (st != P2P_OK) return st;
    if (lambda == out && plan->n > 0 && plan->n_src > 0) return P2P_ERR_INVALID;
    st = p2p_apply_stage(plan, lambda, nrhs, ld, path, stream);
    if (st != P2P_OK) return st;
    return p2p_apply_staged(plan, out, nrhs, ld, adjoint, path, stream);
}

P2P_API p2p_status p2p_apply(const p2p_plan* plan, const void* lambda, void* out, int32_t nrhs, int64_t ld,
                             p2p_stream_t stream) {
    return p2p_apply_path(plan, lambda, out, nrhs, ld, 0, P2P_PATH_AUTO, stream);
}

P2P_API p2p_status p2p_apply_adjoint(const p2p_plan* plan, const void* g, void* out, int32_t nrhs, int64_t ld,
                                     p2p_stream_t stream) {
    // a two-set operator's adjoint maps target space to source space: a plan with the roles exchanged
    if (plan && plan->two_sets) return P2P_ERR_UNSUPPORTED;
    return p2p_apply_path(plan, g, out, nrhs, ld, 1, P2P_PATH_AUTO, stream);
}

P2P_API p2p_status p2p_grad_points(const p2p_plan* plan, const void* lambda, const void* g, float* grad,
                                   int32_t nrhs, int64_t ld, p2p_stream_t stream) {
    p2p_status st = check_apply_args(plan, lambda, g, nrhs, ld);
    if (st != P2P_OK) return st;
    if (plan->n == 0) return P2P_OK;
    if (!grad || ((uintptr_t)grad & 3)) return P2P_ERR_INVALID;
    if (plan->layout == P2P_LAYOUT_SYMMETRIC) return P2P_ERR_UNSUPPORTED;  // needs the full source lists
    if (plan->two_sets) return P2P_ERR_UNSUPPORTED;                         // one point set only
    cudaStream_t s = (cudaStream_t)stream;
    P2P_TRY_CUDA(stage_rows((const float2*)lambda, ld, plan->perm, plan->n, nrhs, plan->lam_buf, s),
                 "p2p_grad_points/stage");
    P2P_TRY_CUDA(stage_rows((const float2*)g, ld, plan->perm, plan->n, nrhs, plan->g_buf, s), "p2p_grad_points/stage");
    P2P_TRY_CUDA(cudaMemsetAsync(grad, 0, (size_t)plan->n * 3 * sizeof(float), s), "p2p_grad_points/zero");
    PairArgs a = base_args(plan);
    a.grad = grad;
    a.nrhs = nrhs;
    const int warps = plan->tune.warps_per_cta;
    const int smem = warps * grad_smem_bytes(a.chunk);
    auto kern = plan->kernel == P2P_HELMHOLTZ ? k_grad<P2P_HELMHOLTZ> : k_grad<P2P_LAPLACE>;
    P2P_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem), "p2p_grad_points");
    kern<<<(unsigned)((a.n_items + warps - 1) / warps), warps * 32, smem, s>>>(a);
    P2P_CHECK_LAUNCH("p2p_grad_points/kernel");
    return P2P_OK;
}

}  // extern "C"
