// Apply path of the P2P operator: strength staging (sorted gather for the
// indexed layout of Sec. 3.2, repack into the per-box redundant tiles of Sec.
// 3.3), the FP32 pair kernel, its adjoint and the coordinate gradient.
//
// The pair kernel's device code (work items, staging, lane mapping) lives in
// p2p_pair.cuh, shared with the persistent batched launch.
#include <math.h>

#include "p2p_pair.cuh"

using namespace p2p_detail;
using namespace p2p_pair;

namespace {


template <int KERN, int R, bool RED>
__global__ void __launch_bounds__(512, P2P_PAIR_MIN_BLOCKS) k_pair(const PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (item >= a.n_items) return;
    process_item<KERN, R, RED>(a, item, smem_raw + (size_t)warp * warp_smem_bytes(a.chunk, R), lane);
}

// ------------------------------------------------------ coordinate gradient --

__host__ __device__ inline int grad_smem_bytes(int chunk) {
    return chunk * 16 + chunk * 16 + chunk * 4 + 64 * 4 + 32 * kMaxTT * 16;
}

template <int KERN, int TT>
__device__ __forceinline__ void grad_targets(const PairArgs& a, const float4* __restrict__ sx,
                                             const float4* __restrict__ slg, float4* red, int ns, int tbase, int nt,
                                             int rhs, int lane) {
    const int G = (nt + TT - 1) / TT;
    const int Q = 32 / G;
    const int g = lane % G, q = lane / G;
    float4 tx[TT];
    float2 tl[TT], tgv[TT];
    float acc[TT][3];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const int t = g + u * G;
        const bool ok = t < nt;
        tx[u] = ok ? a.xs[tbase + t] : make_float4(0.f, 0.f, 0.f, 0.f);
        tl[u] = ok ? a.lam[(int64_t)(tbase + t) * a.nrhs + rhs] : make_float2(0.f, 0.f);
        tgv[u] = ok ? a.gsrc[(int64_t)(tbase + t) * a.nrhs + rhs] : make_float2(0.f, 0.f);
        acc[u][0] = acc[u][1] = acc[u][2] = 0.f;
    }
    if (q < Q) {
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
        const int gg = t % G, u = t / G;
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

template <int KERN>
__global__ void __launch_bounds__(512) k_grad(const PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (item >= a.n_items) return;
    const int chunk = a.chunk;
    unsigned char* ws = smem_raw + (size_t)warp * grad_smem_bytes(chunk);
    float4* sx = reinterpret_cast<float4*>(ws);
    float4* slg = reinterpret_cast<float4*>(ws + chunk * 16);
    int* sj = reinterpret_cast<int*>(ws + chunk * 32);
    int* seg = sj + chunk;
    float4* red = reinterpret_cast<float4*>(seg + 64);
    const int4 it = a.items[item];
    const int b = it.x, s0 = it.y;
    const int ns = min(chunk, a.box_src[b] - s0);
    stage_sources<false>(a, b, s0, ns, sx, sj, seg, lane);
    const int tb = a.box_ptr[b];
    const int nt_all = a.box_ptr[b + 1] - tb;
    for (int rhs = 0; rhs < a.nrhs; ++rhs) {
        __syncwarp();
        for (int p = lane; p < ns; p += 32) {
            const int64_t row = (int64_t)sj[p] * a.nrhs + rhs;
            const float2 l = a.lam[row], gg = a.gsrc[row];
            slg[p] = make_float4(l.x, l.y, gg.x, gg.y);
        }
        __syncwarp();
        for (int t0 = 0; t0 < nt_all; t0 += a.tg) {
            const int nt = min(a.tg, nt_all - t0);
            const int tt = choose_tt(nt, ns);
            if (tt == 1) grad_targets<KERN, 1>(a, sx, slg, red, ns, tb + t0, nt, rhs, lane);
            else if (tt == 2) grad_targets<KERN, 2>(a, sx, slg, red, ns, tb + t0, nt, rhs, lane);
            else grad_targets<KERN, 4>(a, sx, slg, red, ns, tb + t0, nt, rhs, lane);
        }
    }
}

// ----------------------------------------------------------------- staging --

// dst[s * nrhs + q] = src[perm[s] * ld + q]
__global__ void k_gather_rows(const float2* __restrict__ src, int64_t ld, const int32_t* __restrict__ rows, int64_t n,
                              int32_t nrhs, float2* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    const int64_t s = i / nrhs;
    const int q = (int)(i - s * nrhs);
    const int32_t r = rows[s];
    dst[i] = r >= 0 ? src[(int64_t)r * ld + q] : make_float2(0.f, 0.f);
}

template <int KERN, int R, bool RED>
cudaError_t launch_pair(const PairArgs& a, int warps, cudaStream_t s) {
    const int smem = warps * warp_smem_bytes(a.chunk, R);
    auto kern = k_pair<KERN, R, RED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (a.n_items + warps - 1) / warps;
    kern<<<(unsigned)blocks, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int KERN, bool RED>
cudaError_t launch_pair_r(const PairArgs& a, int R, int warps, cudaStream_t s) {
    if (R == 1) return launch_pair<KERN, 1, RED>(a, warps, s);
    if (R == 2) return launch_pair<KERN, 2, RED>(a, warps, s);
    return launch_pair<KERN, 4, RED>(a, warps, s);
}

p2p_status check_apply_args(const p2p_plan* plan, const void* lam, const void* out, int32_t nrhs, int64_t ld) {
    if (!plan || nrhs < 1 || nrhs > plan->max_nrhs || ld < nrhs) return P2P_ERR_INVALID;
    if (plan->n > 0 && (!lam || !out)) return P2P_ERR_INVALID;
    if (((uintptr_t)lam & 7) || ((uintptr_t)out & 7)) return P2P_ERR_INVALID;
    return P2P_OK;
}

}  // namespace

// Entry shared with the tensor-core translation unit.
p2p_status p2p_apply_tc(const p2p_plan* plan, const float2* lam_sorted, float2* out, int32_t nrhs, int64_t ld,
                        int32_t adjoint, cudaStream_t s);
bool p2p_tc_supported(const p2p_plan* plan, int32_t nrhs);

extern "C" {

static p2p_path resolve_path(const p2p_plan* plan, int32_t nrhs, p2p_path path) {
    if (path == P2P_PATH_AUTO)
        return (nrhs >= 16 && p2p_tc_supported(plan, nrhs)) ? P2P_PATH_TC_BF16X3 : P2P_PATH_FP32_SHARED;
    return path;
}

P2P_API p2p_status p2p_apply_stage(const p2p_plan* plan, const void* lambda, int32_t nrhs, int64_t ld, p2p_path path,
                                   p2p_stream_t stream) {
    p2p_status st = check_apply_args(plan, lambda, lambda, nrhs, ld);
    if (st != P2P_OK) return st;
    if (path < P2P_PATH_AUTO || path > P2P_PATH_TC_BF16X3) return P2P_ERR_INVALID;
    if (plan->n == 0) return P2P_OK;
    path = resolve_path(plan, nrhs, path);
    if (path == P2P_PATH_TC_BF16X3 && !p2p_tc_supported(plan, nrhs)) return P2P_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const bool red = plan->layout == P2P_LAYOUT_REDUNDANT && path != P2P_PATH_TC_BF16X3;
    const int32_t* rows = red ? plan->pk_src : plan->perm;
    const int64_t nrows = red ? plan->packed : plan->n;
    const int64_t total = nrows * nrhs;
    if (total > 0) {
        k_gather_rows<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const float2*)lambda, ld, rows, nrows, nrhs,
                                                                     plan->lam_buf);
        P2P_CHECK_LAUNCH("p2p_apply_stage");
    }
    return P2P_OK;
}

P2P_API p2p_status p2p_apply_staged(const p2p_plan* plan, void* out, int32_t nrhs, int64_t ld, int32_t adjoint,
                                    p2p_path path, p2p_stream_t stream) {
    p2p_status st = check_apply_args(plan, out, out, nrhs, ld);
    if (st != P2P_OK) return st;
    if (path < P2P_PATH_AUTO || path > P2P_PATH_TC_BF16X3) return P2P_ERR_INVALID;
    if (plan->n == 0) return P2P_OK;
    path = resolve_path(plan, nrhs, path);
    if (path == P2P_PATH_TC_BF16X3 && !p2p_tc_supported(plan, nrhs)) return P2P_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (path == P2P_PATH_TC_BF16X3) return p2p_apply_tc(plan, plan->lam_buf, (float2*)out, nrhs, ld, adjoint, s);
    const bool red = plan->layout == P2P_LAYOUT_REDUNDANT;
    PairArgs a = base_args(plan);
    a.out = (float2*)out;
    a.ld = ld;
    a.nrhs = nrhs;
    if (adjoint) a.k = -a.k;
    if (a.atomic_out)
        P2P_TRY_CUDA(cudaMemset2DAsync(out, (size_t)ld * 8, 0, (size_t)nrhs * 8, (size_t)plan->n, s), "p2p_apply/zero");
    const int R = path == P2P_PATH_FP32_PER_RHS ? 1 : (nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1));
    const int warps = plan->tune.warps_per_cta;
    cudaError_t e;
    if (plan->kernel == P2P_HELMHOLTZ)
        e = red ? launch_pair_r<P2P_HELMHOLTZ, true>(a, R, warps, s) : launch_pair_r<P2P_HELMHOLTZ, false>(a, R, warps, s);
    else
        e = red ? launch_pair_r<P2P_LAPLACE, true>(a, R, warps, s) : launch_pair_r<P2P_LAPLACE, false>(a, R, warps, s);
    P2P_TRY_CUDA(e, "p2p_apply/pair");
    return P2P_OK;
}

P2P_API p2p_status p2p_apply_path(const p2p_plan* plan, const void* lambda, void* out, int32_t nrhs, int64_t ld,
                                  int32_t adjoint, p2p_path path, p2p_stream_t stream) {
    p2p_status st = check_apply_args(plan, lambda, out, nrhs, ld);
    if (st != P2P_OK) return st;
    if (lambda == out && plan->n > 0) return P2P_ERR_INVALID;
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
    return p2p_apply_path(plan, g, out, nrhs, ld, 1, P2P_PATH_AUTO, stream);
}

P2P_API p2p_status p2p_grad_points(const p2p_plan* plan, const void* lambda, const void* g, float* grad,
                                   int32_t nrhs, int64_t ld, p2p_stream_t stream) {
    p2p_status st = check_apply_args(plan, lambda, g, nrhs, ld);
    if (st != P2P_OK) return st;
    if (plan->n == 0) return P2P_OK;
    if (!grad || ((uintptr_t)grad & 3)) return P2P_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t total = plan->n * nrhs;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    k_gather_rows<<<blocks, 256, 0, s>>>((const float2*)lambda, ld, plan->perm, plan->n, nrhs, plan->lam_buf);
    P2P_CHECK_LAUNCH("p2p_grad_points/stage");
    k_gather_rows<<<blocks, 256, 0, s>>>((const float2*)g, ld, plan->perm, plan->n, nrhs, plan->g_buf);
    P2P_CHECK_LAUNCH("p2p_grad_points/stage");
    P2P_TRY_CUDA(cudaMemsetAsync(grad, 0, (size_t)plan->n * 3 * sizeof(float), s), "p2p_grad_points/zero");
    PairArgs a = base_args(plan);
    a.src_xyz = plan->xs;
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
