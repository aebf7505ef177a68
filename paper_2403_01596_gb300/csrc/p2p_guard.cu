// Guarded apply: the per-target FP64 re-evaluation of results whose FP32 error
// bound exceeds a tolerance.
//
// An FP32 evaluation whose every term G(r_ij) lambda_j is accurate to a relative
// delta has |out_i - exact_i| <= delta S_i with S_i = sum_j |G(r_ij) lambda_j|,
// however much the terms cancel.  The relative error of target i is then at
// most delta kappa_i, kappa_i = S_i / |out_i|, which is large exactly where the
// sum cancels.  The guarded apply evaluates out as usual, computes S (the
// Laplace sum of |lambda|, since |exp(ikr)| = 1), flags every target and
// right-hand side with delta S_i > tol |out_i|, and re-evaluates the flagged
// targets with FP64 arithmetic throughout (coordinates, distance, sin / cos and
// the sum over the target's whole neighbourhood), so every result it returns
// meets tol.  delta is the measured normwise error of the path: FP32 paths and
// the three-part tensor-core path 2^-20 (largest max_i |err_i| / S_i seen on the
// test workloads: 7.8e-7 and 5.2e-7 against 9.5e-7), hi/lo tensor-core path 2^-14.
#include <math.h>

#include "p2p_internal.cuh"

using namespace p2p_detail;

// Implemented in p2p_apply.cu.
p2p_status p2p_abs_sums(const p2p_plan* plan, const float2* lam, int64_t ld, int32_t nrhs, float2* S, cudaStream_t s);
bool p2p_tc_supported(const p2p_plan* plan, int32_t nrhs);

namespace {

constexpr double kDeltaFp32 = 9.5367431640625e-07;  // 2^-20
constexpr double kDeltaTc = 6.103515625e-05;        // 2^-14
constexpr double kPi = 3.14159265358979323846;

struct GuardLayout {
    float2* S;        // [n * nrhs] sums of the terms' magnitudes (leading dimension nrhs)
    int32_t* flag;    // [n] 1: target (sorted position) already listed
    int32_t* list;    // [n] flagged targets (sorted positions)
    int32_t* count;   // [1]
    size_t bytes;
};

GuardLayout guard_layout(int64_t n, int32_t nrhs, void* work) {
    Carver c{static_cast<char*>(work), 0, (size_t)-1};
    GuardLayout L;
    const size_t m = (size_t)(n > 0 ? n : 1);
    L.S = c.take<float2>(m * (size_t)nrhs);
    L.flag = c.take<int32_t>(m);
    L.list = c.take<int32_t>(m);
    L.count = c.take<int32_t>(4);
    L.bytes = align_up(c.off, 256);
    return L;
}

// One thread per (target, right-hand side): flags the target when delta S > tol |out|.
__global__ void k_guard_flag(const float2* __restrict__ out, int64_t ld, const float2* __restrict__ S,
                             const int32_t* __restrict__ perm, int64_t n, int32_t nrhs, double delta, double tol,
                             int32_t* __restrict__ flag, int32_t* __restrict__ list, int32_t* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    const int64_t s = i / nrhs;
    const int q = (int)(i - s * nrhs);
    const int64_t row = (int64_t)perm[s];
    const float2 o = out[row * ld + q];
    const double mag = sqrt((double)o.x * o.x + (double)o.y * o.y);
    if (delta * (double)S[row * nrhs + q].x > tol * mag) {
        if (atomicExch(flag + s, 1) == 0) list[atomicAdd(count, 1)] = (int32_t)s;
    }
}

// One warp per flagged target: its whole neighbourhood sum in FP64 from the caller's FP32 inputs, for every
// right-hand side, written over the FP32 result.
__global__ void k_guard_refine(const int32_t* __restrict__ list, int32_t count, const int32_t* __restrict__ box_ptr,
                               int32_t nb, const int32_t* __restrict__ pk_off, const int32_t* __restrict__ nb_src,
                               const int32_t* __restrict__ box_src, const int32_t* __restrict__ perm,
                               const float* __restrict__ pts, const int32_t* __restrict__ src_perm,
                               const float* __restrict__ src_pts, const float2* __restrict__ lam, int64_t ld,
                               int32_t nrhs, int laplace, double k, float2* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= count) return;
    const int32_t s = list[w];
    // box of target s: the last b with box_ptr[b] <= s
    int32_t lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (box_ptr[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    const int32_t b = lo;
    const int64_t ti = perm[s];
    const double tx = pts[3 * ti], ty = pts[3 * ti + 1], tz = pts[3 * ti + 2];
    const int32_t* srcs = nb_src + pk_off[b];
    const int32_t S = box_src[b];
    for (int q = 0; q < nrhs; ++q) {
        double re = 0.0, im = 0.0;
        for (int32_t p = lane; p < S; p += 32) {
            const int64_t j = src_perm[srcs[p]];
            const double dx = tx - (double)src_pts[3 * j], dy = ty - (double)src_pts[3 * j + 1],
                         dz = tz - (double)src_pts[3 * j + 2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            const double r = sqrt(r2);
            const double a = 1.0 / (4.0 * kPi * r);
            double gr = a, gi = 0.0;
            if (!laplace) {
                double sn, cs;
                sincos(k * r, &sn, &cs);
                gr = cs * a;
                gi = sn * a;
            }
            const float2 l = lam[j * ld + q];
            re += gr * (double)l.x - gi * (double)l.y;
            im += gr * (double)l.y + gi * (double)l.x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(P2P_FULL_MASK, re, o);
            im += __shfl_xor_sync(P2P_FULL_MASK, im, o);
        }
        if (lane == 0) out[ti * ld + q] = make_float2((float)re, (float)im);
    }
}

}  // namespace

extern "C" {

P2P_API p2p_status p2p_apply_guarded_workspace_size(const p2p_plan* plan, int32_t nrhs, size_t* bytes) {
    if (!plan || !bytes || nrhs < 1 || nrhs > plan->max_nrhs) return P2P_ERR_INVALID;
    *bytes = guard_layout(plan->n, nrhs, nullptr).bytes;
    return P2P_OK;
}

P2P_API p2p_status p2p_apply_guarded(const p2p_plan* plan, const void* lambda, void* out, int32_t nrhs, int64_t ld,
                                     int32_t adjoint, p2p_path path, double tol, void* work, size_t work_bytes,
                                     int64_t* refined, p2p_stream_t stream) {
    if (refined) *refined = 0;
    if (!plan || !(tol >= 0.0) || !isfinite(tol)) return P2P_ERR_INVALID;
    if (plan->layout == P2P_LAYOUT_SYMMETRIC) return P2P_ERR_UNSUPPORTED;  // its lists hold half neighbourhoods
    if (path < P2P_PATH_AUTO || path > P2P_PATH_TC_BF16X6) return P2P_ERR_INVALID;
    if (plan->n > 0 && (!work || ((uintptr_t)work & 255))) return P2P_ERR_INVALID;
    const GuardLayout L = guard_layout(plan->n, nrhs, work);
    if (plan->n > 0 && work_bytes < L.bytes) return P2P_ERR_WORKSPACE;
    // AUTO takes the hi/lo tensor-core path only where its bound leaves typical targets unflagged: random-phase
    // sums have S_i / |out_i| of 10 - 30, so below tol = 32 * 2^-14 nearly every target would be re-evaluated in
    // FP64 (measured: 19 999 of 20 000 at tol = 1e-4); there the three-part path, with the FP32 paths' bound and
    // faster than them from 16 RHS on, is the start
    if (path == P2P_PATH_AUTO) {
        const bool tc = nrhs >= 16 && p2p_tc_supported(plan, nrhs);
        path = !tc ? P2P_PATH_FP32_SHARED : (32.0 * kDeltaTc <= tol ? P2P_PATH_TC_BF16X3 : P2P_PATH_TC_BF16X6);
    }
    p2p_status st = p2p_apply_path(plan, lambda, out, nrhs, ld, adjoint, path, stream);
    if (st != P2P_OK || plan->n == 0 || plan->n_src == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = p2p_abs_sums(plan, (const float2*)lambda, ld, nrhs, L.S, s);
    if (st != P2P_OK) return st;
    P2P_TRY_CUDA(cudaMemsetAsync(L.flag, 0, (size_t)plan->n * sizeof(int32_t), s), "p2p_apply_guarded");
    P2P_TRY_CUDA(cudaMemsetAsync(L.count, 0, sizeof(int32_t), s), "p2p_apply_guarded");
    const double delta = path == P2P_PATH_TC_BF16X3 ? kDeltaTc : kDeltaFp32;
    const int64_t total = plan->n * nrhs;
    k_guard_flag<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const float2*)out, ld, L.S, plan->perm, plan->n,
                                                                 nrhs, delta, tol, L.flag, L.list, L.count);
    P2P_CHECK_LAUNCH("p2p_apply_guarded/flag");
    int32_t count = 0;
    P2P_TRY_CUDA(cudaMemcpyAsync(&count, L.count, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "p2p_apply_guarded");
    P2P_TRY_CUDA(cudaStreamSynchronize(s), "p2p_apply_guarded");
    if (count > 0) {
        const double k = plan->kernel == P2P_LAPLACE ? 0.0 : (adjoint ? -(double)plan->k : (double)plan->k);
        const int64_t threads = (int64_t)count * 32;
        k_guard_refine<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
            L.list, count, plan->box_ptr, plan->nb, plan->pk_off, plan->nb_src, plan->box_src, plan->perm, plan->pts,
            plan->src_perm, plan->src_pts, (const float2*)lambda, ld, nrhs, plan->kernel == P2P_LAPLACE, k,
            (float2*)out);
        P2P_CHECK_LAUNCH("p2p_apply_guarded/refine");
    }
    if (refined) *refined = count;
    return P2P_OK;
}

}  // extern "C"
