// Host-buffer apply: strengths uploaded from host memory, the operator applied,
// results downloaded, for a sequence of plans, with the copies of neighbouring
// plans overlapping each plan's kernels (two device slots, one copy stream).
#include <cstdlib>

#include "p2p_internal.cuh"

using p2p_detail::align_up;
using p2p_detail::set_cuda_error;

namespace {
constexpr int32_t kMaxHostPlans = 64;
constexpr int32_t kMaxHostNrhs = 256;

size_t slot_bytes(int64_t max_n, int32_t nrhs) { return align_up((size_t)max_n * (size_t)nrhs * 8, 256); }
}  // namespace

struct p2p_host_pipe {
    int64_t max_n;
    int32_t nrhs;
    float2* lam[2];
    float2* out[2];
    cudaStream_t copy;
    cudaEvent_t start, done;
    cudaEvent_t in_ready[2];   // slot's strengths uploaded
    cudaEvent_t out_ready[2];  // slot's results written
};

extern "C" {

P2P_API p2p_status p2p_host_pipe_workspace_size(int64_t max_n, int32_t nrhs, size_t* bytes) {
    if (!bytes || max_n < 1 || max_n > (int64_t)INT32_MAX || nrhs < 1 || nrhs > kMaxHostNrhs) return P2P_ERR_INVALID;
    *bytes = 4 * slot_bytes(max_n, nrhs);
    return P2P_OK;
}

P2P_API p2p_status p2p_host_pipe_create(p2p_host_pipe** pipe, int64_t max_n, int32_t nrhs, void* workspace,
                                        size_t workspace_bytes) {
    if (!pipe) return P2P_ERR_INVALID;
    *pipe = nullptr;
    size_t need = 0;
    p2p_status st = p2p_host_pipe_workspace_size(max_n, nrhs, &need);
    if (st != P2P_OK) return st;
    if (!workspace || ((uintptr_t)workspace & 255)) return P2P_ERR_INVALID;
    if (workspace_bytes < need) return P2P_ERR_WORKSPACE;
    p2p_host_pipe* p = (p2p_host_pipe*)calloc(1, sizeof(p2p_host_pipe));
    if (!p) return P2P_ERR_ALLOC;
    p->max_n = max_n;
    p->nrhs = nrhs;
    const size_t sb = slot_bytes(max_n, nrhs);
    char* base = (char*)workspace;
    for (int i = 0; i < 2; ++i) {
        p->lam[i] = (float2*)(base + (size_t)i * sb);
        p->out[i] = (float2*)(base + (size_t)(2 + i) * sb);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking);
    cudaEvent_t* evs[6] = {&p->start, &p->done, &p->in_ready[0], &p->in_ready[1], &p->out_ready[0], &p->out_ready[1]};
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(evs[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        set_cuda_error(e, "p2p_host_pipe_create");
        p2p_host_pipe_destroy(p);
        return P2P_ERR_CUDA;
    }
    *pipe = p;
    return P2P_OK;
}

P2P_API p2p_status p2p_apply_host(p2p_host_pipe* pipe, const p2p_plan* const* plans, int32_t count,
                                  const void* const* lambdas, void* const* outs, p2p_stream_t stream) {
    if (!pipe || !plans || !lambdas || !outs || count < 1 || count > kMaxHostPlans) return P2P_ERR_INVALID;
    const int32_t nrhs = pipe->nrhs;
    for (int g = 0; g < count; ++g) {
        const p2p_plan* pl = plans[g];
        if (!pl || pl->n > pipe->max_n || pl->n_src > pipe->max_n || pl->max_nrhs < nrhs) return P2P_ERR_INVALID;
        if (pl->n > 0 && (!lambdas[g] || !outs[g])) return P2P_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream, c = pipe->copy;
    // Issue order (copy stream): up(0), up(1), down(0), up(2), down(1), ...  The copy stream is FIFO, so
    // up(g + 2) follows down(g), which waited for plan g's kernels: slot g % 2 is free when it is refilled.
    auto upload = [&](int g) -> cudaError_t {
        const int sl = g & 1;
        const size_t bytes = (size_t)plans[g]->n_src * nrhs * 8;  // strengths: one row per source
        cudaError_t e = bytes ? cudaMemcpyAsync(pipe->lam[sl], lambdas[g], bytes, cudaMemcpyHostToDevice, c)
                              : cudaSuccess;
        return e == cudaSuccess ? cudaEventRecord(pipe->in_ready[sl], c) : e;
    };
    P2P_TRY_CUDA(cudaEventRecord(pipe->start, s), "p2p_apply_host");
    P2P_TRY_CUDA(cudaStreamWaitEvent(c, pipe->start, 0), "p2p_apply_host");
    P2P_TRY_CUDA(upload(0), "p2p_apply_host/upload");
    for (int g = 0; g < count; ++g) {
        const int sl = g & 1;
        if (g + 1 < count) P2P_TRY_CUDA(upload(g + 1), "p2p_apply_host/upload");
        P2P_TRY_CUDA(cudaStreamWaitEvent(s, pipe->in_ready[sl], 0), "p2p_apply_host");
        const p2p_status st = p2p_apply(plans[g], pipe->lam[sl], pipe->out[sl], nrhs, nrhs, stream);
        if (st != P2P_OK) return st;
        P2P_TRY_CUDA(cudaEventRecord(pipe->out_ready[sl], s), "p2p_apply_host");
        P2P_TRY_CUDA(cudaStreamWaitEvent(c, pipe->out_ready[sl], 0), "p2p_apply_host");
        const size_t bytes = (size_t)plans[g]->n * nrhs * 8;
        if (bytes)
            P2P_TRY_CUDA(cudaMemcpyAsync(outs[g], pipe->out[sl], bytes, cudaMemcpyDeviceToHost, c),
                         "p2p_apply_host/download");
    }
    P2P_TRY_CUDA(cudaEventRecord(pipe->done, c), "p2p_apply_host");
    P2P_TRY_CUDA(cudaStreamWaitEvent(s, pipe->done, 0), "p2p_apply_host");
    return P2P_OK;
}

P2P_API p2p_status p2p_host_pipe_destroy(p2p_host_pipe* pipe) {
    if (!pipe) return P2P_OK;
    if (pipe->copy) cudaStreamSynchronize(pipe->copy);
    cudaEvent_t evs[6] = {pipe->start, pipe->done, pipe->in_ready[0], pipe->in_ready[1], pipe->out_ready[0],
                          pipe->out_ready[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (pipe->copy) cudaStreamDestroy(pipe->copy);
    free(pipe);
    return P2P_OK;
}

}  // extern "C"
