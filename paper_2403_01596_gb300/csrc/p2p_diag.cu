// Self-check of the bounded-wait mechanism used by the pipelined kernels.
//
// One warp initialises an mbarrier that expects one arrival and then waits on
// it with the same bounded poll loop the pair and tensor-core kernels use --
// but nothing ever arrives.  The wait gives up after `limit` polls, the kernel
// records P2P_DEV_TIMEOUT in the status word and returns, and the context
// stays usable.  This exercises the timeout path without faulting the GPU.
#include "p2p_pair.cuh"

namespace {

__global__ void k_wait_timeout(unsigned int* __restrict__ status, uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        p2p_pair::mbar_init(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool ok = p2p_pair::mbar_wait(&bar, 0u, limit);
    if (!__all_sync(P2P_FULL_MASK, ok) && threadIdx.x == 0) atomicOr(status, P2P_DEV_TIMEOUT);
}

}  // namespace

extern "C" P2P_API p2p_status p2p_diag_wait_timeout(unsigned int* status, int32_t limit, p2p_stream_t stream) {
    if (!status || limit < 1) return P2P_ERR_INVALID;
    k_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(status, (uint32_t)limit);
    P2P_CHECK_LAUNCH("p2p_diag_wait_timeout");
    return P2P_OK;
}
