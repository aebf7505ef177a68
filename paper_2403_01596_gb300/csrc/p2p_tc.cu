// Multi-RHS tensor-core path (tcgen05, BF16 hi/lo split).  Placeholder until the
// kernel lands: reports the path as unsupported so callers take the FP32 path.
#include "p2p_internal.cuh"

bool p2p_tc_supported(const p2p_plan* plan, int32_t nrhs) {
    (void)plan;
    (void)nrhs;
    return false;
}

p2p_status p2p_apply_tc(const p2p_plan* plan, const float2* lam_sorted, float2* out, int32_t nrhs, int64_t ld,
                        int32_t adjoint, cudaStream_t s) {
    (void)plan; (void)lam_sorted; (void)out; (void)nrhs; (void)ld; (void)adjoint; (void)s;
    return P2P_ERR_UNSUPPORTED;
}
