"""Failure detection on the GPU without a fault.

The pipelined kernels cap every mbarrier wait; a wait that runs out sets a
status bit and the kernel returns.  Here a wait is made to run out on purpose
(a barrier nothing arrives at, capped at a few thousand polls); the status
word must report it and the context must still run a correct apply afterwards.
Invalid host inputs are rejected with status codes before any launch.
"""
import numpy as np
import pytest

import oracle
from paper_2403_01596_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import _capi as C, api
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    C.p2p_diag_wait_timeout(status, 4096)
    torch.cuda.synchronize()
    assert int(status.item()) & 2
    # the context is intact: a normal apply still matches the oracle
    wl = W.Workload("s", W.unit_sphere(5000, 3), (-1, -1, -1), 2 / 15, 15, 20.0, 3)
    lam = W.strengths(wl.n, 1, 3)
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, layout="redundant")
    out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5
    assert plan.async_status() == 0


def test_host_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import _capi as C, api
    wl = W.Workload("s", W.unit_sphere(2000, 4), (-1, -1, -1), 2 / 10, 10, 20.0, 4)
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, max_nrhs=2)
    lam = torch.zeros(wl.n, 3, dtype=torch.complex64, device="cuda")
    with pytest.raises(C.P2PError):          # nrhs above the plan's maximum
        plan.apply(lam)
    lam = torch.zeros(wl.n, 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(C.P2PError):          # result aliasing the strengths
        C.p2p_apply_path(plan._plan, lam, lam, 2, 2, 0, C.P2P_PATH_AUTO)
    with pytest.raises(C.P2PError):          # ld smaller than nrhs
        C.p2p_apply_path(plan._plan, lam, torch.empty_like(lam), 2, 1, 0, C.P2P_PATH_AUTO)
    with pytest.raises(C.P2PError):
        C.p2p_diag_wait_timeout(torch.zeros(1, dtype=torch.int32, device="cuda"), 0)


def test_tensor_core_abort_path_frees_tensor_memory():
    """The tensor-core kernel's abort path: with every pipeline wait capped at 0, 1 or 3 polls a wait runs out
    (at 0 polls at once; at 1 or 3 polls, when it does, with copies and MMAs in flight), the status word reports
    the timeout, and the block drains its own copies and MMAs and frees its tensor memory -- the next launch
    allocates tensor memory again and, with the normal bound restored, matches the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import _capi as C, api
    wl = W.Workload("s", W.unit_sphere(30000, 5), (-1, -1, -1), 2 / 36, 36, 30.0, 5)
    lam = W.strengths(wl.n, 16, 5)
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, max_nrhs=16)
    lam_d = torch.from_numpy(lam).cuda()

    def rel(out):
        return (np.linalg.norm(out - ref, axis=0) / np.linalg.norm(ref, axis=0)).max()

    assert rel(plan.apply(lam_d, path="tc_bf16x3").cpu().numpy()) <= 1e-5
    assert plan.async_status() == C.P2P_OK
    seen = {}
    for polls in (0, 1, 3):
        C.p2p_diag_tc_wait_limit(plan._plan, polls)
        out = plan.apply(lam_d, path="tc_bf16x3").cpu().numpy()
        st = plan.async_status()
        seen[polls] = st
        if polls == 0:
            assert st == C.P2P_ERR_TIMEOUT
        else:
            assert st in (C.P2P_OK, C.P2P_ERR_TIMEOUT)
            if st == C.P2P_OK:
                assert rel(out) <= 1e-5
    C.p2p_diag_tc_wait_limit(plan._plan, -1)
    for _ in range(2):
        assert rel(plan.apply(lam_d, path="tc_bf16x3").cpu().numpy()) <= 1e-5
        assert plan.async_status() == C.P2P_OK
    print("tensor-core abort path, status per poll bound:", seen)
