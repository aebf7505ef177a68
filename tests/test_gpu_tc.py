"""Tensor-core (tcgen05, BF16 hi/lo) multi-RHS path against the FP64 oracle.

Tolerance: relative L2 error per right-hand side <= 1e-5, the bound the FP32
path meets; the three-product BF16 split (hi.hi + hi.lo + lo.hi) leaves a
per-product error near 2^-17 that averages down over the neighbourhood sums.
The six-product split (hi + mid + lo) is held to the FP32 path's per-target
bound as well: |err_i| <= 2^-20 S_i with S_i = sum_j |G(r_ij) lambda_j|.
"""
import numpy as np
import pytest

import oracle
from paper_2403_01596_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import api
    return api


def rel_l2(x, ref):
    x = np.asarray(x).reshape(ref.shape[0], -1)
    ref = np.asarray(ref).reshape(ref.shape[0], -1)
    return np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)


@pytest.mark.parametrize("n,K", [(16, 64), (64, 128), (256, 192), (48, 320)])
def test_tc_operand_layout(n, K):
    _api()
    from paper_2403_01596_gb300 import _capi as C
    g = torch.Generator().manual_seed(n + K)
    A = torch.randn(128, K, generator=g, dtype=torch.float32)
    B = torch.randn(n, K, generator=g, dtype=torch.float32)
    D = torch.empty(128, n, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    C.p2p_diag_tc_gemm(A.cuda(), B.cuda(), D, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = (A.double() @ B.double().T).numpy()
    err = np.linalg.norm(D.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 2e-5, err


def _sphere(n, ng, seed):
    p = W.unit_sphere(n, seed)
    h = 2.0 / ng
    return W.Workload("sphere", p, (-1.0, -1.0, -1.0), h, ng, 2 * np.pi / (5 * h), seed)


TC_PATHS = ["tc_bf16x3", "tc_bf16x6"]


@pytest.mark.parametrize("path", TC_PATHS)
@pytest.mark.parametrize("nrhs", [16, 24, 64])
@pytest.mark.parametrize("kernel", ["helmholtz", "laplace"])
def test_tc_apply_parity(nrhs, kernel, path):
    api = _api()
    wl = _sphere(20000, 24, 31)
    lam = W.strengths(wl.n, nrhs, 31)
    k = wl.k if kernel == "helmholtz" else 0.0
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, k, kernel=kernel, max_nrhs=nrhs)
    out = plan.apply(torch.from_numpy(lam).cuda(), path=path).cpu().numpy()
    assert plan.async_status() == 0
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, k,
                     kernel=oracle.HELMHOLTZ if kernel == "helmholtz" else oracle.LAPLACE)
    err = rel_l2(out, ref)
    print(f"{kernel} nrhs={nrhs} {path} rel-L2 max {err.max():.3e}")
    assert err.max() <= TOL, err


@pytest.mark.parametrize("path", TC_PATHS)
@pytest.mark.parametrize("nrhs", [96, 200, 256])
def test_tc_several_rhs_blocks(nrhs, path):
    """More than 64 right-hand sides: several RHS blocks share each G tile (at 256 and three parts, one
    pipeline slot per set)."""
    api = _api()
    wl = _sphere(12000, 20, 37)
    lam = W.strengths(wl.n, nrhs, 37)
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, max_nrhs=nrhs)
    out = plan.apply(torch.from_numpy(lam).cuda(), path=path).cpu().numpy()
    assert plan.async_status() == 0
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    err = rel_l2(out, ref)
    print(f"nrhs={nrhs} {path} rel-L2 max {err.max():.3e}")
    assert err.max() <= TOL, err


@pytest.mark.parametrize("path", TC_PATHS)
@pytest.mark.parametrize("n", [1, 2, 7, 33, 500])
def test_tc_tiny_plans_and_single_rhs(n, path):
    """Few points: units with fewer source groups than G sets (padding entries), boxes of one point, and a
    single right-hand side through the tensor-core path (RHS rows padded with zeros)."""
    api = _api()
    rng = np.random.default_rng(n)
    pts = rng.random((n, 3)).astype(np.float32)
    ng = 3
    lo, h, k = (0.0, 0.0, 0.0), 1.0 / ng, 2 * np.pi * 1.5
    plan = api.Plan(torch.from_numpy(pts).cuda(), lo, h, ng, k, max_nrhs=16)
    for nrhs in (1, 16):
        lam = W.strengths(n, nrhs, n + nrhs).reshape(n, nrhs)
        out = plan.apply(torch.from_numpy(lam).cuda(), path=path).cpu().numpy().reshape(n, nrhs)
        assert plan.async_status() == 0
        ref = oracle.p2p(pts, lam, lo, h, ng, k).reshape(n, nrhs)
        if not np.linalg.norm(ref):
            np.testing.assert_array_equal(out, 0)  # no pair with r > 0 (one point, or no neighbouring boxes)
            continue
        assert rel_l2(out, ref).max() <= TOL


def test_tc_dense_boxes_and_adjoint():
    """Boxes with more than 64 targets take several target groups."""
    api = _api()
    wl = W.cube_dense(32768, 0)
    nrhs = 32
    lam = W.strengths(wl.n, nrhs, 5)
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, max_nrhs=nrhs)
    assert plan.info["n"] == wl.n
    out = plan.apply(torch.from_numpy(lam).cuda(), path="tc_bf16x3").cpu().numpy()
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    err = rel_l2(out, ref)
    print("dense cube tensor-core rel-L2 per RHS: max %.3e mean %.3e" % (err.max(), err.mean()))
    assert err.max() <= TOL, err
    adj = plan.apply(torch.from_numpy(lam).cuda(), adjoint=True, path="tc_bf16x3").cpu().numpy()
    ref_adj = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k, adjoint=True)
    assert rel_l2(adj, ref_adj).max() <= TOL


def test_tc_matches_fp32_paths_and_auto_dispatch():
    api = _api()
    wl = _sphere(30000, 28, 33)
    nrhs = 64
    lam = torch.from_numpy(W.strengths(wl.n, nrhs, 33)).cuda()
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, max_nrhs=nrhs)
    tc = plan.apply(lam, path="tc_bf16x3").cpu().numpy()
    auto = plan.apply(lam).cpu().numpy()
    fp = plan.apply(lam, path="fp32_shared").cpu().numpy()
    np.testing.assert_array_equal(auto, tc)  # nrhs >= 16 dispatches to the tensor-core path
    assert rel_l2(tc, fp).max() <= 2 * TOL
    targets = np.random.default_rng(0).choice(wl.n, 500, replace=False)
    ref = oracle.p2p_targets(wl.points, lam.cpu().numpy(), targets, wl.lo, wl.h, wl.ng, wl.k)
    assert rel_l2(tc[targets], ref).max() <= TOL


def test_tc_full_size_ellipsoid_sampled():
    """The 64-RHS workload at full size (2^21 points on the 2:1:1 ellipsoid, 188^3 grid), in the launch
    configuration the benchmark times: sampled targets against the oracle, every RHS."""
    api = _api()
    wl = W.ellipsoid_multirhs()
    nrhs = 64
    lam = W.strengths(wl.n, nrhs, 2).reshape(wl.n, nrhs)
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, max_nrhs=nrhs)
    out = plan.apply(torch.from_numpy(lam).cuda(), path="tc_bf16x3").cpu().numpy()
    assert plan.async_status() == 0
    targets = np.random.default_rng(21).choice(wl.n, 400, replace=False)
    ref = oracle.p2p_targets(wl.points, lam, targets, wl.lo, wl.h, wl.ng, wl.k)
    assert rel_l2(out[targets], ref).max() <= TOL


@pytest.mark.parametrize("path,occupancy", [("tc_bf16x3", 16), ("tc_bf16x6", 32)])
def test_tc_two_target_groups_per_box(path, occupancy):
    """Two units per box on a grid of one CTA per SM (152 SMs: every round of the grid covers whole boxes, and
    the units' target groups rotate between rounds): the hi/lo split's 32-target units on the 2^20-point sphere
    at 16 points per box (max 50), the three-part split's 64-target units at 32 points per box (max 90); sampled
    targets against the oracle, all targets against the FP32 path."""
    api = _api()
    wl = W.sphere_density(occupancy)
    nrhs = 64
    lam = W.strengths(wl.n, nrhs, 12)
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, max_nrhs=nrhs)
    unit = 32 if path == "tc_bf16x3" else 64
    assert unit < int(torch.diff(plan.structure.box_ptr.long()).max().item()) <= 2 * unit
    lam_d = torch.from_numpy(lam).cuda()
    out = plan.apply(lam_d, path=path).cpu().numpy()
    assert plan.async_status() == 0
    fp32 = plan.apply(lam_d, path="fp32_shared").cpu().numpy()
    assert rel_l2(out, fp32).max() <= TOL
    targets = np.random.default_rng(12).choice(wl.n, 300, replace=False)
    ref = oracle.p2p_targets(wl.points, lam, targets, wl.lo, wl.h, wl.ng, wl.k)
    err = rel_l2(out[targets], ref)
    print(f"{path} two target groups per box: rel-L2 max {err.max():.3e}")
    assert err.max() <= TOL


@pytest.mark.parametrize("kernel", ["helmholtz", "laplace"])
def test_tc_six_products_meet_fp32_bound(kernel):
    """Per target and RHS, |err| / S_i of the six-product path stays under the FP32 path's 2^-20 (the
    three-product path's own bound is 2^-14), and its adjoint as well.  S_i is the Laplace sum of |lambda|
    (|exp(ikr)| = 1)."""
    api = _api()
    wl = _sphere(20000, 24, 41)
    nrhs = 32
    lam = W.strengths(wl.n, nrhs, 41)
    # the plan holds k in float32: the oracle takes the same value, so the bound sees arithmetic error only
    k = float(np.float32(wl.k)) if kernel == "helmholtz" else 0.0
    kid = oracle.HELMHOLTZ if kernel == "helmholtz" else oracle.LAPLACE
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, k, kernel=kernel, max_nrhs=nrhs)
    targets = np.random.default_rng(41).choice(wl.n, 600, replace=False)
    S = oracle.p2p_targets(wl.points, np.abs(lam).astype(np.float64), targets, wl.lo, wl.h, wl.ng, 0.0,
                           kernel=oracle.LAPLACE).real
    for adjoint in (False, True):
        ref = oracle.p2p_targets(wl.points, lam, targets, wl.lo, wl.h, wl.ng, k, kernel=kid, adjoint=adjoint)
        worst = {}
        for path in TC_PATHS:
            out = plan.apply(torch.from_numpy(lam).cuda(), adjoint=adjoint, path=path).cpu().numpy()
            assert plan.async_status() == 0
            worst[path] = float((np.abs(out[targets] - ref) / S).max())
        print(f"{kernel} adjoint={adjoint} max |err| / S: {worst}")
        assert worst["tc_bf16x6"] <= 2.0 ** -20, worst
        assert worst["tc_bf16x3"] <= 2.0 ** -14, worst
