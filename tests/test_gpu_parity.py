"""GPU parity of the CUDA path against the FP64 oracle (call through the C ABI).

Tolerances (FP32 kernel vs FP64 oracle): relative L2 error per right-hand
side <= 1e-5 for potentials and for the coordinate gradient; box ids,
permutation, box pointers and neighbour lists bit-exact.  Where a test also
checks targets one by one, the error of target i is measured against
S_i = sum_j |G(r_ij) lambda_j| (the sum of the magnitudes of its terms, i.e. the
oracle's Laplace sum of |lambda|, since |exp(ikr)| = 1): an FP32 evaluation
whose every term is accurate to a few units of 2^-24 has
|out_i - ref_i| <= c 2^-24 S_i however much the terms cancel, so
max_i |out_i - ref_i| / S_i <= 2e-6 is asserted and the plain per-target
maximum relative error is printed beside it.
"""
import numpy as np
import pytest

import oracle
from paper_2403_01596_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import api
    return api


def rel_l2(x, ref):
    x = np.asarray(x).reshape(ref.shape[0], -1)
    ref = np.asarray(ref).reshape(ref.shape[0], -1)
    return np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)


def per_target(out, ref, wl, lam, kernel=None):
    """(max over targets of |out - ref| / S_i, max over targets of |out - ref| / |ref|), see the docstring."""
    absl = np.abs(np.asarray(lam)).astype(np.float64)
    S = oracle.p2p(wl.points, absl, wl.lo, wl.h, wl.ng, 0.0, kernel=oracle.LAPLACE).real
    S = S.reshape(S.shape[0], -1)
    d = np.abs(np.asarray(out).reshape(S.shape[0], -1) - np.asarray(ref).reshape(S.shape[0], -1))
    r = np.abs(np.asarray(ref).reshape(S.shape[0], -1))
    ok = S > 0
    return float((d[ok] / S[ok]).max()), float((d[r > 0] / r[r > 0]).max())


def _plan(api, wl, kernel="helmholtz", layout="indexed", max_nrhs=1, tuning=None, k=None):
    pts = torch.from_numpy(wl.points).cuda()
    return api.Plan(pts, wl.lo, wl.h, wl.ng, wl.k if k is None else k, kernel=kernel, layout=layout,
                    max_nrhs=max_nrhs, tuning=tuning)


def _small_sphere(n=40000, ng=40, seed=5):
    p = W.unit_sphere(n, seed)
    return W.Workload(f"sphere{n}", p, (-1.0, -1.0, -1.0), 2.0 / ng, ng, 2 * np.pi / (4 * 2.0 / ng), seed)


def _clustered(n=30000, seed=12):
    p = W.cylinder_plates(n, seed)
    ng = 48
    h = 2.6 / ng
    return W.Workload("clustered", p, (-1.3, -1.3, -1.3), h, ng, 2 * np.pi * 0.2 / h, seed)


STRUCT_CASES = {
    "cube8": lambda: W.cube_dense(),
    "sphere40": lambda: _small_sphere(),
    "clustered": lambda: _clustered(),
    "ellipsoid": lambda: W.Workload("ell", W.ellipsoid_211(20000, 7), (-2.0, -2.0, -2.0), 4.0 / 37, 37, 10.0, 7),
}


@pytest.mark.parametrize("case", sorted(STRUCT_CASES))
def test_binning_and_neighbors_bit_exact(case):
    api = _cuda()
    wl = STRUCT_CASES[case]()
    st = api.BoxStructure(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng)
    ref = oracle.bin_points(wl.points, wl.lo, wl.h, wl.ng)
    assert st.num_boxes == ref["num_boxes"]
    np.testing.assert_array_equal(st.perm.cpu().numpy()[:wl.n], ref["perm"])
    np.testing.assert_array_equal(st.point_box.cpu().numpy()[:wl.n], ref["point_box"])
    np.testing.assert_array_equal(st.box_keys.cpu().numpy(), ref["box_keys"])
    np.testing.assert_array_equal(st.box_ptr.cpu().numpy(), ref["box_ptr"])
    nptr, nidx = oracle.neighbors(ref["box_keys"], wl.ng)
    np.testing.assert_array_equal(st.nbr_ptr.cpu().numpy(), nptr)
    np.testing.assert_array_equal(st.nbr_idx.cpu().numpy()[:st.nnz], nidx)
    sizes = np.diff(ref["box_ptr"])
    assert st.sources == int(sum(sizes[nidx[nptr[b]:nptr[b + 1]]].sum() for b in range(ref["num_boxes"])))


@pytest.mark.parametrize("kernel", ["helmholtz", "laplace"])
@pytest.mark.parametrize("layout", ["indexed", "redundant", "symmetric"])
def test_apply_dense_cube(kernel, layout):
    """Uniform cube, 8^3 boxes (~64 points per box, ~1350 sources per box: several chunks)."""
    api = _cuda()
    wl = W.cube_dense()
    lam = W.strengths(wl.n, 1, wl.seed)
    plan = _plan(api, wl, kernel, layout)
    out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
    kern = oracle.HELMHOLTZ if kernel == "helmholtz" else oracle.LAPLACE
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k if kernel == "helmholtz" else 0.0, kernel=kern)
    err = rel_l2(out, ref)
    assert err.max() <= TOL, err
    assert plan.async_status() == 0
    assert plan.pair_count() == oracle.pair_count(wl.points, wl.lo, wl.h, wl.ng)


@pytest.mark.parametrize("layout", ["indexed", "redundant", "symmetric"])
@pytest.mark.parametrize("case", ["sphere40", "clustered", "ellipsoid"])
def test_apply_surfaces(layout, case):
    api = _cuda()
    wl = STRUCT_CASES[case]()
    lam = W.strengths(wl.n, 1, wl.seed)
    plan = _plan(api, wl, "helmholtz", layout)
    out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    err = rel_l2(out, ref).max()
    normwise, relmax = per_target(out, ref, wl, lam)
    print(f"{case} {layout}: rel-L2 {err:.2e}, max |err|/S {normwise:.2e}, max per-target relative {relmax:.2e}")
    assert err <= TOL
    assert normwise <= 2e-6


@pytest.mark.parametrize("edge", [1.0, 2.0, 4.0])
@pytest.mark.parametrize("layout", ["indexed", "redundant"])
def test_apply_high_frequency(edge, layout):
    """Leaf edges of 1, 2 and 4 wavelengths (k r up to 22, 44 and 87 rad inside a neighbourhood): the FP32
    phase k * r carries a relative error of a few 2^-24, i.e. an absolute phase error that grows with k r, so
    the error grows with the leaf size in wavelengths; up to 4 wavelengths it stays within the tolerance."""
    api = _cuda()
    n, ng = 24000, 12
    wl = W.Workload(f"cube_hf{edge}", W.uniform_cube(n, 31), (0.0, 0.0, 0.0), 1.0 / ng, ng, 2 * np.pi * edge * ng, 31)
    lam = W.strengths(n, 1, 31)
    plan = _plan(api, wl, "helmholtz", layout)
    out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    err = rel_l2(out, ref).max()
    normwise, relmax = per_target(out, ref, wl, lam)
    print(f"leaf edge {edge} wavelengths, {layout}: rel-L2 {err:.2e}, max |err|/S {normwise:.2e}, "
          f"max per-target relative {relmax:.2e}")
    assert err <= TOL


@pytest.mark.parametrize("tuning", [{"chunk": 32, "warps_per_cta": 4, "target_group": 32, "warp_boxes": -1},
                                    {"chunk": 64, "warps_per_cta": 1, "target_group": 64, "warp_boxes": -1},
                                    {"chunk": 256, "warps_per_cta": 16, "target_group": 128, "warp_boxes": -1},
                                    {"chunk": 1024, "warps_per_cta": 2, "target_group": 96, "warp_boxes": -1},
                                    {"warp_boxes": 1}, {"warp_boxes": 4}, {"warp_boxes": 32}])
def test_apply_tunings(tuning):
    api = _cuda()
    wl = _clustered(12000, 13)
    lam = W.strengths(wl.n, 1, 3)
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    for layout in ("indexed", "redundant", "symmetric"):
        plan = _plan(api, wl, "helmholtz", layout, tuning=tuning)
        out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
        assert rel_l2(out, ref).max() <= TOL, (layout, tuning)
        want = -1 if layout == "symmetric" else tuning["warp_boxes"]
        assert plan.info["tuning"]["warp_boxes"] == want


@pytest.mark.parametrize("warp_boxes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("kernel", ["helmholtz", "laplace"])
@pytest.mark.parametrize("layout", ["indexed", "redundant"])
def test_direct_kernel(warp_boxes, kernel, layout):
    """The direct kernel (1 - 32 whole boxes per warp, sources read through the L1) on the dense cube (boxes
    of ~64 targets: several passes per box at 8 lanes or fewer per box), a sparse sphere and the clustered assembly
    (occupancy 1 - 128), forward and adjoint; every result row is stored once (the output starts as garbage)."""
    api = _cuda()
    kern = oracle.HELMHOLTZ if kernel == "helmholtz" else oracle.LAPLACE
    for wl in (W.cube_dense(), _small_sphere(30000, 48, 22), _clustered(20000, 23)):
        k = wl.k if kernel == "helmholtz" else 0.0
        lam = W.strengths(wl.n, 1, 24)
        plan = _plan(api, wl, kernel, layout, tuning={"warp_boxes": warp_boxes}, k=k)
        assert plan.info["tuning"]["warp_boxes"] == warp_boxes
        for adjoint in (False, True):
            out = torch.full((wl.n, 1), 5.0 - 3.0j, dtype=torch.complex64, device="cuda")
            plan.apply(torch.from_numpy(lam).cuda(), out=out, adjoint=adjoint)
            ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, k, kernel=kern, adjoint=adjoint)
            err = rel_l2(out.cpu().numpy(), ref).max()
            assert err <= TOL, (wl.name, adjoint, err)
        assert plan.async_status() == 0


@pytest.mark.parametrize("kernel", ["helmholtz", "laplace"])
def test_group_kernel(kernel):
    """The box-group kernel (tuning warp_boxes = -2: groups of sixteen consecutive boxes stage the union of their
    neighbourhoods once; every box sweeps its own neighbour boxes as segments of that buffer): dense cube (64
    targets per box, a 4 096-source union), sparse sphere, clustered assembly (occupancy 1 - 128) and the edge
    case of one 700-point box (several passes of 128 targets), forward and adjoint, output rows stored once
    (the output starts as garbage); per target within 2e-6 of S_i."""
    api = _cuda()
    kern = oracle.HELMHOLTZ if kernel == "helmholtz" else oracle.LAPLACE
    rng = np.random.default_rng(4)
    p = np.concatenate([rng.random((700, 3)) * 0.1 + 0.45, rng.random((300, 3)) * 1.4 - 0.2]).astype(np.float32)
    p[10] = p[11]
    p[20] = p[21] = p[22]
    edge = W.Workload("edge", p, (0, 0, 0), 0.125, 8, 9.0, 0)
    for wl in (W.cube_dense(), _small_sphere(30000, 48, 22), _clustered(20000, 23), edge):
        k = wl.k if kernel == "helmholtz" else 0.0
        lam = W.strengths(wl.n, 1, 24)
        plan = _plan(api, wl, kernel, "indexed", tuning={"warp_boxes": -2}, k=k)
        assert plan.info["tuning"]["warp_boxes"] == -2, wl.name
        for adjoint in (False, True):
            out = torch.full((wl.n, 1), 5.0 - 3.0j, dtype=torch.complex64, device="cuda")
            plan.apply(torch.from_numpy(lam).cuda(), out=out, adjoint=adjoint)
            ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, k, kernel=kern, adjoint=adjoint)
            got = out.cpu().numpy()
            err = rel_l2(got, ref).max()
            normwise, rel = per_target(got, ref, wl, lam)
            print(f"group kernel {wl.name} {kernel} adjoint={adjoint}: rel-L2 {err:.2e}, max |err|/S {normwise:.2e}")
            assert err <= TOL and normwise <= 2e-6, (wl.name, adjoint, err, normwise)
        assert plan.async_status() == 0
    # the redundant layout keeps its own kernels
    plan = _plan(api, W.cube_dense(), kernel, "redundant", tuning={"warp_boxes": -2})
    assert plan.info["tuning"]["warp_boxes"] == -1
    # a union beyond the kernel's 8 192-source buffer: the plan reports and runs the staged pipeline
    # (4^3 boxes of ~256 points: a group of 16 boxes has a union of at least 36 boxes, ~9 200 sources)
    dense = W.Workload("dense4", W.uniform_cube(16384, 7), (0.0, 0.0, 0.0), 0.25, 4, 2 * np.pi * 2, 7)
    lamd = W.strengths(dense.n, 1, 7)
    kd = dense.k if kernel == "helmholtz" else 0.0
    plan = _plan(api, dense, kernel, "indexed", tuning={"warp_boxes": -2}, k=kd)
    assert plan.info["tuning"]["warp_boxes"] == -1
    out = plan.apply(torch.from_numpy(lamd).cuda()).cpu().numpy()
    assert rel_l2(out, oracle.p2p(dense.points, lamd, dense.lo, dense.h, dense.ng, kd, kernel=kern)).max() <= TOL
    # a plan left to choose takes the box-group kernel at 12 < D <= 24 (here ~18 points per box)
    p18 = W.unit_sphere(20000, 4)
    wl18 = W.Workload("sphere18", p18, (-1.0, -1.0, -1.0), 2.0 / 16, 16, 2 * np.pi / (4 * 2.0 / 16), 4)
    plan = _plan(api, wl18, kernel, "indexed", k=wl18.k if kernel == "helmholtz" else 0.0)
    assert plan.info["tuning"]["warp_boxes"] == -2


@pytest.mark.parametrize("path", ["fp32_per_rhs", "fp32_shared"])
@pytest.mark.parametrize("nrhs", [2, 3, 5, 8])
def test_multi_rhs(path, nrhs):
    api = _cuda()
    wl = _small_sphere(20000, 30, 8)
    lam = W.strengths(wl.n, nrhs, 8)
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    for layout in ("indexed", "redundant", "symmetric"):
        plan = _plan(api, wl, "helmholtz", layout, max_nrhs=nrhs)
        out = plan.apply(torch.from_numpy(lam).cuda(), path=path).cpu().numpy()
        err = rel_l2(out, ref)
        assert err.shape == (nrhs,) and err.max() <= TOL, err


def test_adjoint():
    api = _cuda()
    wl = _small_sphere(30000, 36, 9)
    g = W.strengths(wl.n, 2, 9)
    for layout in ("indexed", "redundant", "symmetric"):
        plan = _plan(api, wl, "helmholtz", layout, max_nrhs=2)
        out = plan.apply(torch.from_numpy(g).cuda(), adjoint=True).cpu().numpy()
        ref = oracle.p2p(wl.points, g, wl.lo, wl.h, wl.ng, wl.k, adjoint=True)
        assert rel_l2(out, ref).max() <= TOL


@pytest.mark.parametrize("kernel", ["helmholtz", "laplace"])
def test_grad_points(kernel):
    api = _cuda()
    wl = W.sphere_grad(1 << 15, 3)
    wl = W.Workload(wl.name, wl.points, wl.lo, 2.0 / 22, 22, 2 * np.pi * 3, 3)
    lam = W.strengths(wl.n, 1, 3)
    g = W.strengths(wl.n, 1, 4)
    plan = _plan(api, wl, kernel, "indexed")
    kern = oracle.HELMHOLTZ if kernel == "helmholtz" else oracle.LAPLACE
    k = wl.k if kernel == "helmholtz" else 0.0
    gx = plan.grad_points(torch.from_numpy(lam).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    ref = oracle.grad_points(wl.points, lam, g, wl.lo, wl.h, wl.ng, k, kernel=kern)
    err = np.linalg.norm(gx - ref) / np.linalg.norm(ref)
    print(f"coordinate gradient ({kernel}): rel-L2 {err:.3e}")
    assert err <= TOL, err


@pytest.mark.parametrize("layout,nrhs,tuning", [("indexed", 1, None), ("redundant", 1, None),
                                                 ("indexed", 1, {"chunk": 64, "warps_per_cta": 4}),
                                                 ("redundant", 3, None), ("indexed", 2, {"chunk": 64})])
def test_grad_points_layouts_rhs_and_chunks(layout, nrhs, tuning):
    """Both layouts' box lists, one and several right-hand sides (summed as the oracle does), and boxes split
    over several items when the chunk is short (their partial gradients meet in the atomic output)."""
    api = _cuda()
    wl = W.Workload("grad_ell", W.ellipsoid_211(12000, 17), (-2.0, -2.0, -2.0), 4.0 / 30, 30, 9.0, 17)
    lam = W.strengths(wl.n, nrhs, 18).reshape(wl.n, nrhs)
    g = W.strengths(wl.n, nrhs, 19).reshape(wl.n, nrhs)
    plan = _plan(api, wl, "helmholtz", layout, max_nrhs=nrhs, tuning=tuning)
    gx = plan.grad_points(torch.from_numpy(lam).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    assert plan.async_status() == 0
    ref = oracle.grad_points(wl.points, lam, g, wl.lo, wl.h, wl.ng, wl.k)
    assert np.linalg.norm(gx - ref) / np.linalg.norm(ref) <= TOL


def test_autograd_function():
    api = _cuda()
    wl = _small_sphere(8000, 20, 14)
    pts = torch.from_numpy(wl.points).cuda().requires_grad_(True)
    plan = api.Plan(pts.detach(), wl.lo, wl.h, wl.ng, wl.k)
    lam = torch.from_numpy(W.strengths(wl.n, 1, 14)).cuda().requires_grad_(True)
    b = torch.from_numpy(W.strengths(wl.n, 1, 15)).cuda()
    out = api.p2p(lam, pts, plan)
    loss = (out - b).abs().pow(2).sum()
    loss.backward()
    g = 2 * (out.detach() - b)
    ref_lam = oracle.p2p(wl.points, g.cpu().numpy(), wl.lo, wl.h, wl.ng, wl.k, adjoint=True)
    assert rel_l2(lam.grad.cpu().numpy(), ref_lam).max() <= TOL
    ref_x = oracle.grad_points(wl.points, lam.detach().cpu().numpy(), g.cpu().numpy(), wl.lo, wl.h, wl.ng, wl.k)
    assert np.linalg.norm(pts.grad.cpu().numpy() - ref_x) / np.linalg.norm(ref_x) <= TOL


def test_edge_cases():
    api = _cuda()
    # one point: no pairs, zero output
    one = W.Workload("one", np.array([[0.3, 0.3, 0.3]], np.float32), (0, 0, 0), 0.5, 2, 3.0, 0)
    plan = _plan(api, one)
    out = plan.apply(torch.ones(1, dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert out[0] == 0
    # empty point set
    empty = W.Workload("empty", np.zeros((0, 3), np.float32), (0, 0, 0), 0.5, 2, 3.0, 0)
    plan = _plan(api, empty)
    assert plan.apply(torch.zeros(0, dtype=torch.complex64, device="cuda")).numel() == 0
    # duplicates, points outside the grid, one dense box of 700 points (> target group, > chunk)
    rng = np.random.default_rng(4)
    p = np.concatenate([rng.random((700, 3)) * 0.1 + 0.45, rng.random((300, 3)) * 1.4 - 0.2])
    p = p.astype(np.float32)
    p[10] = p[11]
    p[20] = p[21] = p[22]
    wl = W.Workload("edge", p, (0, 0, 0), 0.125, 8, 9.0, 0)
    lam = W.strengths(len(p), 1, 4)
    ref = oracle.p2p(p, lam, wl.lo, wl.h, wl.ng, wl.k)
    for layout in ("indexed", "redundant", "symmetric"):
        for tuning in (None, {"chunk": 32, "target_group": 32, "warp_boxes": -1},
                       {"chunk": 256, "target_group": 128, "warp_boxes": -1}, {"warp_boxes": 4}, {"warp_boxes": 1}):
            plan = _plan(api, wl, "helmholtz", layout, tuning=tuning)
            out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
            assert rel_l2(out, ref).max() <= TOL
    assert plan.pair_count() == oracle.pair_count(p, wl.lo, wl.h, wl.ng)
    # ng = 1: a single box, the dense all-pairs case
    wl1 = W.Workload("single", W.uniform_cube(3000, 5), (0, 0, 0), 1.0, 1, 6.0, 0)
    lam1 = W.strengths(3000, 1, 5)
    out = _plan(api, wl1).apply(torch.from_numpy(lam1).cuda()).cpu().numpy()
    assert rel_l2(out, oracle.p2p(wl1.points, lam1, (0, 0, 0), 1.0, 1, 6.0)).max() <= TOL


def test_invalid_points_rejected():
    api = _cuda()
    from paper_2403_01596_gb300._capi import P2PError
    p = W.uniform_cube(100, 1)
    p[17, 1] = np.nan
    with pytest.raises(P2PError):
        api.BoxStructure(torch.from_numpy(p).cuda(), (0, 0, 0), 0.25, 4)


@pytest.mark.parametrize("occ", [8, 64])
def test_full_size_sphere_sampled(occ):
    """Bench workload at full size (2^20 points on the sphere): bit-exact structure, sampled outputs."""
    api = _cuda()
    wl = W.sphere_density(occ)
    lam = W.strengths(wl.n, 1, wl.seed)
    ref_bins = oracle.bin_points(wl.points, wl.lo, wl.h, wl.ng)
    targets = np.random.default_rng(occ).choice(wl.n, 3000, replace=False)
    ref = oracle.p2p_targets(wl.points, lam, targets, wl.lo, wl.h, wl.ng, wl.k)
    for layout in ("indexed", "redundant", "symmetric"):
        plan = _plan(api, wl, "helmholtz", layout)
        assert plan.num_boxes == ref_bins["num_boxes"]
        np.testing.assert_array_equal(plan.structure.perm.cpu().numpy(), ref_bins["perm"])
        out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
        assert rel_l2(out[targets], ref).max() <= TOL


def test_symmetric_plan_refuses_gradients():
    api = _cuda()
    from paper_2403_01596_gb300._capi import P2PError
    wl = _small_sphere(3000, 12, 21)
    plan = _plan(api, wl, "helmholtz", "symmetric")
    lam = torch.from_numpy(W.strengths(wl.n, 1, 21)).cuda()
    with pytest.raises(P2PError):
        plan.grad_points(lam, lam)
