"""Near field between separate target and source point sets (Sec. 3.1 keeps
target and source coordinates as separate arrays), CUDA path against the FP64
oracle's two-set sum, through the C ABI.

Both sets are binned on one grid; the neighbours of a target box are the
source boxes within Chebyshev cell distance 1; a target and a source at the
same position (r = 0) are skipped.  Binning and neighbour lists (with the
position of each target box's own-cell source box) are compared bit-exactly,
results at relative L2 <= 1e-5 per right-hand side.
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


def _cube_case():
    """Targets and sources uniform in the unit cube (different sizes and seeds), a third of the targets placed
    on source positions (r = 0 pairs), 8^3 boxes, k = 8 pi."""
    t = W.uniform_cube(20000, 51)
    s = W.uniform_cube(31000, 52)
    t[::3] = s[: len(t[::3])]
    return t, s, (0.0, 0.0, 0.0), 1.0 / 8, 8, 8 * np.pi


def _sphere_case():
    """Targets on the unit sphere; sources on the part x > -0.3 of a sphere of radius 0.97 and on the cap
    z > 0.5 of the unit sphere: target boxes with a source box in their own cell (the cap), target boxes whose
    nearby sources all lie in other cells, and target boxes with no source nearby at all (x < -0.4, z < 0.4)."""
    t = W.unit_sphere(40000, 53)
    s1 = W.unit_sphere(25000, 54) * np.float32(0.97)
    s1 = s1[s1[:, 0] > -0.3]
    s2 = W.unit_sphere(20000, 55)
    s2 = s2[s2[:, 2] > 0.5]
    s = np.ascontiguousarray(np.concatenate([s1, s2]).astype(np.float32))
    ng = 40
    return t, s, (-1.0, -1.0, -1.0), 2.0 / ng, ng, 2 * np.pi / (4 * 2.0 / ng)


CASES = {"cube": _cube_case, "sphere": _sphere_case}


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_set_structure_bit_exact(case):
    api = _api()
    t, s, lo, h, ng, _ = CASES[case]()
    st = api.TwoSetStructure(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), lo, h, ng)
    rt, rs = oracle.bin_points(t, lo, h, ng), oracle.bin_points(s, lo, h, ng)
    assert st.tgt.num_boxes == rt["num_boxes"] and st.src.num_boxes == rs["num_boxes"]
    np.testing.assert_array_equal(st.tgt.perm.cpu().numpy()[:len(t)], rt["perm"])
    np.testing.assert_array_equal(st.src.box_ptr.cpu().numpy(), rs["box_ptr"])
    nptr, nidx = oracle.neighbors_st(rt["box_keys"], rs["box_keys"], ng)
    np.testing.assert_array_equal(st.nbr_ptr.cpu().numpy(), nptr)
    np.testing.assert_array_equal(st.nbr_idx.cpu().numpy()[:st.nnz], nidx)
    # own-cell source box: its key equals the target box's key
    tk, sk = rt["box_keys"], rs["box_keys"]
    self_ref = np.full(len(tk), -1)
    for b in range(len(tk)):
        lst = nidx[nptr[b]:nptr[b + 1]]
        hit = np.nonzero(sk[lst] == tk[b])[0]
        if hit.size:
            self_ref[b] = hit[0]
    np.testing.assert_array_equal(st.nbr_self.cpu().numpy()[:len(tk)], self_ref)
    sizes = np.diff(rs["box_ptr"])
    assert st.sources == int(sum(sizes[nidx[nptr[b]:nptr[b + 1]]].sum() for b in range(len(tk))))
    if case == "sphere":
        assert (self_ref < 0).sum() > 0 and (np.diff(nptr) == 0).sum() > 0  # the edge cases are present


@pytest.mark.parametrize("layout", ["indexed", "redundant", "indexed_groups"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_two_set_apply(case, layout):
    """indexed_groups: the box-group kernel (tuning warp_boxes = -2)."""
    api = _api()
    t, s, lo, h, ng, k = CASES[case]()
    lam = W.strengths(len(s), 1, 56)
    tuning = {"warp_boxes": -2} if layout == "indexed_groups" else None
    plan = api.TwoSetPlan(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), lo, h, ng, k,
                          layout=layout.replace("_groups", ""), tuning=tuning)
    if tuning:
        assert plan.info["tuning"]["warp_boxes"] == -2
    out = torch.full((len(t),), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")  # every row must be written
    plan.apply(torch.from_numpy(lam).cuda(), out=out.reshape(-1, 1))
    ref = oracle.p2p_st(t, s, lam, lo, h, ng, k)
    err = rel_l2(out.cpu().numpy(), ref).max()
    print(f"two sets, {case} {layout}: rel-L2 {err:.2e}")
    assert err <= TOL
    assert plan.async_status() == 0
    # pair count: n_b * S_b over target boxes minus coincident (target, source) pairs
    rt, rs = oracle.bin_points(t, lo, h, ng), oracle.bin_points(s, lo, h, ng)
    nptr, nidx = oracle.neighbors_st(rt["box_keys"], rs["box_keys"], ng)
    sizes = np.diff(rs["box_ptr"])
    per_box = np.array([sizes[nidx[nptr[b]:nptr[b + 1]]].sum() for b in range(rt["num_boxes"])])
    same = np.intersect1d(t.view(np.dtype((np.void, 12))).ravel(), s.view(np.dtype((np.void, 12))).ravel()).size
    assert same == 0 or case == "cube"
    dup = sum(int(np.all(s == row, axis=1).sum()) for row in t[::3]) if case == "cube" else 0
    assert plan.pair_count() == int(per_box[rt["point_box"]].sum()) - dup


@pytest.mark.parametrize("path,nrhs", [("fp32_per_rhs", 3), ("fp32_shared", 5), ("tc_bf16x3", 16),
                                       ("tc_bf16x3", 64)])
def test_two_set_multi_rhs_and_laplace(path, nrhs):
    api = _api()
    t, s, lo, h, ng, k = _sphere_case()
    lam = W.strengths(len(s), nrhs, 57)
    for kernel in ("helmholtz", "laplace"):
        plan = api.TwoSetPlan(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), lo, h, ng, k, kernel=kernel,
                              max_nrhs=nrhs)
        out = plan.apply(torch.from_numpy(lam).cuda(), path=path).cpu().numpy()
        ref = oracle.p2p_st(t, s, lam, lo, h, ng, k if kernel == "helmholtz" else 0.0,
                            kernel=oracle.HELMHOLTZ if kernel == "helmholtz" else oracle.LAPLACE)
        err = rel_l2(out, ref)
        assert err.shape == (nrhs,) and err.max() <= TOL, (kernel, err.max())
        assert plan.async_status() == 0


def test_two_set_adjoint_and_refusals():
    api = _api()
    from paper_2403_01596_gb300._capi import P2PError
    t, s, lo, h, ng, k = _cube_case()
    plan = api.TwoSetPlan(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), lo, h, ng, k, max_nrhs=2)
    g = W.strengths(len(t), 2, 58)
    adj = plan.adjoint_plan().apply(torch.from_numpy(g).cuda(), adjoint=True).cpu().numpy()
    ref = oracle.p2p_st(s, t, g, lo, h, ng, k, conj=True)
    assert rel_l2(adj, ref).max() <= TOL
    # <A lam, g> = <lam, A^H g>
    lam = W.strengths(len(s), 2, 59)
    fwd = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(g.astype(np.complex128), fwd)
    rhs = np.vdot(adj.astype(np.complex128), lam.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    from paper_2403_01596_gb300 import _capi as C
    with pytest.raises(P2PError):
        out = torch.empty((len(t), 2), dtype=torch.complex64, device="cuda")
        C.p2p_apply_adjoint(plan._plan, torch.from_numpy(g).cuda(), out, 2, 2)
    with pytest.raises(P2PError):
        api.TwoSetPlan(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), lo, h, ng, k, layout="symmetric")


def test_two_set_batch_and_host_pipe():
    api = _api()
    t, s, lo, h, ng, k = _sphere_case()
    t2, s2, lo2, h2, ng2, k2 = _cube_case()
    plans = [api.TwoSetPlan(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), lo, h, ng, k, max_nrhs=2),
             api.TwoSetPlan(torch.from_numpy(t2).cuda(), torch.from_numpy(s2).cuda(), lo2, h2, ng2, k2, max_nrhs=2,
                            layout="redundant")]
    lams = [W.strengths(len(s), 2, 60), W.strengths(len(s2), 2, 61)]
    refs = [oracle.p2p_st(t, s, lams[0], lo, h, ng, k), oracle.p2p_st(t2, s2, lams[1], lo2, h2, ng2, k2)]
    batch = api.Batch(plans, nrhs=2)
    outs = [torch.full((p.n, 2), 3.0 + 0j, dtype=torch.complex64, device="cuda") for p in plans]
    batch.apply([torch.from_numpy(l).cuda() for l in lams], outs)
    for o, r in zip(outs, refs):
        assert rel_l2(o.cpu().numpy(), r).max() <= TOL
    pipe = api.HostPipe(max(max(p.n, p.n_src) for p in plans), 2)
    host_out = [torch.empty((p.n, 2), dtype=torch.complex64).pin_memory() for p in plans]
    pipe.apply(plans, [torch.from_numpy(l).pin_memory() for l in lams], host_out)
    torch.cuda.synchronize()
    for o, r in zip(host_out, refs):
        assert rel_l2(o.numpy(), r).max() <= TOL


def test_two_set_without_sources_nearby():
    """Targets far from every source get zero; an empty source set gives zeros everywhere."""
    api = _api()
    t = W.uniform_cube(3000, 62) * np.float32(0.3)
    s = W.uniform_cube(4000, 63) * np.float32(0.3) + np.float32(0.7)
    lo, h, ng, k = (0, 0, 0), 0.1, 10, 5.0
    lam = W.strengths(len(s), 1, 63)
    plan = api.TwoSetPlan(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), lo, h, ng, k)
    out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
    assert np.all(out == 0) and plan.pair_count() == 0
    empty = np.zeros((0, 3), np.float32)
    plan0 = api.TwoSetPlan(torch.from_numpy(t).cuda(), torch.from_numpy(empty).cuda(), lo, h, ng, k)
    out0 = plan0.apply(torch.zeros(0, dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert out0.shape == (len(t),) and np.all(out0 == 0)
