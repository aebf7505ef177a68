"""The paper's own repetition layout (Sec. 3.3): one thread per target reading
its own contiguous record (its coordinates, then a copy of every source of its
box's neighbourhood), strengths repacked into the records at every apply.
CUDA path against the FP64 oracle at relative L2 <= 1e-5; record sizes against
the paper's count, sum over boxes of n_b (1 + S_b)."""
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
    return np.linalg.norm(np.asarray(x) - ref) / np.linalg.norm(ref)


def _plate(n, ng, seed):
    """n points uniform on the square z = 0.5 of the unit cube (the paper's plate), ng^3 grid."""
    rng = np.random.default_rng(seed)
    p = np.concatenate([rng.random((n, 2)), np.full((n, 1), 0.5)], axis=1).astype(np.float32)
    return W.Workload(f"plate{n}", p, (0.0, 0.0, 0.0), 1.0 / ng, ng, 2 * np.pi * 0.25 * ng, seed)


CASES = {
    "cube": lambda: W.cube_dense(8192, 3),
    "plate": lambda: _plate(16384, 64, 4),
    "sphere": lambda: W.Workload("s", W.unit_sphere(20000, 5), (-1, -1, -1), 2 / 32, 32, 2 * np.pi / (4 * 2 / 32), 5),
}


@pytest.mark.parametrize("kernel", ["helmholtz", "laplace"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_repetition_layout(case, kernel):
    api = _api()
    wl = CASES[case]()
    k = wl.k if kernel == "helmholtz" else 0.0
    kern = oracle.HELMHOLTZ if kernel == "helmholtz" else oracle.LAPLACE
    lam = W.strengths(wl.n, 1, 6)
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, k, kernel=kernel, layout="repetition")
    # the paper's record count: every target holds its own box's sources and its neighbours', plus itself
    b = oracle.bin_points(wl.points, wl.lo, wl.h, wl.ng)
    nptr, nidx = oracle.neighbors(b["box_keys"], wl.ng)
    sizes = np.diff(b["box_ptr"])
    S = np.add.reduceat(sizes[nidx], nptr[:-1])
    assert plan.records == int((sizes * (1 + S)).sum())
    for adjoint in (False, True):
        out = torch.full((wl.n, 1), 9.0 + 9.0j, dtype=torch.complex64, device="cuda")
        plan.apply(torch.from_numpy(lam).cuda(), out=out, adjoint=adjoint)
        ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, k, kernel=kern, adjoint=adjoint)
        assert rel_l2(out.cpu().numpy().ravel(), ref) <= TOL
    assert plan.async_status() == 0


def test_repetition_edge_cases_and_other_calls():
    api = _api()
    from paper_2403_01596_gb300._capi import P2PError
    rng = np.random.default_rng(8)
    p = np.concatenate([rng.random((300, 3)) * 0.1 + 0.45, rng.random((200, 3))]).astype(np.float32)
    p[5] = p[6]  # a duplicate point: r = 0 pair skipped
    wl = W.Workload("edge", p, (0, 0, 0), 0.125, 8, 9.0, 0)
    lam = W.strengths(len(p), 1, 8)
    plan = api.Plan(torch.from_numpy(p).cuda(), wl.lo, wl.h, wl.ng, wl.k, layout="repetition")
    out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
    assert rel_l2(out, oracle.p2p(p, lam, wl.lo, wl.h, wl.ng, wl.k)) <= TOL
    # the coordinate gradient runs on the plan's indexed lists
    g = W.strengths(len(p), 1, 9)
    gx = plan.grad_points(torch.from_numpy(lam).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    ref = oracle.grad_points(p, lam, g, wl.lo, wl.h, wl.ng, wl.k)
    assert np.linalg.norm(gx - ref) / np.linalg.norm(ref) <= TOL
    with pytest.raises(P2PError):  # one right-hand side only
        api.Plan(torch.from_numpy(p).cuda(), wl.lo, wl.h, wl.ng, wl.k, layout="repetition", max_nrhs=2)
