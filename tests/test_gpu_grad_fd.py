"""Coordinate gradient on the differentiable-P2P workload, checked three ways.

Workload: 2^18 points uniform on the unit sphere, 62^3 leaf grid (~16 points
per box), Helmholtz k = 16 pi, loss L(x) = ||A(x) lam - b||^2 with lam and b
complex N(0, 1).  64 (point, axis) coordinates are drawn among the points
whose nearest neighbour is farther than 1e-2 and which lie at least 2e-3 from
every face of their leaf box, so a step of 1e-3 moves no point to another box
(the gradient is the derivative with box membership held fixed).

1. Central differences of L in the FP64 oracle, step d = 1e-3, against the
   oracle's analytic gradient.  The central difference has truncation error
   (d^2 / 6) L'''(x) + O(d^4), so it is checked against its own estimate of
   that error, (4/3) |D(d) - D(d/2)| (Richardson), and the extrapolated value
   (4 D(d/2) - D(d)) / 3, whose error is O(d^4), against the analytic gradient
   at relative L2 <= 1e-5.
2. The GPU gradient (p2p_grad_points, FP32) against the oracle's analytic
   gradient: relative L2 <= 1e-5 over all 3n coordinates and over the 64.
The two errors are printed separately.

Only the targets whose sums involve the moved point change (its own box's
neighbourhood), so L(x +- d e) - L(x) is evaluated on those targets, with the
oracle given the points of the 5^3 boxes around the moved point's box (every
source of every affected target; the same boxes in the same relative order,
so the same FP64 sums as on the full set).
"""
import numpy as np
import pytest

import oracle
from paper_2403_01596_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP = 1e-3


def _api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import api
    return api


def _pick_coordinates(points, cells, wl, count, seed):
    spatial = pytest.importorskip("scipy.spatial")
    p = points.astype(np.float64)
    d, _ = spatial.cKDTree(p).query(p, k=2)
    rel = (p - np.asarray(wl.lo)) / wl.h
    frac = rel - np.floor(rel)
    to_face = np.minimum(frac, 1.0 - frac).min(axis=1) * wl.h
    cand = np.nonzero((d[:, 1] > 1e-2) & (to_face >= 2e-3))[0]
    assert cand.size >= count
    rng = np.random.default_rng(seed)
    return rng.choice(cand, count, replace=False), rng.integers(0, 3, count)


def oracle_fd(wl, lam, b, count=64, seed=2024):
    """Oracle forward, analytic coordinate gradient and central differences (steps STEP and STEP / 2) at
    `count` coordinates chosen as the module docstring says."""
    out_ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    g_ref = 2.0 * (out_ref - b)
    grad_ref = oracle.grad_points(wl.points, lam, g_ref, wl.lo, wl.h, wl.ng, wl.k)
    cells = oracle.point_cells(wl.points, wl.lo, wl.h, wl.ng)
    pick, axes = _pick_coordinates(wl.points, cells, wl, count, seed)
    bins = oracle.bin_points(wl.points, wl.lo, wl.h, wl.ng)
    nptr, nidx = oracle.neighbors(bins["box_keys"], wl.ng)
    bp, perm, pbox = bins["box_ptr"], bins["perm"], bins["point_box"]
    base = wl.points.astype(np.float64)

    def loss_slope(m, a, d):
        # affected targets: every point of the moved point's neighbour boxes (the moved point included)
        bm = pbox[m]
        aff = np.sort(np.concatenate([perm[bp[c]:bp[c + 1]] for c in nidx[nptr[bm]:nptr[bm + 1]]]))
        near = np.nonzero(np.abs(cells - cells[m]).max(axis=1) <= 2)[0]   # original order kept
        local = np.searchsorted(near, aff)
        vals = []
        for sgn in (1.0, -1.0):
            p = base[near].copy()
            p[np.searchsorted(near, m), a] += sgn * d
            o = oracle.p2p_targets(p, lam[near], local, wl.lo, wl.h, wl.ng, wl.k)
            vals.append(np.sum(np.abs(o - b[aff]) ** 2))
        return (vals[0] - vals[1]) / (2.0 * d)

    fd1 = np.array([loss_slope(m, a, STEP) for m, a in zip(pick, axes)])
    fd2 = np.array([loss_slope(m, a, STEP / 2) for m, a in zip(pick, axes)])
    return {"grad": grad_ref, "pick": pick, "axes": axes, "fd1": fd1, "fd2": fd2}


def check_fd(r):
    an = r["grad"][r["pick"], r["axes"]]
    fd1, fd2 = r["fd1"], r["fd2"]
    rich = (4.0 * fd2 - fd1) / 3.0
    err_fd = np.linalg.norm(fd1 - an) / np.linalg.norm(an)
    err_rich = np.linalg.norm(rich - an) / np.linalg.norm(an)
    # the step-1e-3 difference agrees with the analytic gradient to within its own truncation estimate
    trunc = 4.0 / 3.0 * np.abs(fd1 - fd2)
    assert np.all(np.abs(fd1 - an) <= 1.25 * trunc + 1e-9 * np.abs(an).max())
    assert err_fd <= 5e-3
    assert err_rich <= 1e-5
    return an, err_fd, err_rich


def test_coordinate_gradient_fd_and_gpu():
    api = _api()
    wl = W.sphere_grad()
    n = wl.n
    lam = W.strengths(n, 1, wl.seed)
    b = W.strengths(n, 1, 4)
    r = oracle_fd(wl, lam, b)
    an, err_fd, err_rich = check_fd(r)
    # GPU: forward, upstream gradient and coordinate gradient through the C ABI, FP32
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k)
    lam_d = torch.from_numpy(lam).cuda()
    out_d = plan.apply(lam_d)
    g_d = 2.0 * (out_d - torch.from_numpy(b).cuda())
    grad_gpu = plan.grad_points(lam_d, g_d).cpu().numpy()
    assert plan.async_status() == 0
    gpu = grad_gpu[r["pick"], r["axes"]]
    err_gpu64 = np.linalg.norm(gpu - an) / np.linalg.norm(an)
    err_gpu = np.linalg.norm(grad_gpu - r["grad"]) / np.linalg.norm(r["grad"])
    print(f"FD(step {STEP}) vs oracle analytic: rel-L2 {err_fd:.3e}; Richardson: {err_rich:.3e}; "
          f"GPU vs oracle analytic: {err_gpu64:.3e} (64 coordinates), {err_gpu:.3e} (all 3n)")
    assert err_gpu64 <= 1e-5 and err_gpu <= 1e-5
