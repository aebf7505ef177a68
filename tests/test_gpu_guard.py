"""Guarded apply: every result within a relative tolerance of the exact sum.

The sums of some targets are made to cancel on purpose: one strength in each
chosen target's own box is adjusted (in FP64, from the oracle's row) so that
the target's result is about 1e-4 of the sum of its terms' magnitudes
S_i = sum_j |G(r_ij) lambda_j|.  The plain FP32 apply then misses those
results by far more than 1e-5 (a rounding of 2^-24 S_i is a large part of
|out_i|); the guarded apply re-evaluates every target whose bound 2^-20 S_i
exceeds tol |out_i| in FP64 on the GPU, so all results -- the cancelling ones
and the rest -- are within tol of the FP64 oracle, target by target.
"""
import numpy as np
import pytest

import oracle
from paper_2403_01596_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import api
    return api


def _workload():
    """Sphere of 20 000 points, 30^3 grid, leaf edge a quarter wavelength.  The wavenumber is the float32 value
    the plan receives (p2p_plan_create takes k as a float), so that the FP64 re-evaluation and the oracle sum
    the same operator."""
    ng = 30
    k = float(np.float32(2 * np.pi / (4 * 2.0 / ng)))
    return W.Workload("s", W.unit_sphere(20000, 81), (-1.0, -1.0, -1.0), 2.0 / ng, ng, k, 81)


def _cancel(wl, lam, count=60, eps=1e-4):
    """Strengths with `count` near-cancelling targets (complex128 -> complex64), and those targets."""
    lam = lam.astype(np.complex128).copy()
    b = oracle.bin_points(wl.points, wl.lo, wl.h, wl.ng)
    cells = oracle.point_cells(wl.points, wl.lo, wl.h, wl.ng)
    sizes = np.diff(b["box_ptr"])
    chosen, used = [], []
    for box in np.argsort(-sizes):
        if len(chosen) == count:
            break
        members = b["perm"][b["box_ptr"][box]:b["box_ptr"][box + 1]]
        c = cells[members[0]]
        if any(np.abs(c - u).max() <= 2 for u in used):
            continue  # keep the adjusted sources out of each other's neighbourhoods
        t, j0 = int(members[0]), int(members[1])
        out_t = oracle.p2p_targets(wl.points, lam, [t], wl.lo, wl.h, wl.ng, wl.k)[0]
        s_t = oracle.p2p_targets(wl.points, np.abs(lam), [t], wl.lo, wl.h, wl.ng, 0.0, kernel=oracle.LAPLACE)[0].real
        r = np.linalg.norm(wl.points[t].astype(np.float64) - wl.points[j0].astype(np.float64))
        g = np.exp(1j * wl.k * r) / (4 * np.pi * r)
        lam[j0] -= (out_t - eps * s_t) / g
        chosen.append(t)
        used.append(c)
    return lam.astype(np.complex64), np.array(chosen)


def _rel(out, ref):
    return np.abs(out - ref) / np.abs(ref)


@pytest.mark.parametrize("layout", ["indexed", "redundant"])
def test_guarded_apply_meets_tolerance_per_target(layout):
    api = _api()
    wl = _workload()
    lam, chosen = _cancel(wl, W.strengths(wl.n, 1, 82))
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    S = oracle.p2p(wl.points, np.abs(lam).astype(np.float64), wl.lo, wl.h, wl.ng, 0.0, kernel=oracle.LAPLACE).real
    kappa = S / np.abs(ref)
    assert np.median(kappa[chosen]) > 1e3
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, layout=layout)
    lam_d = torch.from_numpy(lam).cuda()
    plain = plan.apply(lam_d).cpu().numpy()
    worst_plain = _rel(plain[chosen], ref[chosen]).max()
    assert worst_plain > 1e-5  # the cancelling sums are beyond FP32
    for tol in (1e-4, 1e-6):
        out, refined = plan.apply_guarded(lam_d, tol=tol)
        out = out.cpu().numpy()
        rel = _rel(out, ref)
        print(f"{layout} tol {tol:g}: {refined} of {wl.n} targets in FP64; worst relative error {rel.max():.2e} "
              f"(cancelling targets {rel[chosen].max():.2e}, plain FP32 {worst_plain:.2e})")
        assert rel.max() <= tol
        assert rel[chosen].max() <= 2e-7  # FP64 sums stored as complex64: 2^-24 relative rounding
        assert refined >= int((kappa * 2.0 ** -20 > tol).sum() * 0.9)
        assert plan.async_status() == 0


def test_guarded_apply_several_rhs_adjoint_and_tensor_cores():
    api = _api()
    wl = _workload()
    lam1, chosen = _cancel(wl, W.strengths(wl.n, 1, 83))
    lam = W.strengths(wl.n, 16, 84)
    lam[:, 0] = lam1
    plan = api.Plan(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng, wl.k, max_nrhs=16)
    lam_d = torch.from_numpy(lam).cuda()
    # adjoint, FP32 path, three right-hand sides
    ref = oracle.p2p(wl.points, lam[:, :3], wl.lo, wl.h, wl.ng, wl.k, adjoint=True)
    out, refined = plan.apply_guarded(lam_d[:, :3].contiguous(), tol=1e-5, adjoint=True)
    assert _rel(out.cpu().numpy(), ref).max() <= 1e-5 and refined > 0
    # 16 right-hand sides: the hi/lo tensor-core path with its own bound 2^-14 (explicit path), the three-part
    # path with the FP32 bound 2^-20, and AUTO, which at tol 1e-4 starts from the three-part path (the hi/lo
    # bound would flag nearly every target)
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    for path in ("tc_bf16x3", "tc_bf16x6", "auto"):
        out, refined = plan.apply_guarded(lam_d, tol=1e-4, path=path)
        rel = _rel(out.cpu().numpy(), ref)
        print(f"16 RHS, path {path}, tol 1e-4: {refined} targets in FP64, worst relative error {rel.max():.2e}")
        assert rel.max() <= 1e-4 and rel[chosen, 0].max() <= 2e-7
        if path != "tc_bf16x3":
            assert refined < wl.n // 10
    assert plan.async_status() == 0
