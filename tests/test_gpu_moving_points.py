"""A plan that follows moving points: three optimisation steps on the point
coordinates through the autograd function, the forward result and both
gradients checked against the FP64 oracle on the moved coordinates after every
step (relative L2 <= 1e-5).

Step 1 moves points by less than their distance to the leaf-box faces, so the
plan only takes the new coordinates (p2p_plan_update_points keeps the binning,
neighbour lists and work items; the redundant layout's per-box copies are
gathered again).  Step 2 also moves 64 points one box over, so the update
reports that points left their boxes and the plan is rebuilt on the same grid.
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


def rel(x, ref):
    return np.linalg.norm(np.asarray(x) - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("layout", ["indexed", "redundant"])
def test_three_steps_follow_moving_points(layout):
    api = _api()
    n, ng = 20000, 24
    h = 2.0 / ng
    lo = (-1.0, -1.0, -1.0)
    k = 2 * np.pi / (4 * h)
    p0 = W.unit_sphere(n, 70)
    pts = torch.from_numpy(p0).cuda().requires_grad_(True)
    plan = api.Plan(pts.detach(), lo, h, ng, k, layout=layout)
    lam = torch.from_numpy(W.strengths(n, 1, 70)).cuda().requires_grad_(True)
    b = torch.from_numpy(W.strengths(n, 1, 71)).cuda()
    rng = np.random.default_rng(72)
    jump = rng.choice(n, 64, replace=False)
    for step in range(3):
        out = api.p2p(lam, pts, plan)
        loss = (out - b).abs().pow(2).sum()
        loss.backward()
        assert plan.rebuilds == (1 if step == 2 else 0)
        assert plan.async_status() == 0
        x = pts.detach().cpu().numpy()
        ref = oracle.p2p(x, lam.detach().cpu().numpy(), lo, h, ng, k)
        g = 2 * (ref - b.cpu().numpy())
        ref_lam = oracle.p2p(x, g, lo, h, ng, k, adjoint=True)
        ref_x = oracle.grad_points(x, lam.detach().cpu().numpy(), g, lo, h, ng, k)
        e_out, e_lam, e_x = rel(out.detach().cpu().numpy(), ref), rel(lam.grad.cpu().numpy(), ref_lam), \
            rel(pts.grad.cpu().numpy(), ref_x)
        print(f"{layout} step {step}: forward {e_out:.2e}, d/dlambda {e_lam:.2e}, d/dx {e_x:.2e}")
        assert e_out <= TOL and e_lam <= TOL and e_x <= TOL
        with torch.no_grad():
            # a gradient step of at most 1e-3 h, applied only to points at least 2e-3 h from every face
            gx = pts.grad
            frac = (pts - torch.tensor(lo, device="cuda")) / h
            frac = frac - torch.floor(frac)
            room = torch.minimum(frac, 1 - frac).min(dim=1).values
            move = -1e-3 * h * gx / gx.abs().max()
            move[room < 2e-3] = 0
            pts += move
            if step == 1:
                pts[torch.from_numpy(jump).cuda(), 0] += h  # one box over in x
        pts.grad = None
        lam.grad = None
