"""The autotuner on a small workload: it times every candidate, caches the winner, reuses the cache, and
the plan it picks is correct."""
import numpy as np
import pytest

import oracle
from paper_2403_01596_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_picks_caches_and_is_correct(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import api, autotune
    wl = W.Workload("s", W.unit_sphere(30000, 71), (-1, -1, -1), 2 / 36, 36, 2 * np.pi / (4 * 2 / 36), 71)
    cache = str(tmp_path / "tune.json")
    st = api.BoxStructure(torch.from_numpy(wl.points).cuda(), wl.lo, wl.h, wl.ng)
    first = autotune.tune(st, wl.k, reps=3, path=cache)
    assert not first["cached"]
    # every (layout, candidate) but the direct-kernel candidates of the symmetric layout, which runs staged, and
    # the box-group candidates of the layouts other than indexed
    direct = sum(1 for c in autotune.DEFAULT_CANDIDATES if c.get("warp_boxes", 0) > 0)
    group = sum(1 for c in autotune.DEFAULT_CANDIDATES if c.get("warp_boxes", 0) == -2)
    others = sum(1 for lay in autotune.DEFAULT_LAYOUTS if lay != "indexed")
    assert len(first["all"]) == (len(autotune.DEFAULT_LAYOUTS) * len(autotune.DEFAULT_CANDIDATES) - direct
                                 - others * group)
    assert abs(first["ms"] - min(t[4] for t in first["all"])) <= 1e-5  # "all" keeps 5 decimals
    again = autotune.tune(st, wl.k, reps=3, path=cache)
    assert again["cached"] and again["layout"] == first["layout"] and again["tuning"] == first["tuning"]
    plan = api.Plan(st.points, wl.lo, wl.h, wl.ng, wl.k, layout=first["layout"], tuning=first["tuning"],
                    structure=st)
    lam = W.strengths(wl.n, 1, 71)
    out = plan.apply(torch.from_numpy(lam).cuda()).cpu().numpy()
    ref = oracle.p2p(wl.points, lam, wl.lo, wl.h, wl.ng, wl.k)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5
