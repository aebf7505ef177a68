"""Persistent batched launch over several geometries, and its CUDA-graph replay.

The batched result of every geometry must equal that geometry's own apply
(same arithmetic, only the order of atomic additions differs) and the FP64
oracle within the FP32 tolerance (relative L2 <= 1e-5 per right-hand side).
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


def _geometries(api, nrhs):
    geo = []
    p = W.unit_sphere(20000, 61)
    geo.append(dict(points=p, lo=(-1, -1, -1), h=2 / 30, ng=30, k=2 * np.pi / (4 * 2 / 30), kernel="helmholtz",
                    layout="indexed", tuning=None))
    c = W.cylinder_plates(15000, 62)
    st = api.choose_grid_ct(torch.from_numpy(c).cuda(), (-1.3, -1.3, -1.3), 2.6, 64)
    geo.append(dict(points=c, lo=(-1.3, -1.3, -1.3), h=st.h, ng=st.ng, k=2 * np.pi * 0.2 / st.h,
                    kernel="helmholtz", layout="redundant", tuning={"chunk": 256}))
    u = W.uniform_cube(8192, 63)
    geo.append(dict(points=u, lo=(0, 0, 0), h=0.25, ng=4, k=0.0, kernel="laplace", layout="indexed",
                    tuning={"chunk": 64, "warps_per_cta": 4}))
    e = W.ellipsoid_211(12000, 64)
    geo.append(dict(points=e, lo=(-2, -2, -2), h=4 / 40, ng=40, k=12.0, kernel="helmholtz", layout="symmetric",
                    tuning=None))
    plans = []
    for g in geo:
        plans.append(api.Plan(torch.from_numpy(g["points"]).cuda(), g["lo"], g["h"], g["ng"], g["k"],
                              kernel=g["kernel"], layout=g["layout"], max_nrhs=nrhs, tuning=g["tuning"]))
    lams = [torch.from_numpy(W.strengths(len(g["points"]), nrhs, 70 + i)).cuda().reshape(-1, nrhs)
            for i, g in enumerate(geo)]
    return geo, plans, lams


def _oracle(g, lam):
    kern = oracle.HELMHOLTZ if g["kernel"] == "helmholtz" else oracle.LAPLACE
    return oracle.p2p(g["points"], lam.cpu().numpy(), g["lo"], g["h"], g["ng"], g["k"], kernel=kern)


@pytest.mark.parametrize("nrhs", [1, 2, 8])
def test_batch_matches_plans_and_oracle(nrhs):
    api = _api()
    geo, plans, lams = _geometries(api, nrhs)
    batch = api.Batch(plans, nrhs=nrhs)
    assert batch.info["work_items"] == sum(p.info["work_items"] for p in plans)
    outs = batch.apply(lams)
    for g, p, lam, out in zip(geo, plans, lams, outs):
        single = p.apply(lam).cpu().numpy()
        got = out.cpu().numpy()
        assert rel_l2(got, single).max() <= 1e-6
        assert rel_l2(got, _oracle(g, lam)).max() <= TOL


def test_batch_graph_replay_tracks_buffer_contents():
    api = _api()
    geo, plans, lams = _geometries(api, 2)
    batch = api.Batch(plans, nrhs=2, warps_per_cta=4)
    outs = batch.capture(lams)
    batch.replay()
    torch.cuda.synchronize()
    first = [o.cpu().numpy().copy() for o in outs]
    for g, lam, got in zip(geo, lams, first):
        assert rel_l2(got, _oracle(g, lam)).max() <= TOL
    # new strengths written in place: the replayed graph reads them
    for i, lam in enumerate(lams):
        lam.copy_(torch.from_numpy(W.strengths(lam.shape[0], 2, 90 + i)).cuda())
    batch.replay()
    batch.replay()
    torch.cuda.synchronize()
    for g, lam, out in zip(geo, lams, outs):
        assert rel_l2(out.cpu().numpy(), _oracle(g, lam)).max() <= TOL


def test_choose_grid_ct():
    api = _api()
    c = torch.from_numpy(W.cylinder_plates(30000, 64)).cuda()
    st = api.choose_grid_ct(c, (-1.3, -1.3, -1.3), 2.6, 40)
    assert st.max_occupancy <= 40
    coarser = api.BoxStructure(c, (-1.3, -1.3, -1.3), 2.6 / (st.ng // 2), st.ng // 2)
    assert int((coarser.box_ptr[1:] - coarser.box_ptr[:-1]).max().item()) > 40
