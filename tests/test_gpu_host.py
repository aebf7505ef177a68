"""Host-buffer apply (p2p_apply_host): strengths uploaded from page-locked host
memory, the operator applied plan after plan through two device slots, results
downloaded, with the copies of neighbouring plans overlapping the kernels.

Every plan's host result must equal its own device apply (same kernels on the
same strengths; only the order of atomic additions may differ) and the FP64
oracle within the FP32 tolerance (relative L2 <= 1e-5 per right-hand side).
Plans of uneven size exercise the slot reuse; an odd count, plan 0 repeated and
an empty point set exercise the ends of the pipeline.
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


def _plans(api, nrhs):
    geo = [dict(points=W.unit_sphere(30000, 81), lo=(-1, -1, -1), h=2 / 40, ng=40, k=2 * np.pi / (4 * 2 / 40),
                kernel="helmholtz", layout="indexed"),
           dict(points=W.uniform_cube(5000, 82), lo=(0, 0, 0), h=0.125, ng=8, k=0.0, kernel="laplace",
                layout="redundant"),
           dict(points=W.ellipsoid_211(20000, 83), lo=(-2, -2, -2), h=4 / 48, ng=48, k=9.0, kernel="helmholtz",
                layout="symmetric")]
    plans = [api.Plan(torch.from_numpy(g["points"]).cuda(), g["lo"], g["h"], g["ng"], g["k"], kernel=g["kernel"],
                      layout=g["layout"], max_nrhs=nrhs) for g in geo]
    return geo, plans


def _oracle(g, lam):
    kern = oracle.HELMHOLTZ if g["kernel"] == "helmholtz" else oracle.LAPLACE
    return oracle.p2p(g["points"], lam, g["lo"], g["h"], g["ng"], g["k"], kernel=kern)


@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_host_apply_matches_device_apply_and_oracle(nrhs):
    api = _api()
    geo, plans = _plans(api, nrhs)
    order = [0, 1, 2, 0, 1]  # odd count, plans revisited through both slots
    lams = [torch.from_numpy(W.strengths(plans[i].n, nrhs, 90 + j).reshape(plans[i].n, nrhs)).pin_memory()
            for j, i in enumerate(order)]
    pipe = api.HostPipe(max(p.n for p in plans), nrhs)
    outs = pipe.apply([plans[i] for i in order], lams)
    torch.cuda.current_stream().synchronize()
    for j, i in enumerate(order):
        got = outs[j].numpy()
        dev = plans[i].apply(lams[j].cuda()).cpu().numpy()
        tol_dev = 1e-6 if nrhs < 16 else 2e-6
        assert rel_l2(got, dev).max() <= tol_dev
        assert rel_l2(got, _oracle(geo[i], lams[j].numpy())).max() <= TOL
    # a second call on the same pipe reuses its slots and events
    outs2 = pipe.apply([plans[2], plans[1]], [lams[2], lams[1]])
    torch.cuda.current_stream().synchronize()
    assert rel_l2(outs2[0].numpy(), outs[2].numpy()).max() <= 1e-6
    assert rel_l2(outs2[1].numpy(), outs[1].numpy()).max() <= 1e-6
    pipe.close()


def test_host_apply_rejects_oversized_plans_and_handles_empty():
    api = _api()
    geo, plans = _plans(api, 1)
    pipe = api.HostPipe(plans[1].n, 1)
    lam = torch.from_numpy(W.strengths(plans[0].n, 1, 5)).pin_memory()
    with pytest.raises(Exception):
        pipe.apply([plans[0]], [lam])  # plan larger than the pipe's slots
    empty = api.Plan(torch.zeros((0, 3), dtype=torch.float32, device="cuda"), (0, 0, 0), 0.5, 2, 1.0)
    lam1 = torch.from_numpy(W.strengths(plans[1].n, 1, 6)).pin_memory()
    outs = pipe.apply([empty, plans[1]], [torch.zeros(0, dtype=torch.complex64), lam1])
    torch.cuda.current_stream().synchronize()
    assert outs[0].numel() == 0
    assert rel_l2(outs[1].numpy(), _oracle(geo[1], lam1.numpy())).max() <= TOL
    pipe.close()
