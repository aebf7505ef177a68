"""The allocation-free binning entry point against the workspace one.

p2p_bin_points_static serves callers that cannot allocate device memory at the
point where they bin (under a fixed device-memory budget, or inside a host
application's callback that forbids allocations): its scratch is a fixed array
inside the library.  Two calls in a row, with different point sets, must give exactly the
outputs of p2p_bin_points (integer outputs: bit-exact), so nothing left in the
shared array by one call leaks into the next.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2403_01596_gb300 import workloads as W

torch = pytest.importorskip("torch")


def _bin_both(C, pts_np, lo, h, ng):
    n = pts_np.shape[0]
    pts = torch.from_numpy(pts_np).cuda()
    outs = []
    for static in (False, True):
        perm = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        pbox = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        keys = torch.full((n,), -7, dtype=torch.int64, device="cuda")
        ptr = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
        if static:
            nb = C.p2p_bin_points_static(pts, lo, h, ng, perm, pbox, keys, ptr)
        else:
            work = torch.empty(C.p2p_bin_workspace_size(n), dtype=torch.uint8, device="cuda")
            nb = C.p2p_bin_points(pts, lo, h, ng, perm, pbox, keys, ptr, work)
        outs.append((nb, perm.cpu().numpy(), pbox.cpu().numpy(), keys.cpu().numpy()[:nb],
                     ptr.cpu().numpy()[:nb + 1]))
    return outs


@pytest.mark.gpu
def test_static_binning_matches_workspace_binning_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01596_gb300 import _capi as C
    cases = [
        (W.unit_sphere(C.P2P_BIN_STATIC_MAX_POINTS, 41), (-1.0, -1.0, -1.0), 2.0 / 37, 37),
        (W.uniform_cube(20011, 42), (0.0, 0.0, 0.0), 1.0 / 9, 9),
    ]
    for pts, lo, h, ng in cases:
        (nb0, *ref), (nb1, *got) = _bin_both(C, pts, lo, h, ng)
        assert nb0 == nb1 and nb0 > 0
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)
    # more points than the fixed scratch holds: rejected before any device work
    big = torch.zeros((C.P2P_BIN_STATIC_MAX_POINTS + 1, 3), dtype=torch.float32, device="cuda")
    dummy = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(C.P2PError):
        C.p2p_bin_points_static(big, (0, 0, 0), 0.5, 2, dummy, dummy, dummy, dummy)
