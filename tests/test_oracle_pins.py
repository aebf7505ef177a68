"""Pins of the FP64 oracle against facts that do not come from the oracle.

The paper prints no output values (its results are timing ratios only), so
every pin here is fixed by mathematics: closed forms of the Green's function,
a brute-force all-pairs sum with the neighbour mask taken straight from cell
coordinates (no Morton keys, sort or CSR), the dense special case where every
box neighbours every other, the symmetry G(x, y) = G(y, x), the Laplace limit
k -> 0, the adjoint identity, linearity, permutation invariance and central
finite differences for the coordinate gradient.  A dropped neighbour, a wrong
sign, a swapped index or a transposed operand in the oracle fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2403_01596_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cells_numpy(p, lo, h, ng):
    c = np.floor((p.astype(np.float64) - np.asarray(lo)) / h)
    return np.clip(c, 0, ng - 1).astype(np.int64)


def _brute(p, lam, lo, h, ng, k, laplace=False, conj=False):
    """All-pairs sum; neighbour mask = Chebyshev distance of cells <= 1."""
    p64 = p.astype(np.float64)
    c = _cells_numpy(p, lo, h, ng)
    mask = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2) <= 1
    d = p64[:, None, :] - p64[None, :, :]
    r = np.sqrt((d * d).sum(axis=2))
    valid = mask & (r > 0)
    rs = np.where(valid, r, 1.0)
    if laplace:
        g = 1.0 / (4 * np.pi * rs)
    else:
        g = np.exp((-1j if conj else 1j) * k * rs) / (4 * np.pi * rs)
    g = np.where(valid, g, 0.0)
    return g @ lam


def test_morton_closed_form(oracle_lib):
    o = oracle_lib
    assert [o.morton_key(1, 0, 0), o.morton_key(0, 1, 0), o.morton_key(0, 0, 1)] == [1, 2, 4]
    assert o.morton_key(1, 1, 1) == 7
    assert o.morton_key(2, 0, 0) == 8
    assert o.morton_key(3, 5, 6) == int("110101011", 2)  # x=011 y=101 z=110 interleaved z y x
    top = (1 << 21) - 1
    assert o.morton_key(top, top, top) == (1 << 63) - 1


def test_cell_rule_faces_and_clamp(oracle_lib):
    # a point on a face goes to the upper cell; points outside the cube clamp
    pts = np.array([[0.5, 0.0, 0.25], [1.0, 0.999, -3.0], [7.0, 0.125, 0.375]], dtype=np.float32)
    c = oracle_lib.point_cells(pts, (0, 0, 0), 0.125, 8)
    assert c.tolist() == [[4, 0, 2], [7, 7, 0], [7, 1, 3]]


def test_closed_form_single_pair(oracle_lib):
    spec = json.load(open(os.path.join(GOLDEN, "closed_form_pair.json")))
    pts = np.array(spec["points"], dtype=np.float32)
    lam = np.array([1.0 + 0j, 1.0 + 0j])
    out = oracle_lib.p2p(pts, lam, spec["lo"], spec["h"], spec["ng"], spec["k"])
    exp = complex(*spec["helmholtz_out"])
    assert abs(out[0] - exp) < 1e-15 and abs(out[1] - exp) < 1e-15
    out_l = oracle_lib.p2p(pts, lam, spec["lo"], spec["h"], spec["ng"], 0.0, kernel=oracle_lib.LAPLACE)
    assert abs(out_l[0] - complex(*spec["laplace_out"])) < 1e-15
    # the closed form itself: exp(i pi/2) / (4 pi 0.5) = i / (2 pi)
    assert abs(exp - 1j / (2 * math.pi)) < 1e-16


def test_closed_form_three_points(oracle_lib):
    # right triangle with legs 0.375, 0.5 and hypotenuse 0.625 (all exact in float32)
    pts = np.array([[0.25, 0.25, 0.25], [0.625, 0.25, 0.25], [0.25, 0.75, 0.25]], dtype=np.float32)
    lam = np.array([1 + 2j, -0.5 + 0.25j, 3 - 1j])
    k = 2.0
    out = oracle_lib.p2p(pts, lam, (0, 0, 0), 0.5, 2, k)
    g = {r: complex(math.cos(k * r), math.sin(k * r)) / (4 * math.pi * r) for r in (0.375, 0.5, 0.625)}
    exp = [g[0.375] * lam[1] + g[0.5] * lam[2],
           g[0.375] * lam[0] + g[0.625] * lam[2],
           g[0.5] * lam[0] + g[0.625] * lam[1]]
    np.testing.assert_allclose(out, exp, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("seed,n,ng", [(5, 300, 5), (6, 700, 7), (7, 1500, 9)])
def test_oracle_matches_bruteforce(oracle_lib, seed, n, ng):
    p = W.uniform_cube(n, seed)
    lam = W.strengths(n, 1, seed)
    h = 1.0 / ng
    k = 2 * np.pi / (4 * h)
    out = oracle_lib.p2p(p, lam, (0, 0, 0), h, ng, k)
    ref = _brute(p, lam.astype(np.complex128), (0, 0, 0), h, ng, k)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    out_l = oracle_lib.p2p(p, lam, (0, 0, 0), h, ng, 0.0, kernel=oracle_lib.LAPLACE)
    ref_l = _brute(p, lam.astype(np.complex128), (0, 0, 0), h, ng, 0.0, laplace=True)
    np.testing.assert_allclose(out_l, ref_l, rtol=1e-12, atol=1e-12 * np.abs(ref_l).max())


def test_oracle_bruteforce_sphere_with_empty_boxes(oracle_lib):
    p = W.unit_sphere(1200, 9)
    lam = W.strengths(1200, 1, 9)
    ng = 11
    h = 2.0 / ng
    out = oracle_lib.p2p(p, lam, (-1, -1, -1), h, ng, 5.0)
    ref = _brute(p, lam.astype(np.complex128), (-1, -1, -1), h, ng, 5.0)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("ng", [1, 2])
def test_dense_special_case(oracle_lib, ng):
    """With ng <= 2 every box neighbours every other: P2P is the dense MVM.

    (At ng = 3 the cells 0 and 2 of an axis are two apart and not neighbours.)
    """
    from scipy.spatial.distance import cdist
    n = 400
    p = W.uniform_cube(n, 11 + ng)
    lam = W.strengths(n, 1, 3).astype(np.complex128)
    k = 7.5
    r = cdist(p.astype(np.float64), p.astype(np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(r > 0, np.exp(1j * k * r) / (4 * np.pi * r), 0.0)
    out = oracle_lib.p2p(p, lam, (0, 0, 0), 1.0 / ng, ng, k)
    np.testing.assert_allclose(out, g @ lam, rtol=1e-12, atol=1e-12 * np.abs(g @ lam).max())


def test_symmetry_bilinear(oracle_lib):
    """G(x, y) = G(y, x) and the neighbour relation is symmetric: mu^T (A lam) = lam^T (A mu)."""
    n = 2000
    p = W.unit_sphere(n, 21)
    lam = W.strengths(n, 1, 21).astype(np.complex128)
    mu = W.strengths(n, 1, 22).astype(np.complex128)
    args = ((-1, -1, -1), 2.0 / 13, 13, 9.0)
    a = mu @ oracle_lib.p2p(p, lam, *args)
    b = lam @ oracle_lib.p2p(p, mu, *args)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_adjoint_identity(oracle_lib):
    """<A lam, mu> = <lam, A^H mu> with the Hermitian inner product."""
    n = 1500
    p = W.uniform_cube(n, 31)
    lam = W.strengths(n, 1, 31).astype(np.complex128)
    mu = W.strengths(n, 1, 32).astype(np.complex128)
    args = ((0, 0, 0), 1.0 / 6, 6, 11.0)
    lhs = np.vdot(mu, oracle_lib.p2p(p, lam, *args))
    rhs = np.vdot(oracle_lib.p2p(p, mu, *args, adjoint=True), lam)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # and the adjoint differs from the forward operator when k != 0
    assert np.abs(oracle_lib.p2p(p, mu, *args, adjoint=True) - oracle_lib.p2p(p, mu, *args)).max() > 1e-3


def test_helmholtz_k0_is_laplace_and_small_k_limit(oracle_lib):
    n = 1000
    p = W.uniform_cube(n, 41)
    lam = W.strengths(n, 1, 41).astype(np.complex128)
    args = ((0, 0, 0), 0.2, 5)
    lap = oracle_lib.p2p(p, lam, *args, 0.0, kernel=oracle_lib.LAPLACE)
    h0 = oracle_lib.p2p(p, lam, *args, 0.0)
    np.testing.assert_allclose(h0, lap, rtol=0, atol=1e-15 * np.abs(lap).max())
    # k small: exp(ikr)/(4 pi r) = 1/(4 pi r) + i k/(4 pi) + O(k^2 r)
    k = 1e-4
    hk = oracle_lib.p2p(p, lam, *args, k)
    ones = np.ones(n)
    nsum = oracle_lib.p2p(p, ones, *args, 0.0, kernel=oracle_lib.LAPLACE)  # sanity only
    assert np.all(np.abs(nsum) > 0)
    # i k/(4 pi) times the plain sum of neighbouring strengths (r > 0), from brute force
    c = _cells_numpy(p, *args)
    mask = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2) <= 1
    np.fill_diagonal(mask, False)
    lin = 1j * k / (4 * np.pi) * (mask @ lam)
    rmax = np.sqrt(3) * 2 * 0.2
    bound = k * k * rmax / (4 * np.pi) * np.abs(lam).sum()
    assert np.abs(hk - lap - lin).max() <= bound


def test_linearity_and_multi_rhs(oracle_lib):
    n = 800
    p = W.unit_sphere(n, 51)
    args = ((-1, -1, -1), 2.0 / 9, 9, 6.0)
    l1 = W.strengths(n, 1, 51).astype(np.complex128)
    l2 = W.strengths(n, 1, 52).astype(np.complex128)
    a, b = 0.7 - 0.2j, -1.3 + 2j
    lhs = oracle_lib.p2p(p, a * l1 + b * l2, *args)
    rhs = a * oracle_lib.p2p(p, l1, *args) + b * oracle_lib.p2p(p, l2, *args)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())
    panel = np.stack([l1, l2], axis=1)
    out = oracle_lib.p2p(p, panel, *args)
    np.testing.assert_allclose(out[:, 1], oracle_lib.p2p(p, l2, *args), rtol=0, atol=0)


def test_permutation_invariance(oracle_lib):
    n = 900
    p = W.uniform_cube(n, 61)
    lam = W.strengths(n, 1, 61).astype(np.complex128)
    args = ((0, 0, 0), 0.25, 4, 12.0)
    perm = np.random.default_rng(0).permutation(n)
    out = oracle_lib.p2p(p, lam, *args)
    outp = oracle_lib.p2p(p[perm], lam[perm], *args)
    np.testing.assert_allclose(outp, out[perm], rtol=1e-12, atol=1e-12 * np.abs(out).max())


def test_targets_subset_matches_full(oracle_lib):
    n = 1000
    p = W.unit_sphere(n, 71)
    lam = W.strengths(n, 2, 71)
    args = ((-1, -1, -1), 2.0 / 10, 10, 8.0)
    full = oracle_lib.p2p(p, lam, *args)
    t = np.array([0, 5, 999, 17, 5])
    sub = oracle_lib.p2p_targets(p, lam, t, *args)
    np.testing.assert_array_equal(sub, full[t])


def test_pair_count_bruteforce(oracle_lib):
    n = 1200
    p = W.unit_sphere(n, 81)
    lo, h, ng = (-1, -1, -1), 2.0 / 12, 12
    c = _cells_numpy(p, lo, h, ng)
    mask = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2) <= 1
    d = p[:, None, :].astype(np.float64) - p[None, :, :]
    r2 = (d * d).sum(axis=2)
    assert oracle_lib.pair_count(p, lo, h, ng) == int((mask & (r2 > 0)).sum())


def test_duplicates_and_degenerate_inputs(oracle_lib):
    # duplicated points interact with nobody at r = 0, but with the others
    p = np.array([[0.1, 0.1, 0.1], [0.1, 0.1, 0.1], [0.3, 0.1, 0.1]], dtype=np.float32)
    lam = np.array([1.0, 2.0, 4.0], dtype=np.complex128)
    out = oracle_lib.p2p(p, lam, (0, 0, 0), 0.5, 2, 0.0, kernel=oracle_lib.LAPLACE)
    r = np.float64(np.float32(0.3)) - np.float64(np.float32(0.1))
    g = 1 / (4 * np.pi * r)
    np.testing.assert_allclose(out, [4 * g, 4 * g, 3 * g], rtol=1e-15)
    # a single point, and the empty set
    assert oracle_lib.p2p(p[:1], lam[:1], (0, 0, 0), 0.5, 2, 3.0)[0] == 0
    assert oracle_lib.p2p(np.zeros((0, 3), np.float32), np.zeros(0, np.complex128), (0, 0, 0), 0.5, 2,
                          3.0).shape == (0,)
    # non-finite coordinates are rejected
    bad = p.copy()
    bad[1, 2] = np.nan
    with pytest.raises(ValueError):
        oracle_lib.p2p(bad, lam, (0, 0, 0), 0.5, 2, 1.0)


def test_binning_bit_exact_independent(oracle_lib):
    """Box ids, perm and box_ptr against a numpy construction (per-bit Morton, lexsort)."""
    n = 5000
    p = W.unit_sphere(n, 91)
    lo, h, ng = (-1, -1, -1), 2.0 / 23, 23
    c = _cells_numpy(p, lo, h, ng)
    key = np.zeros(n, dtype=np.int64)
    for bit in range(21):
        for a in range(3):
            key |= ((c[:, a] >> bit) & 1) << (3 * bit + a)
    order = np.lexsort((np.arange(n), key))
    uk, first = np.unique(key[order], return_index=True)
    b = oracle_lib.bin_points(p, lo, h, ng)
    np.testing.assert_array_equal(b["perm"], order)
    np.testing.assert_array_equal(b["box_keys"], uk)
    np.testing.assert_array_equal(b["box_ptr"], np.append(first, n))
    inv = np.searchsorted(uk, key)
    np.testing.assert_array_equal(b["point_box"], inv)
    # neighbours: all box pairs with Chebyshev distance <= 1, ascending
    bc = c[order][first]
    cheb = np.abs(bc[:, None, :] - bc[None, :, :]).max(axis=2)
    nptr, nidx = oracle_lib.neighbors(b["box_keys"], ng)
    for i in range(len(uk)):
        np.testing.assert_array_equal(nidx[nptr[i]:nptr[i + 1]], np.nonzero(cheb[i] <= 1)[0])


def test_gradient_finite_differences(oracle_lib):
    """Central differences (step 1e-5, FP64) of L = ||A lam - b||^2 against the analytic gradient."""
    n = 600
    p = W.unit_sphere(n, 101).astype(np.float64)
    lo, h, ng, k = (-1, -1, -1), 2.0 / 8, 8, 10.0
    lam = W.strengths(n, 1, 101).astype(np.complex128)
    b = W.strengths(n, 1, 102).astype(np.complex128)

    def loss(q):
        r = oracle_lib.p2p(q, lam, lo, h, ng, k) - b
        return float(np.vdot(r, r).real)

    g = 2 * (oracle_lib.p2p(p, lam, lo, h, ng, k) - b)  # dL/dRe + i dL/dIm of out
    grad = oracle_lib.grad_points(p, lam, g, lo, h, ng, k)
    c = (p - np.asarray(lo)) / h
    far = np.min(np.abs(c - np.round(c)), axis=1) * h > 2e-3   # keep box membership fixed
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(axis=2))
    np.fill_diagonal(d, np.inf)
    sparse = d.min(axis=1) > 2e-2                               # no very close pair
    idx = np.nonzero(far & sparse)[0][:12]
    assert len(idx) >= 8
    eps = 1e-5
    for i in idx:
        for a in range(3):
            q = p.copy()
            q[i, a] += eps
            lp = loss(q)
            q[i, a] -= 2 * eps
            lm = loss(q)
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - grad[i, a]) <= 1e-5 * max(1.0, abs(grad[i, a])), (i, a, fd, grad[i, a])
    # Laplace gradient as well
    gl = 2 * (oracle_lib.p2p(p, lam, lo, h, ng, 0.0, kernel=oracle_lib.LAPLACE) - b)
    gradl = oracle_lib.grad_points(p, lam, gl, lo, h, ng, 0.0, kernel=oracle_lib.LAPLACE)
    i = idx[0]
    q = p.copy()

    def loss_l(q):
        r = oracle_lib.p2p(q, lam, lo, h, ng, 0.0, kernel=oracle_lib.LAPLACE) - b
        return float(np.vdot(r, r).real)
    q[i, 1] += eps
    lp = loss_l(q)
    q[i, 1] -= 2 * eps
    lm = loss_l(q)
    assert abs((lp - lm) / (2 * eps) - gradl[i, 1]) <= 1e-5 * max(1.0, abs(gradl[i, 1]))


# ------------------------------------------------- separate point sets ----
# Sec. 3.1 keeps target and source coordinates as separate arrays: the same sum
# between two point sets binned on one grid.

def _brute_st(t, s, lam, lo, h, ng, k, laplace=False, conj=False):
    """All target-source pairs; neighbour mask = Chebyshev distance of the two cells <= 1."""
    ct, cs = _cells_numpy(t, lo, h, ng), _cells_numpy(s, lo, h, ng)
    mask = np.abs(ct[:, None, :] - cs[None, :, :]).max(axis=2) <= 1
    d = t.astype(np.float64)[:, None, :] - s.astype(np.float64)[None, :, :]
    r = np.sqrt((d * d).sum(axis=2))
    valid = mask & (r > 0)
    rs = np.where(valid, r, 1.0)
    g = 1.0 / (4 * np.pi * rs) if laplace else np.exp((-1j if conj else 1j) * k * rs) / (4 * np.pi * rs)
    return np.where(valid, g, 0.0) @ lam


@pytest.mark.parametrize("nt,ns,ng,seed", [(700, 1100, 5, 1), (1500, 400, 7, 2), (1, 900, 3, 3), (800, 1, 4, 4)])
def test_st_matches_bruteforce(oracle_lib, nt, ns, ng, seed):
    rng = np.random.default_rng(seed)
    t = rng.random((nt, 3)).astype(np.float32)
    s = (rng.random((ns, 3)) * 1.1 - 0.05).astype(np.float32)  # some sources outside the grid: clamped
    s[: min(ns, nt) // 3] = t[: min(ns, nt) // 3]              # shared positions: r = 0 pairs are skipped
    lam = W.strengths(ns, 2, seed).reshape(ns, 2)
    lo, h = (0.0, 0.0, 0.0), 1.0 / ng
    for laplace in (False, True):
        got = oracle_lib.p2p_st(t, s, lam, lo, h, ng, 7.0, kernel=oracle_lib.LAPLACE if laplace else 0)
        ref = _brute_st(t, s, lam, lo, h, ng, 7.0, laplace=laplace)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    got = oracle_lib.p2p_st(t, s, lam, lo, h, ng, 7.0, conj=True)
    np.testing.assert_allclose(got, _brute_st(t, s, lam, lo, h, ng, 7.0, conj=True), rtol=1e-12,
                               atol=1e-12 * np.abs(got).max())


def test_st_dense_case_and_closed_form(oracle_lib):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(9)
    t = rng.random((300, 3)).astype(np.float32)
    s = rng.random((500, 3)).astype(np.float32)
    lam = W.strengths(500, 1, 9)
    k = 5.5
    r = spatial.distance.cdist(t.astype(np.float64), s.astype(np.float64))
    A = np.exp(1j * k * r) / (4 * np.pi * r)
    # ng = 2: every target box neighbours every source box, so the near field is the dense operator
    got = oracle_lib.p2p_st(t, s, lam, (0, 0, 0), 0.5, 2, k)
    np.testing.assert_allclose(got, A @ lam, rtol=1e-12, atol=1e-13)
    # one target, one source at r = 0.5, k = pi: exp(i pi / 2) / (4 pi 0.5) = i / (2 pi)
    one = oracle_lib.p2p_st(np.array([[0.1, 0.2, 0.3]], np.float32), np.array([[0.1, 0.2, 0.8]], np.float32),
                            np.array([1.0 + 0j]), (0, 0, 0), 1.0, 1, math.pi)
    assert abs(one[0] - 1j / (2 * math.pi)) < 1e-15


def test_st_reduces_to_one_set_and_reciprocity(oracle_lib):
    rng = np.random.default_rng(11)
    p = rng.random((1200, 3)).astype(np.float32)
    q = rng.random((900, 3)).astype(np.float32)
    lo, h, ng, k = (0, 0, 0), 1.0 / 6, 6, 9.0
    lam = W.strengths(1200, 1, 11)
    # sources = targets: the one-set operator, summed in the same order, bit for bit
    np.testing.assert_array_equal(oracle_lib.p2p_st(p, p, lam, lo, h, ng, k), oracle_lib.p2p(p, lam, lo, h, ng, k))
    # G(x, y) = G(y, x) and the cell relation is symmetric: mu^T (A_pq lam) = lam^T (A_qp mu), no conjugation,
    # and the adjoint A_pq^H = conj(A_qp): <A_pq lam, mu> = <lam, A_qp^conj mu>
    lam_q = W.strengths(900, 1, 12)
    mu = W.strengths(1200, 1, 13)
    a = mu @ oracle_lib.p2p_st(p, q, lam_q, lo, h, ng, k)
    b = lam_q @ oracle_lib.p2p_st(q, p, mu, lo, h, ng, k)
    assert abs(a - b) <= 1e-12 * abs(a)
    lhs = np.vdot(mu, oracle_lib.p2p_st(p, q, lam_q, lo, h, ng, k))
    rhs = np.vdot(oracle_lib.p2p_st(q, p, mu, lo, h, ng, k, conj=True), lam_q)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_st_neighbors_independent(oracle_lib):
    rng = np.random.default_rng(14)
    ng = 9
    t = (rng.random((400, 3)) * 0.6).astype(np.float32)          # targets in one corner
    s = (rng.random((700, 3)) * 0.7 + 0.3).astype(np.float32)    # sources overlapping it partly
    lo, h = (0, 0, 0), 1.0 / ng
    bt, bs = oracle_lib.bin_points(t, lo, h, ng), oracle_lib.bin_points(s, lo, h, ng)
    nptr, nidx = oracle_lib.neighbors_st(bt["box_keys"], bs["box_keys"], ng)
    # independent construction from the cells of the points of each box
    ct = _cells_numpy(t, lo, h, ng)[bt["perm"][bt["box_ptr"][:-1]]]
    cs = _cells_numpy(s, lo, h, ng)[bs["perm"][bs["box_ptr"][:-1]]]
    for b in range(bt["num_boxes"]):
        want = np.nonzero(np.abs(cs - ct[b]).max(axis=1) <= 1)[0]
        np.testing.assert_array_equal(nidx[nptr[b]:nptr[b + 1]], want)
    assert nptr[-1] < 27 * bt["num_boxes"] and nptr[-1] > 0
    # sampled targets equal the full evaluation
    lam = W.strengths(700, 1, 14)
    full = oracle_lib.p2p_st(t, s, lam, lo, h, ng, 4.0)
    which = np.array([0, 17, 399, 200])
    np.testing.assert_array_equal(oracle_lib.p2p_st_targets(t, s, lam, which, lo, h, ng, 4.0), full[which])
