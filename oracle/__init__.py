"""FP64 CPU oracle for the near-field P2P operator (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never imports, links or calls it, and the two share no code: the oracle is the
plain C file ``p2p_oracle.c`` compiled with gcc and loaded with ctypes.

Every function takes float64 numpy arrays (FP32 inputs are promoted exactly)
and returns float64 / complex128 results in the caller's original point order.
The operator definition (Sec. 3.1 leaf boxes, Sec. 3.2 / 3.3 neighbour sum,
Sec. 4.1 baseline traversal) is stated in the C file's header.

Pins of the oracle against facts that do not come from the oracle itself live
in ``tests/test_oracle_pins.py`` (brute force, dense special case, closed form,
symmetry, Laplace limit, adjoint identity, finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "p2p_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

HELMHOLTZ = 0
LAPLACE = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32, dbl, cint = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
            lib.oracle_morton_key.argtypes = [i64, i64, i64, P]
            lib.oracle_point_cells.argtypes = [P, i64, P, dbl, i32, P]
            lib.oracle_bin.argtypes = [P, i64, P, dbl, i32, P, P, P, P, P]
            lib.oracle_neighbors.argtypes = [P, i32, i32, P, P]
            lib.oracle_p2p.argtypes = [P, i64, P, dbl, i32, cint, dbl, cint, P, i32, P]
            lib.oracle_p2p_targets.argtypes = [P, i64, P, dbl, i32, cint, dbl, cint, P, i32, P, i64, P]
            lib.oracle_pair_count.argtypes = [P, i64, P, dbl, i32, P]
            lib.oracle_grad_points.argtypes = [P, i64, P, dbl, i32, cint, dbl, P, P, i32, P]
            lib.oracle_neighbors_st.argtypes = [P, i32, P, i32, i32, P, P]
            lib.oracle_p2p_st.argtypes = [P, i64, P, i64, P, dbl, i32, cint, dbl, cint, P, i32, P]
            lib.oracle_p2p_st_targets.argtypes = [P, i64, P, i64, P, dbl, i32, cint, dbl, cint, P, i32, P, i64, P]
            for f in ("oracle_morton_key", "oracle_point_cells", "oracle_bin", "oracle_neighbors",
                      "oracle_p2p", "oracle_p2p_targets", "oracle_pair_count", "oracle_grad_points",
                      "oracle_neighbors_st", "oracle_p2p_st", "oracle_p2p_st_targets"):
                getattr(lib, f).restype = cint
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _pts64(points) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    return p


def _lo(lo) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(lo, dtype=np.float64).reshape(3))


def _lam64(lam, n: int) -> tuple[np.ndarray, int]:
    lam = np.asarray(lam)
    if lam.ndim == 1:
        lam = lam.reshape(n, 1)
    nrhs = lam.shape[1]
    out = np.empty((n, nrhs, 2), dtype=np.float64)
    out[..., 0] = lam.real
    out[..., 1] = lam.imag
    return np.ascontiguousarray(out), nrhs


def _check(st: int, what: str):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def morton_key(cx: int, cy: int, cz: int) -> int:
    k = np.zeros(1, dtype=np.int64)
    _check(_load().oracle_morton_key(cx, cy, cz, _ptr(k)), "morton_key")
    return int(k[0])


def point_cells(points, lo, h: float, ng: int) -> np.ndarray:
    p = _pts64(points)
    cells = np.empty((p.shape[0], 3), dtype=np.int64)
    _check(_load().oracle_point_cells(_ptr(p), p.shape[0], _ptr(_lo(lo)), h, ng, _ptr(cells)), "cells")
    return cells


def bin_points(points, lo, h: float, ng: int) -> dict:
    """Leaf binning: perm, point_box, box_keys, box_ptr (bit-exact reference)."""
    p = _pts64(points)
    n = p.shape[0]
    m = max(n, 1)
    perm = np.empty(m, dtype=np.int32)
    point_box = np.empty(m, dtype=np.int32)
    keys = np.empty(m, dtype=np.int64)
    ptr = np.empty(m + 1, dtype=np.int32)
    nb = np.zeros(1, dtype=np.int32)
    _check(_load().oracle_bin(_ptr(p), n, _ptr(_lo(lo)), h, ng, _ptr(perm), _ptr(point_box),
                              _ptr(keys), _ptr(ptr), _ptr(nb)), "bin")
    B = int(nb[0])
    return {"perm": perm[:n].copy(), "point_box": point_box[:n].copy(), "box_keys": keys[:B].copy(),
            "box_ptr": ptr[:B + 1].copy(), "num_boxes": B}


def neighbors(box_keys, ng: int) -> tuple[np.ndarray, np.ndarray]:
    keys = np.ascontiguousarray(np.asarray(box_keys, dtype=np.int64))
    B = keys.shape[0]
    nptr = np.empty(B + 1, dtype=np.int32)
    nidx = np.empty(max(27 * B, 1), dtype=np.int32)
    _check(_load().oracle_neighbors(_ptr(keys), B, ng, _ptr(nptr), _ptr(nidx)), "neighbors")
    return nptr, nidx[:nptr[-1]].copy()


def p2p(points, lam, lo, h: float, ng: int, k: float, kernel: int = HELMHOLTZ,
        adjoint: bool = False) -> np.ndarray:
    """out = A lam (or A^H lam); lam: (n,) or (n, nrhs) complex. Returns complex128."""
    p = _pts64(points)
    n = p.shape[0]
    l64, nrhs = _lam64(lam, n)
    out = np.zeros((n, nrhs, 2), dtype=np.float64)
    _check(_load().oracle_p2p(_ptr(p), n, _ptr(_lo(lo)), h, ng, kernel, k, int(adjoint), _ptr(l64),
                              nrhs, _ptr(out)), "p2p")
    res = out[..., 0] + 1j * out[..., 1]
    return res[:, 0] if np.asarray(lam).ndim == 1 else res


def p2p_targets(points, lam, targets, lo, h: float, ng: int, k: float, kernel: int = HELMHOLTZ,
                adjoint: bool = False) -> np.ndarray:
    """The same sum for selected targets (original indices) only."""
    p = _pts64(points)
    n = p.shape[0]
    l64, nrhs = _lam64(lam, n)
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
    out = np.zeros((t.shape[0], nrhs, 2), dtype=np.float64)
    _check(_load().oracle_p2p_targets(_ptr(p), n, _ptr(_lo(lo)), h, ng, kernel, k, int(adjoint),
                                      _ptr(l64), nrhs, _ptr(t), t.shape[0], _ptr(out)), "p2p_targets")
    res = out[..., 0] + 1j * out[..., 1]
    return res[:, 0] if np.asarray(lam).ndim == 1 else res


def pair_count(points, lo, h: float, ng: int) -> int:
    p = _pts64(points)
    c = np.zeros(1, dtype=np.int64)
    _check(_load().oracle_pair_count(_ptr(p), p.shape[0], _ptr(_lo(lo)), h, ng, _ptr(c)), "pair_count")
    return int(c[0])


def grad_points(points, lam, g, lo, h: float, ng: int, k: float, kernel: int = HELMHOLTZ) -> np.ndarray:
    """dL/dx (n x 3) for out = A lam with upstream gradient g = dL/dRe(out) + i dL/dIm(out)."""
    p = _pts64(points)
    n = p.shape[0]
    l64, nrhs = _lam64(lam, n)
    g64, nrhs_g = _lam64(g, n)
    if nrhs_g != nrhs:
        raise ValueError("lam and g must have the same number of right-hand sides")
    grad = np.zeros((n, 3), dtype=np.float64)
    _check(_load().oracle_grad_points(_ptr(p), n, _ptr(_lo(lo)), h, ng, kernel, k, _ptr(l64), _ptr(g64),
                                      nrhs, _ptr(grad)), "grad_points")
    return grad


# ---------------------------------------------------- separate point sets --

def neighbors_st(tgt_keys, src_keys, ng: int) -> tuple[np.ndarray, np.ndarray]:
    """Per target box, the source boxes within Chebyshev cell distance 1 (ascending source box id)."""
    tk = np.ascontiguousarray(np.asarray(tgt_keys, dtype=np.int64))
    sk = np.ascontiguousarray(np.asarray(src_keys, dtype=np.int64))
    B = tk.shape[0]
    nptr = np.empty(B + 1, dtype=np.int32)
    nidx = np.empty(max(27 * B, 1), dtype=np.int32)
    _check(_load().oracle_neighbors_st(_ptr(tk), B, _ptr(sk), sk.shape[0], ng, _ptr(nptr), _ptr(nidx)),
           "neighbors_st")
    return nptr, nidx[:nptr[-1]].copy()


def p2p_st(targets, sources, lam, lo, h: float, ng: int, k: float, kernel: int = HELMHOLTZ,
           conj: bool = False) -> np.ndarray:
    """out (n_tgt[, nrhs]) = A lam with A the near field from the source set to the target set (both binned on
    one grid); conj=True gives conj(A) lam.  The adjoint A^H g is p2p_st(sources, targets, g, ..., conj=True)."""
    t = _pts64(targets)
    s = _pts64(sources)
    l64, nrhs = _lam64(lam, s.shape[0])
    out = np.zeros((t.shape[0], nrhs, 2), dtype=np.float64)
    _check(_load().oracle_p2p_st(_ptr(t), t.shape[0], _ptr(s), s.shape[0], _ptr(_lo(lo)), h, ng, kernel, k,
                                 int(conj), _ptr(l64), nrhs, _ptr(out)), "p2p_st")
    res = out[..., 0] + 1j * out[..., 1]
    return res[:, 0] if np.asarray(lam).ndim == 1 else res


def p2p_st_targets(targets, sources, lam, which, lo, h: float, ng: int, k: float, kernel: int = HELMHOLTZ,
                   conj: bool = False) -> np.ndarray:
    """p2p_st for the selected target indices `which` only."""
    t = _pts64(targets)
    s = _pts64(sources)
    l64, nrhs = _lam64(lam, s.shape[0])
    w = np.ascontiguousarray(np.asarray(which, dtype=np.int64))
    out = np.zeros((w.shape[0], nrhs, 2), dtype=np.float64)
    _check(_load().oracle_p2p_st_targets(_ptr(t), t.shape[0], _ptr(s), s.shape[0], _ptr(_lo(lo)), h, ng, kernel,
                                         k, int(conj), _ptr(l64), nrhs, _ptr(w), w.shape[0], _ptr(out)),
           "p2p_st_targets")
    res = out[..., 0] + 1j * out[..., 1]
    return res[:, 0] if np.asarray(lam).ndim == 1 else res
