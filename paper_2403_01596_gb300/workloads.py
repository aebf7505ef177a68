"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and fixes the grid / wavenumber of each
workload.  It holds none of the operator's arithmetic (no binning, no
neighbour search, no kernel evaluation), so both the FP64 oracle tests and the
CUDA path can take their inputs from it.

The paper measures on random source/target points spread over a surface (a
2D PEC plate, Sec. 4); these generators stand in for that with 3D point
clouds: uniform in a cube, on a sphere, on a 2:1:1 ellipsoid, and on a
cylinder-plus-plates assembly with clustered sampling.  Coordinates are drawn
in float64 with numpy's default_rng(seed) and rounded to float32; that float32
array is the canonical input for every consumer.  Strengths lambda have real
and imaginary parts i.i.d. N(0, 1) from default_rng(seed + 100).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclass
class Workload:
    """Points plus the uniform leaf grid [lo, lo + ng*h)^3 and wavenumber k."""
    name: str
    points: np.ndarray          # (n, 3) float32
    lo: tuple                   # grid origin (3 floats)
    h: float                    # leaf box edge
    ng: int                     # leaf boxes per axis
    k: float                    # Helmholtz wavenumber
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])


def _to_f32(p: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(p.astype(np.float32))


def uniform_cube(n: int, seed: int) -> np.ndarray:
    """n points uniform in [0, 1)^3."""
    rng = np.random.default_rng(seed)
    return _to_f32(rng.random((n, 3)))


def unit_sphere(n: int, seed: int) -> np.ndarray:
    """n points uniform on the unit sphere surface (normalised Gaussian vectors)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return _to_f32(v)


def ellipsoid_211(n: int, seed: int) -> np.ndarray:
    """n points area-uniform on the ellipsoid with semi-axes (2, 1, 1).

    A unit-sphere sample u is mapped to (2 u_x, u_y, u_z) and accepted with
    probability sqrt(u_x^2 + 4 u_y^2 + 4 u_z^2) / 2, the ratio of the
    ellipsoid's area element to its maximum.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = int(1.4 * (n - out.shape[0])) + 1024
        u = rng.standard_normal((m, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        w = np.sqrt(u[:, 0] ** 2 + 4 * u[:, 1] ** 2 + 4 * u[:, 2] ** 2) / 2.0
        keep = rng.random(m) < w
        p = u[keep] * np.array([2.0, 1.0, 1.0])
        out = np.concatenate([out, p])
    return _to_f32(out[:n])


def cylinder_plates(n: int, seed: int, sigma: float = 0.02, clusters: int = 64) -> np.ndarray:
    """Open cylinder (radius 0.5, z in [-1, 1]) plus two 2x2 plates at z = +-1.25.

    Half the points are uniform by area; the other half come from `clusters`
    Gaussian clusters (std `sigma` in arc-length / plate coordinates) whose
    centres are uniform by area.
    """
    rng = np.random.default_rng(seed)
    a_cyl, a_plate = 2.0 * math.pi * 0.5 * 2.0, 4.0
    probs = np.array([a_cyl, a_plate, a_plate]) / (a_cyl + 2 * a_plate)

    def surface_params(m):
        part = rng.choice(3, size=m, p=probs)
        s = np.where(part == 0, rng.random(m) * TWO_PI * 0.5, rng.random(m) * 2.0 - 1.0)
        t = np.where(part == 0, rng.random(m) * 2.0 - 1.0, rng.random(m) * 2.0 - 1.0)
        return part, s, t

    def embed(part, s, t):
        p = np.empty((part.shape[0], 3))
        cyl = part == 0
        th = s[cyl] / 0.5
        p[cyl, 0] = 0.5 * np.cos(th)
        p[cyl, 1] = 0.5 * np.sin(th)
        p[cyl, 2] = np.clip(t[cyl], -1.0, 1.0)
        for q, z in ((1, -1.25), (2, 1.25)):
            sel = part == q
            p[sel, 0] = np.clip(s[sel], -1.0, 1.0)
            p[sel, 1] = np.clip(t[sel], -1.0, 1.0)
            p[sel, 2] = z
        return p

    n_uni = n // 2
    n_clu = n - n_uni
    part_u, s_u, t_u = surface_params(n_uni)
    cpart, cs, ct = surface_params(max(1, clusters))
    which = rng.integers(0, max(1, clusters), size=n_clu)
    part_c = cpart[which]
    s_c = cs[which] + sigma * rng.standard_normal(n_clu)
    t_c = ct[which] + sigma * rng.standard_normal(n_clu)
    # the cylinder's arc-length coordinate wraps around its circumference; coordinates that leave
    # [-1, 1] (plate sides, cylinder height) are mirrored back so no edge collects points
    def mirror(x):
        y = np.mod(x + 1.0, 4.0)
        return 1.0 - np.abs(y - 2.0)
    s_c = np.where(part_c == 0, np.mod(s_c, TWO_PI * 0.5), mirror(s_c))
    t_c = mirror(t_c)
    pts = np.concatenate([embed(part_u, s_u, t_u), embed(part_c, s_c, t_c)])
    pts = pts[rng.permutation(n)]
    return _to_f32(pts)


#: area of the cylinder-plus-plates surface
CYLINDER_PLATES_AREA = 2.0 * math.pi * 0.5 * 2.0 + 2 * 4.0


def strengths(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Complex64 strengths (n,) for nrhs == 1 or (n, nrhs): re, im i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed + 100)
    re = rng.standard_normal((n, nrhs))
    im = rng.standard_normal((n, nrhs))
    lam = (re + 1j * im).astype(np.complex64)
    return lam[:, 0].copy() if nrhs == 1 else np.ascontiguousarray(lam)


# ------------------------------------------------------------------ configs --

def cube_dense(n: int = 32768, seed: int = 0) -> Workload:
    """Uniform unit cube, 8^3 leaf grid (~64 points per box at n = 32768), k = 2 pi * 4."""
    return Workload("cube_uniform_8x8x8", uniform_cube(n, seed), (0.0, 0.0, 0.0), 0.125, 8,
                    TWO_PI * 4.0, seed, {"shape": "cube", "target_occupancy": n / 512})


#: leaf grid per target mean occupancy on the unit sphere with n = 2^20 points
SPHERE_GRID = {8: 180, 16: 124, 32: 86, 64: 61}


def sphere_density(occupancy: int, n: int = 1 << 20, seed: int = 1) -> Workload:
    """Unit sphere surface in [-1, 1]^3; leaf edge = 0.25 wavelength."""
    ng = SPHERE_GRID[occupancy]
    h = 2.0 / ng
    return Workload(f"sphere_n{n}_d{occupancy}", unit_sphere(n, seed), (-1.0, -1.0, -1.0), h, ng,
                    TWO_PI / (4.0 * h), seed, {"shape": "sphere", "target_occupancy": occupancy})


def ellipsoid_multirhs(n: int = 1 << 21, seed: int = 2) -> Workload:
    """2:1:1 ellipsoid in [-2, 2]^3, 188^3 grid (~32 points per box), leaf edge = 0.2 wavelength."""
    ng = 188
    h = 4.0 / ng
    return Workload(f"ellipsoid211_n{n}", ellipsoid_211(n, seed), (-2.0, -2.0, -2.0), h, ng,
                    TWO_PI / (5.0 * h), seed, {"shape": "ellipsoid211", "target_occupancy": 32})


def sphere_grad(n: int = 1 << 18, seed: int = 3) -> Workload:
    """Unit sphere, 62^3 grid (~16 points per box), k = 2 pi * 8."""
    ng = 62
    return Workload(f"sphere_grad_n{n}", unit_sphere(n, seed), (-1.0, -1.0, -1.0), 2.0 / ng, ng,
                    TWO_PI * 8.0, seed, {"shape": "sphere", "target_occupancy": 16})


#: sizes of the eight geometries of the batched uneven workload (40M points in total)
BATCH_SIZES = (500_000, 1_000_000, 2_000_000, 3_000_000, 4_000_000, 6_000_000, 7_500_000, 16_000_000)


def batch_geometry(g: int, scale: float = 1.0) -> dict:
    """Geometry g of the batched workload: points, leaf grid and leaf edge in wavelengths.

    The leaf edge h is chosen so that the uniform half of the points fills the
    surface boxes at about 6 points per box (a surface box holds ~h^2 of area);
    the clustered half comes in clusters of ~2000 points with std 2h, whose peak
    occupancy is ~2000 / (8 pi) + 6, about 90 points per box.  Box occupancy
    therefore spans 1 to ~128.  The grid covers [-1.3, 1.3]^3; the wavenumber
    follows from h as k = 2 pi * edge / h.
    """
    n = max(1, int(round(BATCH_SIZES[g] * scale)))
    h = math.sqrt(CYLINDER_PLATES_AREA * 6.0 / max(n // 2, 1))
    ng = max(1, int(math.ceil(2.6 / h)))
    h = 2.6 / ng
    clusters = max(1, (n - n // 2) // 2000)
    return {"points": cylinder_plates(n, 10 + g, sigma=2.0 * h, clusters=clusters), "lo": (-1.3, -1.3, -1.3),
            "extent": 2.6, "h": h, "ng": ng, "edge_wavelengths": 0.1 + 0.2 * g / 7.0, "seed": 10 + g, "nrhs": 8}
