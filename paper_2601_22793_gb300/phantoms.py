"""Seeded synthetic inputs for eikonal phase retrieval.

These stand in for the paper's HiP-CT and bamboo radiographs, which are not
available.  The module holds geometry and random numbers only: analytic
projected thickness of spheres and ellipsoids, spectrum tables and Poisson
counting noise.  It contains none of the retrieval arithmetic (no transport,
no filter, no solver), so that the FP64 oracle and the CUDA library can both
take their inputs from it.

All thickness maps are in metres, row-major ``[ny][nx]`` (y = row index).
Random streams are numpy PCG64, seeded by the caller.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Materials (refractive index decrement delta, absorption index beta).
BONE = (2e-7, 1e-10)
WATER = (6e-8, 1e-11)
TISSUE = (6e-8, 1e-11)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# spheres
# --------------------------------------------------------------------------

def spheres(ny: int, nx: int, n_spheres: int, r_min: float, r_max: float,
            margin: float, pixel: float, seed: int) -> np.ndarray:
    """Sum of analytic chord lengths 2 sqrt(r^2 - rho^2) (metres) of
    ``n_spheres`` spheres with radii U[r_min, r_max] px and centres at least
    r + margin px from every edge."""
    g = rng(seed)
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    tau = np.zeros((ny, nx))
    for _ in range(n_spheres):
        r = g.uniform(r_min, r_max)
        lo = r + margin
        cy = g.uniform(lo, ny - 1 - lo)
        cx = g.uniform(lo, nx - 1 - lo)
        rho2 = (yy - cy) ** 2 + (xx - cx) ** 2
        tau += 2.0 * np.sqrt(np.clip(r * r - rho2, 0.0, None))
    return tau * pixel


# --------------------------------------------------------------------------
# ellipsoids
# --------------------------------------------------------------------------

@dataclass
class Ellipsoid:
    centre: np.ndarray   # (x, y, z) in px, object frame
    axes: np.ndarray     # semi-axes (a, b, c) in px
    rot: np.ndarray      # 3x3 rotation, columns = principal directions
    weight: float        # phase-equivalent thickness factor of the material


def _random_rotation(g: np.random.Generator) -> np.ndarray:
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_ellipsoids(ny: int, nx: int, n: int, semi_min: float, semi_max: float,
                      fractions=(0.5, 0.35, 0.15), weights=(0.3, 1.0, -0.3),
                      margin: float = 12.0, seed: int = 0) -> list[Ellipsoid]:
    """``n`` ellipsoids with semi-axes U[semi_min, semi_max] px and random
    orientation; materials tissue / bone / void drawn with ``fractions``.
    ``weights`` are the phase-equivalent factors delta_m / delta_ref (tissue
    6e-8 / 2e-7 = 0.3, bone 1, a void inside tissue removes 0.3).  Voids are
    centred inside an earlier tissue ellipsoid when there is one.  Every
    ellipsoid keeps its projected extent ``margin`` px inside the field of
    view for all rotations about y (the extent uses the largest semi-axis)."""
    g = rng(seed)
    out: list[Ellipsoid] = []
    tissues: list[Ellipsoid] = []
    for _ in range(n):
        kind = g.choice(3, p=np.asarray(fractions, dtype=np.float64))
        axes = g.uniform(semi_min, semi_max, size=3)
        rot = _random_rotation(g)
        if kind == 2 and tissues:
            host = tissues[int(g.integers(len(tissues)))]
            axes = np.minimum(axes, 0.6 * host.axes.min())
            offs = g.uniform(-0.3, 0.3, size=3) * host.axes.min()
            centre = host.centre + offs
        else:
            ext = axes.max() + margin
            half = 0.5 * min(nx, ny)
            lo_x, hi_x = ext, nx - 1 - ext
            lo_y, hi_y = ext, ny - 1 - ext
            if lo_x >= hi_x or lo_y >= hi_y:
                axes = axes * (0.45 * min(nx, ny) - margin) / axes.max()
                ext = axes.max() + margin
                lo_x, hi_x, lo_y, hi_y = ext, nx - 1 - ext, ext, ny - 1 - ext
            cx = g.uniform(lo_x, hi_x)
            cy = g.uniform(lo_y, hi_y)
            # z stays within the x extent so rotations about y keep it inside
            cz = g.uniform(-(half - ext), (half - ext)) if half > ext else 0.0
            centre = np.array([cx, cy, cz])
        e = Ellipsoid(centre=np.asarray(centre, dtype=np.float64), axes=axes, rot=rot,
                      weight=float(weights[kind]))
        out.append(e)
        if kind == 0:
            tissues.append(e)
    return out


def project_ellipsoids(ells: list[Ellipsoid], ny: int, nx: int, pixel: float,
                       angle: float = 0.0, clamp: bool = True) -> np.ndarray:
    """Phase-equivalent projected thickness (metres) along z after rotating
    the object by ``angle`` (radians) about the y axis through the centre of
    the field of view: sum over ellipsoids of weight * chord length.  The
    chord through {v : (v-c)^T A (v-c) <= 1} along z at transverse (x, y) is
    2 sqrt(disc) / A_zz with disc = b^2 - A_zz (q - 1), b = A_xz dx + A_yz dy,
    q = A_xx dx^2 + 2 A_xy dx dy + A_yy dy^2."""
    return _project(ells, ny, nx, pixel, angle, clamp, lambda e: e.weight)


def project_materials(ells: list[Ellipsoid], ny: int, nx: int, pixel: float,
                      angle: float = 0.0) -> np.ndarray:
    """Chord lengths (metres) through each material of a tissue / bone /
    void phantom of ``random_ellipsoids`` (default weights): [2][ny][nx],
    tissue net of the voids inside it, then bone, each clamped at 0.  With
    the phase-equivalent factors 0.3 and 1 they sum to project_ellipsoids
    wherever no void reaches past its tissue."""
    tissue = _project(ells, ny, nx, pixel, angle, True,
                      lambda e: 1.0 if e.weight == 0.3 else (-1.0 if e.weight == -0.3 else 0.0))
    bone = _project(ells, ny, nx, pixel, angle, True, lambda e: 1.0 if e.weight == 1.0 else 0.0)
    return np.stack([tissue, bone])


def _project(ells, ny, nx, pixel, angle, clamp, factor) -> np.ndarray:
    ca, sa = np.cos(angle), np.sin(angle)
    Ry = np.array([[ca, 0.0, sa], [0.0, 1.0, 0.0], [-sa, 0.0, ca]])
    ox, oz = 0.5 * (nx - 1), 0.0
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    tau = np.zeros((ny, nx))
    for e in ells:
        R = Ry @ e.rot
        A = R @ np.diag(1.0 / e.axes ** 2) @ R.T
        c0 = e.centre - np.array([ox, 0.0, oz])
        c = Ry @ c0 + np.array([ox, 0.0, oz])
        # bounding box of the projection
        Ainv = np.linalg.inv(A)
        hx = np.sqrt(Ainv[0, 0]) + 1.0
        hy = np.sqrt(Ainv[1, 1]) + 1.0
        x0, x1 = max(0, int(np.floor(c[0] - hx))), min(nx, int(np.ceil(c[0] + hx)) + 1)
        y0, y1 = max(0, int(np.floor(c[1] - hy))), min(ny, int(np.ceil(c[1] + hy)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        dx = xx[y0:y1, x0:x1] - c[0]
        dy = yy[y0:y1, x0:x1] - c[1]
        b = A[0, 2] * dx + A[1, 2] * dy
        q = A[0, 0] * dx * dx + 2.0 * A[0, 1] * dx * dy + A[1, 1] * dy * dy
        disc = b * b - A[2, 2] * (q - 1.0)
        chord = 2.0 * np.sqrt(np.clip(disc, 0.0, None)) / A[2, 2]
        tau[y0:y1, x0:x1] += factor(e) * chord
    if clamp:
        np.clip(tau, 0.0, None, out=tau)
    return tau * pixel


# --------------------------------------------------------------------------
# spectrum
# --------------------------------------------------------------------------

def spectrum(n_lines: int, e_lo: float, e_hi: float, centre: float, sigma: float,
             delta_ref: float, beta_ref: float, e_ref: float, seed: int):
    """Line energies E_s = linspace(e_lo, e_hi, n_lines) keV; weights a
    Gaussian(centre, sigma) times (1 + 0.1 sin) with a seeded phase,
    normalised to sum 1; delta_s = delta_ref (e_ref/E_s)^2 and beta_s =
    beta_ref (e_ref/E_s)^4 (away-from-edge scalings)."""
    g = rng(seed)
    E = np.linspace(e_lo, e_hi, n_lines) if n_lines > 1 else np.array([0.5 * (e_lo + e_hi)])
    ph = g.uniform(0.0, 2.0 * np.pi)
    w = np.exp(-0.5 * ((E - centre) / sigma) ** 2) * (1.0 + 0.1 * np.sin(E / 10.0 + ph))
    w /= w.sum()
    delta = delta_ref * (e_ref / E) ** 2
    beta = beta_ref * (e_ref / E) ** 4
    return E, delta, beta, w


# --------------------------------------------------------------------------
# noise
# --------------------------------------------------------------------------

def poisson(P: np.ndarray, photons: float, seed: int) -> np.ndarray:
    """Counting noise: Poisson(photons * P) / photons (flat field = 1)."""
    g = rng(seed)
    lam = np.clip(np.asarray(P, dtype=np.float64), 0.0, None) * photons
    return g.poisson(lam).astype(np.float64) / photons


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    ny: int
    nx: int
    pixel: float
    L: float
    energy_keV: np.ndarray
    delta: np.ndarray
    beta: np.ndarray
    weights: np.ndarray
    n_iter: int
    omega: float
    photons: float


def spheres_mono_256(seed: int = 1000) -> tuple[Workload, np.ndarray]:
    """One monochromatic 256 x 256 projection: 8 spheres (radius 10-40 px) of
    bone in water, E = 60 keV, L = 2 m, p = 6.5 um, 20 iterations.  The
    retrieval material is the bone-water difference (water is a uniform slab
    folded into the flat field)."""
    wl = Workload("spheres_mono_256", 256, 256, 6.5e-6, 2.0, np.array([60.0]),
                  np.array([BONE[0] - WATER[0]]), np.array([BONE[1] - WATER[1]]),
                  np.array([1.0]), 20, 1.0, 1e4)
    tau = spheres(256, 256, 8, 10.0, 40.0, 4.0, wl.pixel, seed)
    return wl, tau


def ellipsoids_mono(n: int = 2048, n_ell: int = 200, seed: int = 2000,
                    semi=(8.0, 120.0), n_iter: int = 50, omega: float = 0.4):
    """Monochromatic n x n projection of ``n_ell`` ellipsoids (bone, tissue,
    voids; semi-axes ``semi`` px), E = 80 keV, L = 30 m, p = 20 um; bone is
    the retrieval material.  2048 / 200 / (8, 120) is the full-size case."""
    wl = Workload(f"ellipsoids_mono_{n}", n, n, 20e-6, 30.0, np.array([80.0]),
                  np.array([BONE[0]]), np.array([BONE[1]]), np.array([1.0]),
                  n_iter, omega, 1e4)
    ells = random_ellipsoids(n, n, n_ell, semi[0], semi[1], seed=seed)
    tau = project_ellipsoids(ells, n, n, wl.pixel)
    return wl, tau


def ellipsoids_poly(n: int = 2048, n_proj: int = 64, n_lines: int = 8, n_ell: int = 200,
                    seed: int = 3000, semi=(8.0, 120.0), n_iter: int = 50,
                    omega: float = 0.4):
    """Polychromatic set: the same 3-D ellipsoid phantom projected at angles
    j pi / n_proj about y; ``n_lines`` lines 60-160 keV, Gaussian(95, 30)
    weights, delta ~ E^-2, beta ~ E^-4 referenced to bone at 80 keV."""
    E, d, b, w = spectrum(n_lines, 60.0, 160.0, 95.0, 30.0, BONE[0], BONE[1], 80.0, seed)
    wl = Workload(f"ellipsoids_poly_{n}x{n_proj}x{n_lines}", n, n, 20e-6, 30.0, E, d, b, w,
                  n_iter, omega, 1e4)
    ells = random_ellipsoids(n, n, n_ell, semi[0], semi[1], seed=seed)
    angles = [j * np.pi / n_proj for j in range(n_proj)]
    return wl, ells, angles
