"""Seeded synthetic inputs for preconditioned-BFGS elastic FWI experiments.

This module is the only code shared by the CUDA path's tests/bench and the
CPU oracle.  It holds no arithmetic of the method itself: only workload
definitions (sizes, acquisition geometry, time axis) and seeded generators of
models, random probing blocks and synthetic BFGS histories.  Models are
evaluated at caller-supplied node coordinates, so each side keeps its own
mesh arithmetic.

The real benchmark models of the paper (the elastic Marmousi model of
Section 3.1 and the Overthrust model of Appendix B) are not available; the
"Marmousi-shaped" generator below stands in for them: seeded folded and
faulted layers whose P speed rises with depth from 1500 to 4700 m/s,
vs = vp / 1.73 and Gardner density rho = 310 vp^0.25.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# workload definitions
# ---------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    nex: int
    nez: int
    h: float
    dt: float
    nt: int
    f0: float
    src_xz: np.ndarray            # [S][2] (x, depth)
    rec_xz: np.ndarray            # [R][2]
    src_type: int = 0             # 0 explosive, 1 force x, 2 force z
    free_top: int = 1
    description: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nx(self):
        return 4 * self.nex + 1

    @property
    def nz(self):
        return 4 * self.nez + 1

    @property
    def nglob(self):
        return self.nx * self.nz

    @property
    def nshot(self):
        return len(self.src_xz)

    @property
    def nrec(self):
        return len(self.rec_xz)

    def sources(self, amp: float = 1.0):
        return [dict(x=float(x), z=float(z), type=self.src_type, f0=self.f0,
                     t0=1.2 / self.f0, amp=amp) for x, z in self.src_xz]


def tiny_homogeneous(nt: int = 1200) -> Workload:
    """40 x 20 elements of 25 m (1000 m x 500 m), free top, Stacey elsewhere,
    one explosive 15 Hz source at x = 500 m, depth 10 m, 41 receivers at
    depth 10 m every 25 m, dt = 0.5 ms."""
    rec = np.stack([25.0 * np.arange(41), np.full(41, 10.0)], axis=1)
    return Workload("homogeneous+anomaly 40x20 (1000x500 m)", 40, 20, 25.0, 5e-4, nt, 15.0,
                    np.array([[500.0, 10.0]]), rec,
                    description="homogeneous vp 3000, vs 1732, rho 2500 with a seeded "
                                "+5% Gaussian vp/vs anomaly (sigma 60 m)")


def marmousi_like_workload(nt: int = 12000, nshot: int = 24, nex: int = 340, nez: int = 70,
                           h: float = 50.0) -> Workload:
    """340 x 70 elements of 50 m (17 km x 3.5 km), 24 explosive 5 Hz sources at
    depth 20 m evenly spaced, 341 surface receivers every 50 m, dt = 0.5 ms."""
    L = nex * h
    sx = L * (np.arange(nshot) + 0.5) / nshot
    src = np.stack([sx, np.full(nshot, 20.0)], axis=1)
    nrec = nex + 1
    rx = np.linspace(0.0, L, nrec)
    rec = np.stack([rx, np.zeros(nrec)], axis=1)
    return Workload(f"marmousi-shaped {nex}x{nez} ({L/1000:g} km x {nez*h/1000:g} km)",
                    nex, nez, h, 5e-4, nt, 5.0, src, rec,
                    description="seeded folded/faulted layers, vp 1500-4700 m/s rising "
                                "with depth, vs = vp/1.73, Gardner density")


def uq_tiny_workload(nt: int = 1500) -> Workload:
    """12 x 6 elements of 50 m (600 m x 300 m), 3 explosive 15 Hz sources at
    depth 20 m, 13 surface receivers every 50 m."""
    src = np.stack([np.array([150.0, 300.0, 450.0]), np.full(3, 20.0)], axis=1)
    rec = np.stack([50.0 * np.arange(13), np.zeros(13)], axis=1)
    return Workload("uq-tiny 12x6 (600x300 m)", 12, 6, 50.0, 5e-4, nt, 15.0, src, rec)


# ---------------------------------------------------------------------------
# models
# ---------------------------------------------------------------------------

def homogeneous(x, z, vp=3000.0, vs=1732.0, rho=2500.0):
    x = np.asarray(x, np.float64)
    return (np.full_like(x, rho), np.full_like(x, vp), np.full_like(x, vs))


def gaussian_anomaly(x, z, seed: int, vp=3000.0, vs=1732.0, rho=2500.0,
                     amp=0.05, sigma=60.0, xrange=(250.0, 750.0), zrange=(150.0, 350.0)):
    """Homogeneous medium plus a +amp Gaussian bump on vp and vs whose centre
    is drawn uniformly from xrange x zrange with the given seed."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(*xrange)
    cz = rng.uniform(*zrange)
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    g = np.exp(-((x - cx) ** 2 + (z - cz) ** 2) / (2 * sigma ** 2))
    return (np.full_like(x, rho), vp * (1 + amp * g), vs * (1 + amp * g))


def _marmousi_vp(x, z, seed, width, depth):
    rng = np.random.default_rng(seed)
    nlay = 12
    zbar = np.sort(rng.uniform(0.04, 0.96, nlay)) * depth
    amp = rng.uniform(20.0, 0.05 * depth, nlay)
    wl = rng.uniform(0.15, 0.5, nlay) * width
    ph = rng.uniform(0, 2 * np.pi, nlay)
    # one shared fold plus per-interface undulation
    fold_amp = rng.uniform(0.03, 0.08) * depth
    fold_wl = rng.uniform(0.3, 0.6) * width
    fold_ph = rng.uniform(0, 2 * np.pi)
    nf = int(rng.integers(2, 5))
    fx = rng.uniform(0.15, 0.85, nf) * width
    fdip = rng.uniform(0.3, 0.8, nf) * rng.choice([-1, 1], nf)   # dx per dz
    fthrow = rng.uniform(0.02, 0.06, nf) * depth
    vfrac = np.arange(1, nlay + 1) / nlay
    jit = rng.uniform(-0.05, 0.05, nlay + 1)
    vlay = np.concatenate([[1500.0], 1500.0 + (4700.0 - 1500.0) * vfrac])
    vlay = np.clip(vlay * (1 + jit), 1500.0, 4700.0)
    vlay = np.maximum.accumulate(vlay)                           # rises with depth

    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    zeff = z.copy()
    for f in range(nf):
        hanging = x > fx[f] + fdip[f] * z
        zeff = np.where(hanging, zeff - fthrow[f], zeff)
    fold = fold_amp * np.sin(2 * np.pi * x / fold_wl + fold_ph)
    idx = np.zeros(x.shape, dtype=np.int64)
    for k in range(nlay):
        zk = zbar[k] + fold + amp[k] * np.sin(2 * np.pi * x / wl[k] + ph[k])
        idx += (zeff > zk).astype(np.int64)
    return vlay[idx]


def marmousi_like(x, z, seed: int, width: float, depth: float):
    """Seeded folded and faulted layered model (rho, vp, vs) at points (x, z)."""
    vp = _marmousi_vp(x, z, seed, width, depth)
    vs = vp / 1.73
    rho = 310.0 * vp ** 0.25
    return rho, vp, vs


def marmousi_like_smooth(x, z, seed: int, width: float, depth: float,
                         sigma: float = 500.0, spacing: float = 25.0):
    """Starting model: the seeded layered model blurred with a Gaussian of
    standard deviation `sigma` metres (on an auxiliary uniform grid), then
    interpolated to the points (x, z)."""
    from scipy.ndimage import gaussian_filter
    from scipy.interpolate import RegularGridInterpolator

    gx = np.arange(0.0, width + spacing / 2, spacing)
    gz = np.arange(0.0, depth + spacing / 2, spacing)
    Z, X = np.meshgrid(gz, gx, indexing="ij")
    vp = _marmousi_vp(X, Z, seed, width, depth)
    vps = gaussian_filter(vp, sigma / spacing, mode="nearest")
    f = RegularGridInterpolator((gz, gx), vps, bounds_error=False, fill_value=None)
    pts = np.stack([np.asarray(z, np.float64).ravel(), np.asarray(x, np.float64).ravel()], axis=1)
    vpi = f(pts).reshape(np.shape(x))
    return 310.0 * vpi ** 0.25, vpi, vpi / 1.73


# ---------------------------------------------------------------------------
# BFGS / UQ inputs
# ---------------------------------------------------------------------------

def gaussian_block(seed: int, p: int, n: int, dtype=np.float32) -> np.ndarray:
    """Seeded standard-normal probing block X[p][n] (numpy PCG64)."""
    return np.random.default_rng(seed).standard_normal((p, n)).astype(dtype)


def synthetic_history(seed: int, n: int, k: int, dtype=np.float32):
    """Seeded BFGS history for inverse-Hessian timing without running FWI:
    s_i ~ N(0, 1) scaled, y_i = A s_i + small noise with A a positive
    diagonal in [1, 10]; pairs with y^T s <= 0 are redrawn.  Returns S, Y
    [k][n] and B0 [n] (a positive diagonal guess)."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(1.0, 10.0, n)
    S = np.empty((k, n), np.float64)
    Y = np.empty((k, n), np.float64)
    i = 0
    while i < k:
        s = rng.standard_normal(n) * 1e-2
        y = A * s + 1e-3 * np.linalg.norm(A * s) / np.sqrt(n) * rng.standard_normal(n)
        if y @ s > 0:
            S[i], Y[i] = s, y
            i += 1
    B0 = (1.0 / A) * rng.uniform(0.5, 2.0, n)
    return S.astype(dtype), Y.astype(dtype), B0.astype(dtype)


def quadratic_problem(seed: int, n: int):
    """Seeded strongly convex quadratic f(x) = 1/2 x^T A x - b^T x (SPD A)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.exp(rng.uniform(0.0, 3.0, n))
    A = (Q * ev) @ Q.T
    b = rng.standard_normal(n)
    return 0.5 * (A + A.T), b
