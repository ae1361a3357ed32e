"""Python face of the FP64 spectral-element oracle (``sem_ref.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function here is
a thin marshalling layer over the C oracle plus the few steps the paper states
in words (misfit, damping and inversion of the preconditioner).

Conventions: node grid ``[nz][nx]`` with ``nx = 4 nex + 1``, ``nz = 4 nez + 1``,
row 0 at the surface, ``z`` = depth.  Vector fields are ``[nz][nx][2]``.
Seismograms are ``[nrec][2][nt]`` with column ``n-1`` holding step ``n``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sem_ref.c")
_OUT = os.path.join(_HERE, "_build", "libsemref.so")
_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build() -> str:
    """Compile the C oracle with gcc (IEEE FP64, no fast-math)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not os.path.exists(_OUT)) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build())
    return _LIB


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_ip)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# mesh-level helpers
# ---------------------------------------------------------------------------

def gll():
    xi, w, D = np.zeros(5), np.zeros(5), np.zeros(25)
    _lib().ref_gll(_d(xi), _d(w), _d(D))
    return xi, w, D.reshape(5, 5)


def lagrange(s: float):
    l, dl = np.zeros(5), np.zeros(5)
    _lib().ref_lagrange(ctypes.c_double(s), _d(l), _d(dl))
    return l, dl


@dataclass
class Mesh:
    nex: int
    nez: int
    h: float

    @property
    def nx(self) -> int:
        return 4 * self.nex + 1

    @property
    def nz(self) -> int:
        return 4 * self.nez + 1

    @property
    def N(self) -> int:
        return self.nx * self.nz

    def _a(self):
        return ctypes.c_int(self.nex), ctypes.c_int(self.nez), ctypes.c_double(self.h)

    def coords(self):
        x, z = np.zeros(self.N), np.zeros(self.N)
        _lib().ref_node_coords(*self._a(), _d(x), _d(z))
        return x.reshape(self.nz, self.nx), z.reshape(self.nz, self.nx)

    def mass(self, rho):
        M = np.zeros(self.N)
        _lib().ref_mass(*self._a(), _d(_c(rho).ravel()), _d(M))
        return M.reshape(self.nz, self.nx)

    def measure(self):
        W = np.zeros(self.N)
        _lib().ref_node_measure(*self._a(), _d(W))
        return W.reshape(self.nz, self.nx)

    def stacey(self, rho, vp, vs, free_top=1, absorb=1):
        C = np.zeros(2 * self.N)
        _lib().ref_stacey(*self._a(), ctypes.c_int(free_top), ctypes.c_int(absorb),
                          _d(_c(rho).ravel()), _d(_c(vp).ravel()), _d(_c(vs).ravel()), _d(C))
        return C.reshape(self.nz, self.nx, 2)

    def stiffness(self, lam, mu, u):
        Ku = np.zeros(2 * self.N)
        _lib().ref_stiffness(*self._a(), _d(_c(lam).ravel()), _d(_c(mu).ravel()),
                             _d(_c(u).ravel()), _d(Ku))
        return Ku.reshape(self.nz, self.nx, 2)

    def interp(self, x: float, z: float):
        idx = np.zeros(25, dtype=np.int32)
        w = np.zeros(25)
        rc = _lib().ref_interp(*self._a(), ctypes.c_double(x), ctypes.c_double(z), _i(idx), _d(w))
        if rc:
            raise ValueError(f"point ({x}, {z}) outside the mesh")
        return idx, w

    def receivers(self, rec_xz):
        rec_xz = np.asarray(rec_xz, dtype=np.float64).reshape(-1, 2)
        idx = np.zeros((len(rec_xz), 25), dtype=np.int32)
        w = np.zeros((len(rec_xz), 25))
        for r, (x, z) in enumerate(rec_xz):
            idx[r], w[r] = self.interp(x, z)
        return idx, w

    def source_vector(self, x: float, z: float, kind: int = 0, amp: float = 1.0):
        f = np.zeros(2 * self.N)
        rc = _lib().ref_source_vector(*self._a(), ctypes.c_double(x), ctypes.c_double(z),
                                      ctypes.c_int(kind), ctypes.c_double(amp), _d(f))
        if rc:
            raise ValueError(f"bad source ({x}, {z}, type {kind})")
        return f.reshape(self.nz, self.nx, 2)

    def smooth(self, field, sigma: float):
        out = np.zeros(self.N)
        _lib().ref_smooth(*self._a(), _d(_c(field).ravel()), ctypes.c_double(sigma), _d(out))
        return out.reshape(self.nz, self.nx)


def ricker(nt: int, dt: float, f0: float, t0: float, amp: float = 1.0) -> np.ndarray:
    stf = np.zeros(nt + 1)
    _lib().ref_ricker(ctypes.c_int(nt), ctypes.c_double(dt), ctypes.c_double(f0),
                      ctypes.c_double(t0), ctypes.c_double(amp), _d(stf))
    return stf


def lame(rho, vp, vs):
    """lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2 (Eq. A7 with lambda + 2 mu = rho vp^2)."""
    rho, vp, vs = _c(rho), _c(vp), _c(vs)
    return rho * (vp ** 2 - 2 * vs ** 2), rho * vs ** 2


# ---------------------------------------------------------------------------
# simulations
# ---------------------------------------------------------------------------

@dataclass
class Setup:
    """Mesh, boundary flags, time axis and receivers of one experiment."""
    mesh: Mesh
    dt: float
    nt: int
    rec_xz: np.ndarray
    free_top: int = 1
    absorb: int = 1

    def __post_init__(self):
        self.rec_xz = np.asarray(self.rec_xz, dtype=np.float64).reshape(-1, 2)
        self.ridx, self.rw = self.mesh.receivers(self.rec_xz)

    @property
    def nrec(self) -> int:
        return len(self.rec_xz)

    def _hdr(self):
        m = self.mesh
        return (ctypes.c_int(m.nex), ctypes.c_int(m.nez), ctypes.c_double(m.h),
                ctypes.c_int(self.free_top), ctypes.c_int(self.absorb))

    def source(self, src):
        """(force vector, source time function) of a source dict
        {x, z, type, f0, t0, amp}: Ricker in time, amp folded into the wavelet."""
        f = self.mesh.source_vector(src["x"], src["z"], int(src.get("type", 0)), 1.0)
        stf = ricker(self.nt, self.dt, src["f0"], src.get("t0", 1.2 / src["f0"]), src.get("amp", 1.0))
        return f, stf

    def forward(self, model, fvec, stf, keep=False):
        """Records [nrec][2][nt]; with keep=True also u_n, a_n for n = 0..nt."""
        rho, vp, vs = (_c(a).ravel() for a in model)
        N, nt = self.mesh.N, self.nt
        seis = np.zeros(self.nrec * 2 * nt)
        uh = np.zeros((nt + 1) * 2 * N) if keep else None
        ah = np.zeros((nt + 1) * 2 * N) if keep else None
        rc = _lib().ref_forward(*self._hdr(), _d(rho), _d(vp), _d(vs),
                                _d(_c(fvec).ravel()), _d(_c(stf)),
                                ctypes.c_int(self.nrec), _i(self.ridx.ravel()), _d(self.rw.ravel()),
                                ctypes.c_double(self.dt), ctypes.c_int(nt), _d(seis),
                                _d(uh) if keep else None, _d(ah) if keep else None)
        if rc:
            raise FloatingPointError("oracle forward field became non-finite")
        seis = seis.reshape(self.nrec, 2, nt)
        if keep:
            return seis, uh.reshape(nt + 1, self.mesh.nz, self.mesh.nx, 2), \
                ah.reshape(nt + 1, self.mesh.nz, self.mesh.nx, 2)
        return seis

    def adjoint(self, model, gsrc):
        """lam_0..lam_{nt+1} for the adjoint source g_k = gsrc[:, :, k-1]."""
        rho, vp, vs = (_c(a).ravel() for a in model)
        N, nt = self.mesh.N, self.nt
        lh = np.zeros((nt + 2) * 2 * N)
        rc = _lib().ref_adjoint(*self._hdr(), _d(rho), _d(vp), _d(vs),
                                ctypes.c_int(self.nrec), _i(self.ridx.ravel()), _d(self.rw.ravel()),
                                _d(_c(gsrc).ravel()), ctypes.c_double(self.dt), ctypes.c_int(nt), _d(lh))
        if rc:
            raise FloatingPointError("oracle adjoint field became non-finite")
        return lh.reshape(nt + 2, self.mesh.nz, self.mesh.nx, 2)

    def gradient_from(self, model, u_hist, lam_hist):
        rho, vp, vs = (_c(a).ravel() for a in model)
        N = self.mesh.N
        g = np.zeros(3 * N)
        _lib().ref_gradient(*self._hdr(), _d(rho), _d(vp), _d(vs),
                            _d(_c(u_hist).ravel()), _d(_c(lam_hist).ravel()),
                            ctypes.c_double(self.dt), ctypes.c_int(self.nt), _d(g))
        return g.reshape(3, self.mesh.nz, self.mesh.nx)

    def precond_sums(self, uA, aA, uB, aB):
        """The four signed time integrals of Eqs. 5-8 (see ref_precond_sums)."""
        m = self.mesh
        S = np.zeros(4 * m.N)
        _lib().ref_precond_sums(ctypes.c_int(m.nex), ctypes.c_int(m.nez), ctypes.c_double(m.h),
                                _d(_c(uA).ravel()), _d(_c(aA).ravel()),
                                _d(_c(uB).ravel()), _d(_c(aB).ravel()),
                                ctypes.c_double(self.dt), ctypes.c_int(self.nt), _d(S))
        return S.reshape(4, m.nz, m.nx)


def misfit(dt: float, syn: np.ndarray, obs: np.ndarray) -> float:
    """f = 1/2 dt sum |s - d|^2 (Eq. A1, rectangle rule in time)."""
    r = np.asarray(syn, np.float64) - np.asarray(obs, np.float64)
    return 0.5 * dt * float(np.sum(r * r))


def misfit_gradient(st: Setup, model, sources, d_obs):
    """Misfit and gradient summed over shots; d_obs[s] is [nrec][2][nt].

    Returns (f, grad[3][nz][nx] in the order rho, vp, vs, synthetics)."""
    f = 0.0
    grad = np.zeros((3, st.mesh.nz, st.mesh.nx))
    syns = []
    for s, src in enumerate(sources):
        fvec, stf = st.source(src)
        seis, uh, _ = st.forward(model, fvec, stf, keep=True)
        syns.append(seis)
        r = seis - d_obs[s]
        f += misfit(st.dt, seis, d_obs[s])
        lam = st.adjoint(model, st.dt * r)          # df/du_k = dt P^T r_k
        grad += st.gradient_from(model, uh, lam)
    return f, grad, np.stack(syns)


def accel_from_hist(u_hist: np.ndarray, dt: float) -> np.ndarray:
    """Second difference (u_{n+1} - 2 u_n + u_{n-1}) / dt^2 at n = 1..len-2,
    stored at index n (entries 0 and len-1 zero)."""
    a = np.zeros_like(u_hist)
    a[1:-1] = (u_hist[2:] - 2.0 * u_hist[1:-1] + u_hist[:-2]) / (dt * dt)
    return a


def receiver_field(st: Setup, model, seis):
    """Receiver wavefield of Eqs. 6 and 8: the backward simulation driven by
    the synthetic data s(m0) (Appendix A, after Eq. A22).  Returns the
    displacement lam_n and its acceleration for n = 0..nt."""
    nt = st.nt
    lam = st.adjoint(model, st.dt * seis)
    acc = np.zeros_like(lam[: nt + 1])
    acc[1:] = (lam[2:nt + 2] - 2.0 * lam[1:nt + 1] + lam[0:nt]) / (st.dt ** 2)
    return lam[: nt + 1], acc


def precond_maps(model, W, S, kind: int):
    """Diagonal Hessian maps [3][nz][nx] for (rho, vp, vs) from the signed
    integrals S (summed over shots):
      H_rho = W |S0|                                  (Eq. 5/6, A21c/A22c)
      H_a   = 8 rho^2 vp^2 |S1|                        (Eq. 7/8, A21a/A22a)
      H_b   = 16 rho^2 vs^2 |S2| + 4 rho^2 vs^2 |S3|   (Eq. 7/8, A21b/A22b)
    P1/P2 use H_rho for every parameter (Eqs. 5-6 impose one map on alpha
    and beta); P3/P4 use (H_rho, H_a, H_b).  For P1/P3 the integrals are
    sums of squares, so the absolute value changes nothing."""
    rho, vp, vs = (_c(a) for a in model)
    r2 = rho * rho
    Hr = W * np.abs(S[0])
    if kind in (1, 2):
        return np.stack([Hr, Hr, Hr])
    Ha = 8.0 * r2 * vp * vp * np.abs(S[1])
    Hb = 16.0 * r2 * vs * vs * np.abs(S[2]) + 4.0 * r2 * vs * vs * np.abs(S[3])
    return np.stack([Hr, Ha, Hb])


def precond_raw(st: Setup, model, sources, kind: int):
    """Unsmoothed diagonal Hessian of kind 1..4 (Eqs. 5-8) summed over shots.
    P1/P3 correlate the source wavefield with itself, P2/P4 with the receiver
    wavefield; the time integrals are summed over shots before |.|."""
    if kind not in (1, 2, 3, 4):
        raise ValueError("kind must be 1..4")
    S = np.zeros((4, st.mesh.nz, st.mesh.nx))
    for src in sources:
        fvec, stf = st.source(src)
        seis, uh, ah = st.forward(model, fvec, stf, keep=True)
        if kind in (1, 3):
            S += st.precond_sums(uh, ah, uh, ah)
        else:
            lb, ab = receiver_field(st, model, seis)
            S += st.precond_sums(uh, ah, lb, ab)
    return precond_maps(model, st.mesh.measure(), S, kind)


def smooth_damp_invert(st: Setup, H, sigma: float, damp_factor: float = 1.0):
    """Smoothing, damping and inversion of a diagonal Hessian (Eq. 4 and the
    Marmousi set-up): each parameter map is Gaussian-smoothed, damped by
    lambda = damp_factor x median of the smoothed map, and inverted:
      B0 = 1 / (S(H) + lambda).
    Returns (smoothed H, B0), both [3][nz][nx]."""
    Hs = np.stack([st.mesh.smooth(H[c], sigma) for c in range(3)])
    B0 = np.empty_like(Hs)
    for c in range(3):
        flat = np.sort(Hs[c].ravel())
        med = flat[(flat.size - 1) // 2]           # lower median
        B0[c] = 1.0 / (Hs[c] + damp_factor * med)
    return Hs, B0
