"""GB300 (sm_103a) preconditioned-BFGS elastic FWI with low-rank uncertainty
quantification (Liu, Beller, Lei, Peter & Tromp 2020).

Python face of the C ABI in ``include/gbfwi.h``.  The entry points keep the
ABI's names:

    mesh_create, set_model, forward, adjoint_gradient, precond_diag,
    bfgs_create, bfgs_update, bfgs_apply, lowrank_invhess

and two small handle classes (:class:`Mesh`, :class:`Bfgs`) carry them as
methods.  Every step of the computation runs in the CUDA library; this module
only marshals arguments.  Arrays may be torch tensors (CUDA or host) or numpy
arrays; outputs are written in place.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (ABI_SYMBOLS, GbfwiError, MeshDesc, Schedule, Source, UnetDesc, check, lib, ptr,
                   stream_of)

__all__ = [
    "Mesh", "Bfgs", "GbfwiError", "ABI_SYMBOLS", "mesh_create", "set_model", "forward", "misfit",
    "adjoint_gradient", "precond_diag", "bfgs_create", "bfgs_update", "bfgs_apply",
    "lowrank_invhess", "num_tiles", "tile_shape", "lib", "launch_count", "Unet", "resample",
]

F32, F64, I32 = np.float32, np.float64, np.int32


def launch_count() -> int:
    """Kernel launches issued through the library by this process."""
    return lib().gbfwi_launch_count()


def num_tiles() -> int:
    return lib().gbfwi_num_tiles()


def tile_shape(tile: int):
    tx, tz = ctypes.c_int(), ctypes.c_int()
    check(lib().gbfwi_tile_shape(tile, ctypes.byref(tx), ctypes.byref(tz)), "tile_shape")
    return tx.value, tz.value


class Mesh:
    """Handle of a structured spectral-element mesh with its sources and
    receivers (gbfwi_mesh)."""

    def __init__(self, nex, nez, h, dt, nt, sources, rec_xz, free_surface_top=1):
        d = MeshDesc(int(nex), int(nez), float(h), 5, int(free_surface_top), float(dt), int(nt), 0)
        srcs = (Source * max(1, len(sources)))()
        for i, s in enumerate(sources):
            srcs[i] = Source(float(s["x"]), float(s["z"]), int(s.get("type", 0)), float(s["f0"]),
                             float(s.get("t0", 1.2 / s["f0"])), float(s.get("amp", 1.0)))
        rec = np.ascontiguousarray(np.asarray(rec_xz, dtype=np.float64).reshape(-1, 2))
        h_ = ctypes.c_void_p()
        check(lib().gbfwi_mesh_create(ctypes.byref(d), srcs, len(sources),
                                      ctypes.c_void_p(rec.ctypes.data), len(rec), ctypes.byref(h_)),
              "mesh_create")
        self._h = h_
        self.nex, self.nez, self.h, self.dt, self.nt = int(nex), int(nez), float(h), float(dt), int(nt)
        self.nsrc, self.nrec = len(sources), len(rec)
        nx, nz = ctypes.c_int(), ctypes.c_int()
        check(lib().gbfwi_mesh_dims(self._h, ctypes.byref(nx), ctypes.byref(nz)), "mesh_dims")
        self.nx, self.nz = nx.value, nz.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                lib().gbfwi_mesh_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def nglob(self) -> int:
        return self.nx * self.nz

    def node_coords(self):
        x = np.zeros(self.nglob)
        z = np.zeros(self.nglob)
        check(lib().gbfwi_node_coords(self._h, ptr(x, F64), ptr(z, F64)), "node_coords")
        return x.reshape(self.nz, self.nx), z.reshape(self.nz, self.nx)

    @property
    def schedule(self) -> dict:
        s = Schedule()
        check(lib().gbfwi_get_schedule(self._h, ctypes.byref(s)), "get_schedule")
        return dict(shots_per_launch=s.shots_per_launch, tile=s.tile, use_graph=s.use_graph,
                    ckpt_every=s.ckpt_every, streams=s.streams)

    def set_schedule(self, shots_per_launch=1, tile=0, use_graph=0, ckpt_every=0, streams=1):
        s = Schedule(int(shots_per_launch), int(tile), int(use_graph), int(ckpt_every), int(streams))
        check(lib().gbfwi_set_schedule(self._h, ctypes.byref(s)), "set_schedule")

    def enable_timing(self, on=True):
        check(lib().gbfwi_enable_timing(self._h, int(bool(on))), "enable_timing")

    def last_phase_times(self) -> dict:
        f, a = ctypes.c_double(), ctypes.c_double()
        nf, na = ctypes.c_longlong(), ctypes.c_longlong()
        check(lib().gbfwi_last_phase_times(self._h, ctypes.byref(f), ctypes.byref(a), ctypes.byref(nf),
                                           ctypes.byref(na)), "last_phase_times")
        return dict(fwd_ms=f.value, adj_ms=a.value, fwd_launches=nf.value, adj_launches=na.value)

    def set_model(self, rho, vp, vs):
        check(lib().gbfwi_set_model(self._h, ptr(rho, F32), ptr(vp, F32), ptr(vs, F32),
                                    stream_of(rho, vp, vs)), "set_model")

    def forward(self, shot_ids, seis):
        ids = np.ascontiguousarray(np.asarray(shot_ids, dtype=np.int32))
        check(lib().gbfwi_forward(self._h, ptr(ids, I32), len(ids), ptr(seis, F32), stream_of(seis)),
              "forward")
        return seis

    def misfit(self, shot_ids, d_obs) -> float:
        ids = np.ascontiguousarray(np.asarray(shot_ids, dtype=np.int32))
        mis = ctypes.c_double()
        check(lib().gbfwi_misfit(self._h, ptr(ids, I32), len(ids), ptr(d_obs, F32), ctypes.byref(mis),
                                 stream_of(d_obs)), "misfit")
        return mis.value

    def adjoint_gradient(self, shot_ids, d_obs, grad, ckpt_every=-1) -> float:
        ids = np.ascontiguousarray(np.asarray(shot_ids, dtype=np.int32))
        mis = ctypes.c_double()
        check(lib().gbfwi_adjoint_gradient(self._h, ptr(ids, I32), len(ids), ptr(d_obs, F32),
                                           ctypes.byref(mis), ptr(grad, F32), int(ckpt_every),
                                           stream_of(d_obs, grad)), "adjoint_gradient")
        return mis.value

    def precond_diag(self, shot_ids, kind, sigma, damp, H, B0):
        ids = np.ascontiguousarray(np.asarray(shot_ids, dtype=np.int32))
        check(lib().gbfwi_precond_diag(self._h, ptr(ids, I32), len(ids), int(kind), float(sigma),
                                       float(damp), ptr(H, F32), ptr(B0, F32), stream_of(H, B0)),
              "precond_diag")

    def precond_from_hessian(self, H, sigma, damp, B0):
        """B0 = 1 / (S(H) + damp median S(H)) from a given raw map H [3][nz][nx]."""
        check(lib().gbfwi_precond_from_hessian(self._h, ptr(H, F32), float(sigma), float(damp), ptr(B0, F32),
                                               stream_of(H, B0)), "precond_from_hessian")
        return B0

    def unet_features(self, rho, vp, vs, sigma, out):
        """The five U-Net input channels [5][H][W] for this model and acquisition."""
        check(lib().gbfwi_unet_features(self._h, ptr(rho, F32), ptr(vp, F32), ptr(vs, F32), float(sigma),
                                        int(out.shape[1]), int(out.shape[2]), ptr(out, F32),
                                        stream_of(rho, vp, vs, out)), "unet_features")
        return out


class Bfgs:
    """Handle of a full-history BFGS store (gbfwi_bfgs)."""

    def __init__(self, n, kmax, B0):
        h_ = ctypes.c_void_p()
        check(lib().gbfwi_bfgs_create(int(n), int(kmax), ptr(B0, F32), ctypes.byref(h_)), "bfgs_create")
        self._h = h_
        self.n, self.kmax = int(n), int(kmax)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                lib().gbfwi_bfgs_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def count(self) -> int:
        return check(lib().gbfwi_bfgs_count(self._h), "bfgs_count")

    def update(self, s, y):
        check(lib().gbfwi_bfgs_update(self._h, ptr(s, F32), ptr(y, F32), stream_of(s, y)), "bfgs_update")

    def apply(self, X, Z, gamma=1.0, minus_B0=False):
        p = X.shape[0] if X.ndim == 2 else 1
        check(lib().gbfwi_bfgs_apply(self._h, ptr(X, F32), p, ptr(Z, F32), float(gamma), int(bool(minus_B0)),
                                     stream_of(X, Z)), "bfgs_apply")
        return Z

    def lowrank_invhess(self, p, rank, seed=0, eps_prior=1.0, X=None, V=None, lam=None, std=None):
        check(lib().gbfwi_lowrank_invhess(self._h, ptr(X, F32), int(p), int(rank), int(seed),
                                          float(eps_prior), ptr(V, F32), ptr(lam, F64), ptr(std, F32),
                                          stream_of(X, V, lam, std)), "lowrank_invhess")

    def lowrank_twopass(self, p, rank, seed=0, eps_prior=1.0, X=None, V=None, lam=None, std=None):
        """Algorithm 3 with the Rayleigh-Ritz second pass C = Q (B - B0) Q^T."""
        check(lib().gbfwi_lowrank_twopass(self._h, ptr(X, F32), int(p), int(rank), int(seed),
                                          float(eps_prior), ptr(V, F32), ptr(lam, F64), ptr(std, F32),
                                          stream_of(X, V, lam, std)), "lowrank_twopass")

    def lowrank_exact(self, rank, eps_prior=1.0, V=None, lam=None, std=None):
        """Exact eigenpairs of B_{n+1} - B0 (rank <= 2k) from a QR of [S, B0 Y]."""
        check(lib().gbfwi_lowrank_exact(self._h, int(rank), float(eps_prior), ptr(V, F32), ptr(lam, F64),
                                        ptr(std, F32), stream_of(V, lam, std)), "lowrank_exact")


# function-style names of the C ABI
def mesh_create(*a, **k) -> Mesh:
    return Mesh(*a, **k)


def set_model(mesh: Mesh, rho, vp, vs):
    return mesh.set_model(rho, vp, vs)


def forward(mesh: Mesh, shot_ids, seis):
    return mesh.forward(shot_ids, seis)


def misfit(mesh: Mesh, shot_ids, d_obs) -> float:
    return mesh.misfit(shot_ids, d_obs)


def adjoint_gradient(mesh: Mesh, shot_ids, d_obs, grad, ckpt_every=-1):
    return mesh.adjoint_gradient(shot_ids, d_obs, grad, ckpt_every)


def precond_diag(mesh: Mesh, shot_ids, kind, sigma, damp, H, B0):
    return mesh.precond_diag(shot_ids, kind, sigma, damp, H, B0)


def bfgs_create(n, kmax, B0) -> Bfgs:
    return Bfgs(n, kmax, B0)


def bfgs_update(b: Bfgs, s, y):
    return b.update(s, y)


def bfgs_apply(b: Bfgs, X, Z, gamma=1.0, minus_B0=False):
    return b.apply(X, Z, gamma, minus_B0)


def lowrank_invhess(b: Bfgs, p, rank, seed=0, eps_prior=1.0, X=None, V=None, lam=None, std=None):
    return b.lowrank_invhess(p, rank, seed, eps_prior, X, V, lam, std)


class Unet:
    """Handle of the learned-preconditioner U-Net (gbfwi_unet): BF16
    weights and activations, FP32 sums, tensor-core convolutions."""

    def __init__(self, levels=4, base=32, cin=5, cout=3, height=256, width=1024):
        d = UnetDesc(int(levels), int(base), int(cin), int(cout), int(height), int(width))
        h_ = ctypes.c_void_p()
        check(lib().gbfwi_unet_create(ctypes.byref(d), ctypes.byref(h_)), "unet_create")
        self._h = h_
        self.levels, self.base, self.cin, self.cout = int(levels), int(base), int(cin), int(cout)
        self.height, self.width = int(height), int(width)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                lib().gbfwi_unet_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def num_params(self) -> int:
        return check(lib().gbfwi_unet_num_params(self._h), "unet_num_params")

    def layers(self):
        """[(cout, cin, k, cout_pad, kc_pad, w_offset, b_offset)] in parameter order."""
        n = check(lib().gbfwi_unet_layer_info(self._h, -1, None), "unet_layer_info")
        out = []
        for i in range(n):
            info = np.zeros(7, I32)
            check(lib().gbfwi_unet_layer_info(self._h, i, ptr(info, I32)), "unet_layer_info")
            out.append(tuple(int(v) for v in info))
        return out

    def set_params(self, params):
        check(lib().gbfwi_unet_set_params(self._h, ptr(params, F32), stream_of(params)), "unet_set_params")

    def get_params(self, params):
        check(lib().gbfwi_unet_get_params(self._h, ptr(params, F32), stream_of(params)), "unet_get_params")
        return params

    def forward(self, x, y):
        check(lib().gbfwi_unet_forward(self._h, ptr(x, F32), ptr(y, F32), stream_of(x, y)), "unet_forward")
        return y

    def gradient(self, x, dy, grad):
        check(lib().gbfwi_unet_gradient(self._h, ptr(x, F32), ptr(dy, F32), ptr(grad, F32),
                                        stream_of(x, dy, grad)), "unet_gradient")
        return grad

    def train_step(self, x, target, lr) -> float:
        batch = x.shape[0] if x.ndim == 4 else 1
        loss = ctypes.c_double()
        check(lib().gbfwi_unet_train_step(self._h, ptr(x, F32), ptr(target, F32), int(batch), float(lr),
                                          ctypes.byref(loss), stream_of(x, target)), "unet_train_step")
        return loss.value


def resample(src, dst, op=0):
    """Bilinear resampling of device arrays [C][sh][sw] -> [C][dh][dw]
    (corners aligned); op 1: of log(src), op 2: exp of the result."""
    C, sh, sw = src.shape
    _, dh, dw = dst.shape
    check(lib().gbfwi_resample(ptr(src, F32), int(C), int(sh), int(sw), ptr(dst, F32), int(dh), int(dw), int(op),
                               stream_of(src, dst)), "resample")
    return dst
