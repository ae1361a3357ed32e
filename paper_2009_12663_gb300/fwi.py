"""Preconditioned BFGS elastic FWI driver (Section 2.1, Algorithm 1) and the
post-convergence uncertainty step (Section 2.3).

Orchestration around the C ABI: misfits and gradients (gbfwi_misfit,
gbfwi_adjoint_gradient), the preconditioner B0 (gbfwi_precond_diag), the
search direction z = -gamma_k B_k g in compact form (gbfwi_bfgs_apply on the
full-history store, or on a store of the last `memory` pairs for L-BFGS), the
history (gbfwi_bfgs_update) and the low-rank inverse Hessian
(gbfwi_lowrank_invhess).  The line search (Armijo backtracking from the unit
quasi-Newton step; a scaled first step) and the model bookkeeping are small
vector operations done with torch; they are not part of the timed path.

Parameters are (rho, vp, vs) on the node grid; `invert` selects which of them
are unknowns (the paper's Marmousi runs keep rho fixed).  The first step (and
a restart) moves the model by step0 max|m| at the 99.9th percentile of the
direction's magnitude.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import torch

from . import Bfgs, GbfwiError, Mesh


@dataclass
class Problem:
    mesh: Mesh
    shot_ids: list
    d_obs: torch.Tensor
    invert: tuple = (False, True, True)
    evaluations: dict = field(default_factory=lambda: {"misfit": 0, "gradient": 0})

    @property
    def mask(self) -> torch.Tensor:
        return torch.tensor(self.invert, dtype=torch.bool)

    def _set(self, m):
        self.mesh.set_model(m[0].contiguous(), m[1].contiguous(), m[2].contiguous())

    def misfit(self, m) -> float:
        self._set(m)
        self.evaluations["misfit"] += 1
        return self.mesh.misfit(self.shot_ids, self.d_obs)

    def gradient(self, m):
        self._set(m)
        g = torch.zeros_like(m)
        f = self.mesh.adjoint_gradient(self.shot_ids, self.d_obs, g)
        self.evaluations["gradient"] += 1
        return f, g


def pack(t: torch.Tensor, mask: torch.Tensor) -> torch.Tensor:
    return t[mask.to(t.device)].reshape(-1).contiguous()


def unpack(v: torch.Tensor, mask: torch.Tensor, like: torch.Tensor) -> torch.Tensor:
    out = torch.zeros_like(like)
    out[mask.to(like.device)] = v.reshape(int(mask.sum()), *like.shape[1:])
    return out


def clamp_model(m: torch.Tensor, vp_bounds=(800.0, 8000.0)) -> torch.Tensor:
    """Keep the model physical: rho > 0, vp within bounds, 0 < vs < 0.7 vp."""
    rho = m[0].clamp(min=100.0)
    vp = m[1].clamp(*vp_bounds)
    vs = torch.minimum(m[2].clamp(min=50.0), 0.7 * vp)
    return torch.stack([rho, vp, vs]).contiguous()


def preconditioner(mesh: Mesh, shot_ids, m0: torch.Tensor, kind: int, sigma: float, damp: float = 1.0):
    """B0 of kind 1..4 (Eqs. 4-8) at the starting model, [3][nz][nx]."""
    mesh.set_model(m0[0].contiguous(), m0[1].contiguous(), m0[2].contiguous())
    H = torch.zeros_like(m0)
    B0 = torch.zeros_like(m0)
    mesh.precond_diag(shot_ids, kind, sigma, damp, H, B0)
    return B0


def robust_max(v: torch.Tensor, q: float = 0.999) -> float:
    """The q-quantile of |v| (on at most ~1M evenly spaced samples): the
    scale of a search direction without its few largest entries (a single
    spike of the preconditioner would otherwise set the first step)."""
    a = v.abs().reshape(-1)
    if a.numel() > 1_000_000:
        a = a[:: (a.numel() + 999_999) // 1_000_000]
    return float(torch.quantile(a.float(), q))


def fwi(problem: Problem, m0: torch.Tensor, iterations: int, B0=None, memory=None, step0=0.02,
        c1=1e-4, max_backtracks=8, callback=None, pairs_out=None):
    """Run (L-)BFGS.  Returns (model, history, store); `store` is the
    full-history BFGS store (None for L-BFGS) that lowrank_invhess probes.
    When `pairs_out` is a list, every stored pair (s, y) is appended to it."""
    mask = problem.mask
    m = clamp_model(m0.clone())
    n = int(mask.sum()) * m[0].numel()
    b0 = pack(B0, mask) if B0 is not None else torch.ones(n, device=m.device)
    store = Bfgs(n, iterations + 1, b0) if memory is None else None
    pairs = []
    f, g = problem.gradient(m)
    gv = pack(g, mask)
    f0 = f
    hist = [dict(iteration=0, misfit=f, rel_misfit=1.0, step=0.0, time=0.0)]
    t_start = time.perf_counter()
    for it in range(1, iterations + 1):
        if memory is not None:                         # L-BFGS: store of the last `memory` pairs
            store_l = Bfgs(n, max(1, memory), b0)
            for s_, y_ in pairs[-memory:]:
                store_l.update(s_, y_)
            cur = store_l
        else:
            cur = store
        k = cur.count
        if k == 0:
            p = -(b0 * gv)
            alpha = step0 * float(m[mask.to(m.device)].abs().max()) / robust_max(p)
        else:
            s_last, y_last = pairs[-1]
            # gamma_k of Algorithm 1 weighted by the preconditioner: the paper's
            # s^T y / y^T y when B0 = I; for a physically scaled B0 the
            # weighted form keeps gamma_k B0 y = s in the mean (unit steps)
            gamma = float((s_last * y_last).sum() / (y_last * b0 * y_last).sum())
            z = torch.zeros(1, n, device=m.device)
            cur.apply(gv[None].contiguous(), z, gamma=gamma, minus_B0=False)
            p = -z[0]
            alpha = 1.0
        gtp = float((gv * p).sum())
        if gtp >= 0:                                   # not a descent direction: restart
            p = -(b0 * gv)
            gtp = float((gv * p).sum())
            alpha = step0 * float(m[mask.to(m.device)].abs().max()) / robust_max(p)
        accepted = False
        for _ in range(max_backtracks):
            m_try = clamp_model(m + alpha * unpack(p, mask, m))
            f_try = problem.misfit(m_try)
            if f_try <= f + c1 * alpha * gtp:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            break
        f_new, g_new = problem.gradient(m_try)
        gv_new = pack(g_new, mask)
        s_vec = pack(m_try - m, mask)
        y_vec = gv_new - gv
        try:
            if store is not None:
                store.update(s_vec, y_vec)
            pairs.append((s_vec, y_vec))
            if pairs_out is not None:
                pairs_out.append((s_vec.clone(), y_vec.clone()))
        except GbfwiError as e:
            if e.name != "ECURV":
                raise
        m, f, gv = m_try, f_new, gv_new
        hist.append(dict(iteration=it, misfit=f, rel_misfit=f / f0, step=alpha,
                         time=time.perf_counter() - t_start))
        if callback:
            callback(it, m, hist[-1])
    return m, hist, store


def model_misfit(m, m_true, m0, mask) -> float:
    """|m - m_true| / |m0 - m_true| over the inverted parameters."""
    mk = mask.to(m.device)
    return float((m[mk] - m_true[mk]).norm() / (m0[mk] - m_true[mk]).norm())
