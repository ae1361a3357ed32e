"""Convergence and uncertainty experiment of the paper, in kind, on seeded
synthetic models (Section 3: BFGS vs L-BFGS(5), preconditioners P1-P4,
RSVD uncertainty maps compared with the true model error).

    python -m paper_2009_12663_gb300.experiments [--iterations 15] [--out result.json]

Prints one JSON document: per variant the relative data misfit and the
relative model misfit (vp, vs) per iteration, iterations to halve the misfit,
wall time; for the P4 run the leading eigenvalues of the retrieved
B_{n+1} - B0, the posterior std of vp / vs and its correlation with the
absolute error of the inverted model.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

from . import Mesh  # noqa: E402
from .fwi import Problem, fwi, model_misfit, preconditioner  # noqa: E402


def build(nex=80, nez=20, h=50.0, nshot=8, f0=8.0, nt=3000, seed=11, smooth=250.0, device="cuda"):
    wl = synth.marmousi_like_workload(nt=nt, nshot=nshot, nex=nex, nez=nez, h=h)
    srcs = [dict(s, f0=f0, t0=1.2 / f0) for s in wl.sources(amp=1e12)]
    m = Mesh(wl.nex, wl.nez, wl.h, wl.dt, nt, srcs, wl.rec_xz)
    m.set_schedule(shots_per_launch=1, tile=0, use_graph=1, streams=4)
    x, z = m.node_coords()
    W, H = nex * h, nez * h
    true = torch.tensor(np.stack(synth.marmousi_like(x, z, seed, W, H)), dtype=torch.float32, device=device)
    start = torch.tensor(np.stack(synth.marmousi_like_smooth(x, z, seed, W, H, sigma=smooth)),
                         dtype=torch.float32, device=device)
    ids = list(range(nshot))
    d_obs = torch.zeros(nshot, wl.nrec, 2, nt, device=device)
    m.set_model(*true)
    m.forward(ids, d_obs)
    return m, ids, d_obs, true.contiguous(), start.contiguous()


def run(iterations=15, sigma=100.0, rank=None):
    mesh, ids, d_obs, true, start = build()
    prob = Problem(mesh, ids, d_obs, invert=(False, True, True))
    mask = prob.mask
    variants = [("BFGS", None, None), ("L-BFGS(5)", None, 5)] + [(f"BFGS+P{k}", k, None) for k in (1, 2, 3, 4)]
    out = {"model": "marmousi-shaped 80x20 elements of 50 m, 8 shots (8 Hz), 81 receivers, 3000 steps",
           "inverted": "vp, vs (rho fixed)", "variants": {}}
    keep = {}
    for name, kind, memory in variants:
        B0 = preconditioner(mesh, ids, start, kind, sigma) if kind else None
        prob.evaluations = {"misfit": 0, "gradient": 0}
        t0 = time.perf_counter()
        m_inv, hist, store = fwi(prob, start, iterations, B0=B0, memory=memory)
        wall = time.perf_counter() - t0
        rel = [h["rel_misfit"] for h in hist]
        half = next((h["iteration"] for h in hist if h["rel_misfit"] <= 0.5), None)
        out["variants"][name] = {
            "rel_misfit": rel, "iterations_to_half_misfit": half,
            "model_misfit_vp": model_misfit(m_inv[1:2], true[1:2], start[1:2], torch.tensor([True])),
            "model_misfit_vs": model_misfit(m_inv[2:3], true[2:3], start[2:3], torch.tensor([True])),
            "evaluations": dict(prob.evaluations), "wall_s": wall}
        keep[name] = (m_inv, store)
    # uncertainty of the P4 run (Section 2.3): p = rank = stored pairs (paper), capped at 2k
    m_inv, store = keep["BFGS+P4"]
    k = store.count
    p = max(2, min(2 * k, k if rank is None else rank))
    r = min(p, k if rank is None else rank)
    n = store.n
    V = torch.zeros(r, n, device=true.device)
    lam = torch.zeros(r, dtype=torch.float64, device=true.device)
    std = torch.zeros(n, device=true.device)
    store.lowrank_invhess(p, r, seed=2020, eps_prior=1.0, V=V, lam=lam, std=std)
    nz, nx = true.shape[1:]
    stdm = std.reshape(int(mask.sum()), nz, nx).cpu().numpy()
    err = (m_inv - true).abs()[mask.to(true.device)].cpu().numpy()
    corr = [float(np.corrcoef(stdm[c].ravel(), err[c].ravel())[0, 1]) for c in range(stdm.shape[0])]
    out["uq_P4"] = {"pairs": k, "probes": p, "rank": r, "eigenvalues": lam.cpu().numpy().tolist(),
                    "std_mean_vp": float(stdm[0].mean()), "std_mean_vs": float(stdm[1].mean()),
                    "corr_std_vs_abs_error": {"vp": corr[0], "vs": corr[1]}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iterations", type=int, default=15)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(a.iterations)
    txt = json.dumps(res)
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
