"""Convergence and uncertainty experiment of the paper, in kind, on seeded
synthetic models (Section 3: BFGS vs L-BFGS(5), preconditioners P1-P4,
RSVD uncertainty maps compared with the true model error).

    python -m paper_2009_12663_gb300.experiments [--iterations 15] [--workload small|marmousi340x70]
                                                 [--variants BFGS+P4] [--probes 60] [--rank 50] [--out result.json]
    python -m paper_2009_12663_gb300.experiments --learned [--train-pairs 48] [--train-steps 2000]
                                                 [--lr-decay 0.999] [--out result.json]

Prints one JSON document: per variant the relative data misfit and the
relative model misfit (vp, vs) per iteration, iterations to halve the misfit,
wall time; for the P4 run the leading eigenvalues of the retrieved
B_{n+1} - B0, the posterior std of vp / vs and its correlation with the
absolute error of the inverted model, and the data misfit along
perturbations shaped by the std maps (Appendix C) next to random ones.
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
from .fwi import Problem, clamp_model, fwi, model_misfit, preconditioner  # noqa: E402

__all__ = ["build", "run", "learned_comparison", "misfit_scan"]


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


WORKLOADS = {
    "small": dict(nex=80, nez=20, h=50.0, nshot=8, f0=8.0, nt=3000, seed=11, smooth=250.0),
    # the benchmark's Marmousi-shaped workload: 340 x 70 elements of 50 m,
    # 24 explosive 5 Hz sources, 341 receivers, dt 0.5 ms, 12000 steps,
    # starting model the truth blurred by a 500 m Gaussian
    "marmousi340x70": dict(nex=340, nez=70, h=50.0, nshot=24, f0=5.0, nt=12000, seed=2024, smooth=500.0),
}


def run(iterations=15, sigma=100.0, rank=None, workload="small", variants=None, probes=None):
    """Section 3 in kind: BFGS, L-BFGS(5) and BFGS with P1-P4, data and
    model misfit per iteration (Figs. 3 and 5), then for the P4 run the
    low-rank uncertainty (Section 2.3: single-pass with p = k probes as the
    paper, the two-pass variant, and the exact decomposition whose rank is
    at most 2k), the std maps against the true model error, and the
    Appendix C misfit scan."""
    w = WORKLOADS[workload]
    mesh, ids, d_obs, true, start = build(**w)
    prob = Problem(mesh, ids, d_obs, invert=(False, True, True))
    mask = prob.mask
    one = torch.tensor([True])
    allv = [("BFGS", None, None), ("L-BFGS(5)", None, 5)] + [(f"BFGS+P{k}", k, None) for k in (1, 2, 3, 4)]
    variants = [v for v in allv if variants is None or v[0] in variants]
    if not any(v[0] == "BFGS+P4" for v in variants):
        raise ValueError("the uncertainty step needs the BFGS+P4 run")
    out = {"model": f"marmousi-shaped {w['nex']}x{w['nez']} elements of {w['h']:g} m, {w['nshot']} shots "
                    f"({w['f0']:g} Hz), {mesh.nrec} receivers, {w['nt']} steps, start = truth blurred by "
                    f"{w['smooth']:g} m",
           "inverted": "vp, vs (rho fixed)", "preconditioner_smoothing_sigma_m": sigma, "variants": {}}
    keep = {}
    for name, kind, memory in variants:
        B0 = preconditioner(mesh, ids, start, kind, sigma) if kind else None
        prob.evaluations = {"misfit": 0, "gradient": 0}
        mm = {"vp": [1.0], "vs": [1.0]}

        def cb(it, mk, h):
            mm["vp"].append(model_misfit(mk[1:2], true[1:2], start[1:2], one))
            mm["vs"].append(model_misfit(mk[2:3], true[2:3], start[2:3], one))

        t0 = time.perf_counter()
        m_inv, hist, store = fwi(prob, start, iterations, B0=B0, memory=memory, callback=cb)
        wall = time.perf_counter() - t0
        rel = [h["rel_misfit"] for h in hist]
        half = next((h["iteration"] for h in hist if h["rel_misfit"] <= 0.5), None)
        out["variants"][name] = {
            "rel_misfit": rel, "iterations_to_half_misfit": half,
            "model_misfit_vp": mm["vp"], "model_misfit_vs": mm["vs"],
            "evaluations": dict(prob.evaluations), "wall_s": wall}
        keep[name] = (m_inv, store)
    # uncertainty of the P4 run (Section 2.3): p = rank = stored pairs (paper), capped at 2k
    m_inv, store = keep["BFGS+P4"]
    k = store.count
    p = max(2, min(2 * k, k if rank is None else rank)) if probes is None else int(probes)
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
    # the spectrum three ways: exact (rank <= 2k), single pass and two pass
    # with the paper's p = k probes
    spectra = {}
    lam2 = torch.zeros(r, dtype=torch.float64, device=true.device)
    store.lowrank_twopass(p, r, seed=2020, eps_prior=1.0, lam=lam2)
    spectra["two_pass_p_k"] = lam2.cpu().numpy().tolist()
    le = torch.zeros(2 * k, dtype=torch.float64, device=true.device)
    Ve = torch.zeros(2 * k, n, device=true.device)
    store.lowrank_exact(2 * k, eps_prior=1.0, V=Ve, lam=le)
    spectra["exact_rank_2k"] = le.cpu().numpy().tolist()
    # resolved directions only: the rows beyond the basis rank are returned as zero
    nres = int((le != 0).sum())
    Vh = Ve[:nres].double()
    spectra["exact_resolved_directions"] = nres
    spectra["exact_V_orthonormality_max_error"] = float((Vh @ Vh.T - torch.eye(nres, device=Vh.device,
                                                                              dtype=Vh.dtype)).abs().max())
    out["uq_P4"] = {"pairs": k, "probes": p, "rank": r, "eigenvalues": lam.cpu().numpy().tolist(),
                    "spectra": spectra,
                    "std_mean_vp": float(stdm[0].mean()), "std_mean_vs": float(stdm[1].mean()),
                    "corr_std_vs_abs_error": {"vp": corr[0], "vs": corr[1]}}
    out["uq_misfit_scan"] = misfit_scan(prob, m_inv, torch.tensor(stdm, device=true.device), mask)
    return out


def misfit_scan(prob, m_inv, std_maps, mask, vmax=250.0, alphas=(-2, -1.5, -1, -0.5, 0, 0.5, 1, 1.5, 2), seed=5):
    """Appendix C in kind: the data misfit along m_inv + alpha m_pert, with
    m_pert the posterior std map of each inverted parameter scaled to a
    maximum of vmax m/s, next to a smooth random perturbation of the same
    maximum (Gaussian bumps).  Misfits relative to the one at m_inv."""
    mk = mask.to(m_inv.device)
    pert = torch.zeros_like(m_inv)
    pert[mk] = std_maps / std_maps.amax(dim=(1, 2), keepdim=True) * vmax
    nz, nx = m_inv.shape[1:]
    rng = np.random.default_rng(seed)
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    rnd = torch.zeros_like(m_inv)
    for c in np.nonzero(mask.numpy())[0]:
        f = np.zeros((nz, nx))
        for _ in range(12):
            cz, cx, w = rng.uniform(0, nz), rng.uniform(0, nx), rng.uniform(6, 20)
            f += rng.standard_normal() * np.exp(-((zz - cz) ** 2 + (xx - cx) ** 2) / (2 * w * w))
        rnd[c] = torch.tensor(f / np.abs(f).max() * vmax, dtype=m_inv.dtype, device=m_inv.device)
    f0 = prob.misfit(clamp_model(m_inv))
    scan = {"alpha": list(alphas), "std_pert": [], "random_pert": []}
    for a in alphas:
        scan["std_pert"].append(prob.misfit(clamp_model(m_inv + a * pert)) / f0)
        scan["random_pert"].append(prob.misfit(clamp_model(m_inv + a * rnd)) / f0)
    scan["vmax_m_per_s"] = vmax
    return scan


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iterations", type=int, default=15)
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="small",
                    help="small: 80x20 elements, 8 shots; marmousi340x70: the benchmark's workload")
    ap.add_argument("--variants", default=None,
                    help="comma-separated subset of BFGS, L-BFGS(5), BFGS+P1..BFGS+P4 (default: all)")
    ap.add_argument("--probes", type=int, default=None, help="probes p of the uncertainty step (default k)")
    ap.add_argument("--rank", type=int, default=None, help="rank of the uncertainty step (default k)")
    ap.add_argument("--learned", action="store_true", help="run the learned-preconditioner comparison")
    ap.add_argument("--train-pairs", type=int, default=48, help="training pairs of the learned comparison")
    ap.add_argument("--train-steps", type=int, default=2000, help="Adam steps of the learned comparison")
    ap.add_argument("--lr-decay", type=float, default=0.999, help="learning-rate factor per Adam step")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    if a.learned:
        res = learned_comparison(n_train=a.train_pairs, steps=a.train_steps, lr_decay=a.lr_decay)
    else:
        res = run(a.iterations, workload=a.workload, rank=a.rank, probes=a.probes,
                  variants=None if a.variants is None else a.variants.split(","))
    txt = json.dumps(res)
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(json.dumps(res, indent=1))



def learned_comparison(n_train=48, n_test=4, nt=3000, img=(256, 1024), steps=2000, iterations=8, seed0=1000,
                       device="cuda", lr_decay=0.999):
    """The learned preconditioner in kind of its intended use, on the
    340 x 70 element Marmousi-shaped mesh (24 shots, 5 Hz, `nt` steps):
    train the U-Net on P4 maps the method computes for seeded models, then
    on a held-out model compare
      plain:   one shot per launch, no graphs, P4 computed by the method;
      fast:    four graph-replayed single-shot lanes, P4 predicted by the U-Net
    by wall time to reach the misfit reduction the plain form reaches in
    `iterations` BFGS iterations, and by the posterior std of the run."""
    from . import Unet
    from . import learned as L

    wl = synth.marmousi_like_workload(nt=nt, nshot=24)
    srcs = wl.sources(amp=1e12)
    m = Mesh(wl.nex, wl.nez, wl.h, wl.dt, nt, srcs, wl.rec_xz)
    x, z = m.node_coords()
    W, H = wl.nex * wl.h, wl.nez * wl.h
    ids = list(range(wl.nshot))
    m.set_schedule(shots_per_launch=1, tile=0, use_graph=1, streams=4)

    def model(s):
        return torch.tensor(np.stack(synth.marmousi_like(x, z, s, W, H)), dtype=torch.float32, device=device)

    t0 = time.perf_counter()
    models = [model(seed0 + i) for i in range(n_train + n_test)]
    X, T = L.make_pairs(m, models, ids, *img)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    net = Unet(levels=4, base=32, cin=5, cout=3, height=img[0], width=img[1])
    lp = L.LearnedPreconditioner(net, seed=1)
    t_train = lp.fit(X[:n_train], T[:n_train], steps=steps, lr=1e-3, batch=4, seed=2, lr_decay=lr_decay)
    errs = []
    for i in range(n_train, n_train + n_test):
        Hc = L.computed_map(m, models[i], ids)
        errs.append(L.rel_log_error(lp.predict_map(m, models[i]), Hc))
    out = {"workload": f"340x70 Marmousi-shaped mesh, 24 shots x {nt} steps; U-Net 4 x 32 on {img[0]}x{img[1]}",
           "train_pairs": n_train, "test_models": n_test, "pair_generation_s": t_pairs, "train_steps": steps,
           "train_s": t_train, "loss_first_last": [lp.history[0], lp.history[-1]],
           "heldout_rel_log_error": errs}

    # inversion of a held-out truth from its smoothed start
    truth = models[n_train]
    start = torch.tensor(np.stack(synth.marmousi_like_smooth(x, z, seed0 + n_train, W, H)),
                         dtype=torch.float32, device=device)
    d_obs = torch.zeros(wl.nshot, wl.nrec, 2, nt, device=device)
    m.set_model(*truth)
    m.forward(ids, d_obs)
    prob = Problem(m, ids, d_obs, invert=(False, True, True))

    def run(schedule, b0_fn, target=None):
        m.set_schedule(**schedule)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B0, info = b0_fn()
        torch.cuda.synchronize()
        t_b0 = time.perf_counter() - t0
        trace = []
        cb = lambda it, mk, h: trace.append((h["rel_misfit"], time.perf_counter() - t0))
        mi, hist, store = fwi(prob, start, iterations, B0=B0, callback=cb)
        reach = None
        if target is not None:
            reach = next((t for r, t in trace if r <= target), None)
        k = store.count
        std = torch.zeros(store.n, device=device)
        store.lowrank_invhess(k, k, seed=2020, eps_prior=1.0, std=std)
        return {"b0_s": t_b0, "b0_info": info, "rel_misfit": [h["rel_misfit"] for h in hist],
                "trace_s": [t for _, t in trace], "time_to_target_s": reach}, std

    plain_sched = dict(shots_per_launch=1, tile=0, use_graph=0, ckpt_every=0, streams=1)
    fast_sched = dict(shots_per_launch=1, tile=0, use_graph=1, ckpt_every=0, streams=4)

    def computed():
        return preconditioner(m, ids, start, 4, 100.0), {"source": "computed P4"}

    def predicted():
        B0, info = lp.b0(m, start, 100.0, 1.0)
        info["source"] = "U-Net"
        return B0, info

    plain, std_p = run(plain_sched, computed)
    target = plain["rel_misfit"][-1]
    plain["time_to_target_s"] = plain["trace_s"][-1]
    fast, std_f = run(fast_sched, predicted, target)
    fast_computed, std_fc = run(fast_sched, computed, target)
    out["target_rel_misfit"] = target
    out["plain_single_shot_computed_P4"] = plain
    out["fast_lanes_graphs_learned_P4"] = fast
    out["fast_lanes_graphs_computed_P4"] = fast_computed
    out["posterior_std_rel_diff_learned_vs_computed"] = float((std_f - std_p).norm() / std_p.norm())
    out["posterior_std_rel_diff_fast_vs_plain_computed"] = float((std_fc - std_p).norm() / std_p.norm())
    return out


if __name__ == "__main__":
    main()
