"""Write the FP64 oracle's values for one full-length shot of the
Marmousi-shaped 340 x 70 element workload (17 km x 3.5 km, 382,441 GLL
points, 5 Hz explosive source at 20 m depth, 341 surface receivers,
dt = 0.5 ms, all 12000 steps) to marmousi_shot11_full.npz.

It calls only oracle/ (and synth/ for the seeded model and acquisition):

* the records of the true model and of the starting model (the 500 m
  Gaussian smoothing of the truth), kept at every 20th receiver and every
  10th time sample;
* the misfit f(m0) of Eq. A1 against the true model's records;
* central differences (f(m0 + eps dm) - f(m0 - eps dm)) / (2 eps) along three
  smooth directions dm, one per parameter (rho, vp, vs): a Gaussian bump of
  400 m standard deviation under the source at 800 m depth, scaled by the
  parameter.  The gradient of the discrete misfit projected on dm must equal
  these (its exactness is pinned by the oracle's finite-difference test).

The models are rounded to FP32 first, so that the GPU and the oracle start
from the same numbers.  The FP64 history of a full-length shot (73 GB) does
not fit in memory, so the gradient is sampled through these projections
instead of element by element.  The eight forward simulations run in
parallel processes (about ten minutes on eight cores).

    python tests/golden/make_marmousi_full_length.py
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "marmousi_shot11_full.npz")
SHOT = 11
SEED = 2024
EPS = 2.5e-4
SIGMA = 400.0
DEPTH = 800.0
REC_STRIDE = 20
T_STRIDE = 10


def models():
    """(true, start) FP32-rounded models on the oracle's node grid, the
    workload and the oracle set-up."""
    import synth
    from oracle import sem
    wl = synth.marmousi_like_workload()
    st = sem.Setup(sem.Mesh(wl.nex, wl.nez, wl.h), wl.dt, wl.nt, wl.rec_xz)
    x, z = st.mesh.coords()
    W, H = wl.nex * wl.h, wl.nez * wl.h
    r32 = lambda t: tuple(np.asarray(a, np.float32).astype(np.float64) for a in t)
    return wl, st, r32(synth.marmousi_like(x, z, SEED, W, H)), r32(synth.marmousi_like_smooth(x, z, SEED, W, H))


def direction(x, z, xs, c, start):
    """Bump of parameter c (0 rho, 1 vp, 2 vs) scaled by the parameter."""
    g = np.exp(-((x - xs) ** 2 + (z - DEPTH) ** 2) / (2.0 * SIGMA ** 2))
    dm = np.zeros((3,) + x.shape)
    dm[c] = np.asarray(start[c], np.float64) * g
    return dm


def _run(job):
    wl, st, true, start = models()
    src = wl.sources(amp=1e12)[SHOT]
    fvec, stf = st.source(src)
    kind, c, sign = job
    if kind == "true":
        model = true
    elif kind == "start":
        model = start
    else:
        x, z = st.mesh.coords()
        dm = direction(x, z, src["x"], c, start)
        model = tuple(np.asarray(start[q], np.float64) + sign * EPS * dm[q] for q in range(3))
    return job, st.forward(model, fvec, stf)


def main():
    from oracle import sem
    jobs = [("true", -1, 0), ("start", -1, 0)] + [("dir", c, s) for c in range(3) for s in (1, -1)]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = dict(pool.map(_run, jobs))
    wl, st, _, _ = models()
    d_obs = res[("true", -1, 0)]
    f0 = sem.misfit(wl.dt, res[("start", -1, 0)], d_obs)
    fp = np.array([sem.misfit(wl.dt, res[("dir", c, 1)], d_obs) for c in range(3)])
    fm = np.array([sem.misfit(wl.dt, res[("dir", c, -1)], d_obs) for c in range(3)])
    ridx = np.arange(0, wl.nrec, REC_STRIDE)
    tidx = np.arange(T_STRIDE - 1, wl.nt, T_STRIDE)
    sub = lambda s: s[ridx][:, :, tidx].astype(np.float32)
    np.savez_compressed(
        OUT, shot=SHOT, seed=SEED, nt=wl.nt, eps=EPS, sigma=SIGMA, depth=DEPTH, rec_idx=ridx, t_idx=tidx,
        seis_true=sub(d_obs), seis_start=sub(res[("start", -1, 0)]), misfit=f0, f_plus=fp, f_minus=fm,
        dfd=(fp - fm) / (2 * EPS),
        norm_true=np.linalg.norm(d_obs), norm_start=np.linalg.norm(res[("start", -1, 0)]))
    print(OUT, f0, (fp - fm) / (2 * EPS))


if __name__ == "__main__":
    main()
