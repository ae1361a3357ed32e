"""Schedule autotuner for the time-step launches.

Times candidate schedules (element-tile shape, shots per launch, CUDA-graph
replay, checkpoint interval) on a short time axis of the same mesh and
acquisition, and returns the fastest one per shot-step.  Results are cached
per GPU model and mesh signature in a JSON file (default
~/.cache/gbfwi/autotune.json).  Every schedule gives bitwise-identical
results (the summation order does not depend on it), so the choice only
affects speed.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import Mesh, num_tiles

CACHE = os.environ.get("GBFWI_AUTOTUNE_CACHE", os.path.expanduser("~/.cache/gbfwi/autotune.json"))


def _signature(nex, nez, nshot, nrec, nt, spl_options, gpu_name):
    return f"{gpu_name}|{nex}x{nez}|shots{nshot}|rec{nrec}|nt{nt}|spl{','.join(map(str, spl_options))}"


def tune(nex, nez, h, dt, nt, sources, rec_xz, model, spl_options=(1, 4, 8, 24), tiles=None,
         probe_nt=120, graphs=(0, 1), ckpt_every=0, use_cache=True, device="cuda"):
    """Return (best schedule dict, timings list).  `model` = (rho, vp, vs)
    float32 CUDA tensors on the node grid."""
    import torch

    gpu = torch.cuda.get_device_name()
    sig = _signature(nex, nez, len(sources), len(rec_xz), nt, spl_options, gpu)
    if use_cache and os.path.exists(CACHE):
        try:
            db = json.load(open(CACHE))
            if sig in db:
                return db[sig]["best"], db[sig]["timings"]
        except Exception:
            pass
    tiles = range(num_tiles()) if tiles is None else tiles
    nshot = len(sources)
    m = Mesh(nex, nez, h, dt, probe_nt, sources, rec_xz)
    m.set_model(*model)
    ids = list(range(nshot))
    obs = torch.zeros(nshot, len(rec_xz), 2, probe_nt, device=model[0].device)
    grad = torch.zeros(3, m.nz, m.nx, device=model[0].device)
    timings = []
    for spl in spl_options:
        if spl > nshot:
            continue
        for tile in tiles:
            for g in graphs:
                sch = dict(shots_per_launch=spl, tile=tile, use_graph=g,
                           ckpt_every=(ckpt_every if spl > 1 else 0))
                m.set_schedule(**sch)
                m.adjoint_gradient(ids, obs, grad)          # warm-up / capture
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                m.adjoint_gradient(ids, obs, grad)
                torch.cuda.synchronize()
                dtm = time.perf_counter() - t0
                timings.append(dict(schedule=sch, us_per_shot_step=1e6 * dtm / (nshot * probe_nt)))
    best = min(timings, key=lambda r: r["us_per_shot_step"])["schedule"]
    if use_cache:
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            db = json.load(open(CACHE)) if os.path.exists(CACHE) else {}
            db[sig] = {"best": best, "timings": timings}
            json.dump(db, open(CACHE, "w"), indent=1)
        except Exception:
            pass
    return best, timings
