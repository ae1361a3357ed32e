"""Schedule autotuner for the time-step launches of gbfwi_adjoint_gradient.

The search space is the whole launch schedule: element-tile shape, shots per
launch (shot-indexed batching), concurrent launch streams (lanes), CUDA-graph
replay and the checkpoint interval.  Every schedule gives bitwise-identical
misfits and gradients (the summation order does not depend on it), so the
choice only affects speed and device memory.

Each candidate is timed on a short time axis of the same mesh and
acquisition with CUDA events on the launching stream (median of `repeats`
timed calls after one untimed call that also captures the graphs).  A
checkpoint interval C of the full time axis is probed as the interval with
the same number of segments on the short axis, so the probe pays the same
recomputation.  Candidates whose device memory on the full time axis
(histories, snapshots, per-shot accumulators) exceeds the budget are
skipped.  The search is staged (tile at the default lane schedule, then
lanes x shots per launch x checkpoint interval, then graphs off) to keep it
to a few dozen probes.  Results are cached per GPU model, mesh,
acquisition and time axis in a JSON file (default
~/.cache/gbfwi/autotune.json).
"""
from __future__ import annotations

import json
import os
import statistics

from . import Mesh, num_tiles

CACHE = os.environ.get("GBFWI_AUTOTUNE_CACHE", os.path.expanduser("~/.cache/gbfwi/autotune.json"))
VERSION = 3


def _signature(nex, nez, nshot, nrec, nt, gpu_name, space):
    return f"v{VERSION}|{gpu_name}|{nex}x{nez}|shots{nshot}|rec{nrec}|nt{nt}|{space}"


def schedule_bytes(nx, nz, nshot, nrec, nt, spl, streams, ckpt):
    """Device bytes of gbfwi_adjoint_gradient's work buffers for a schedule
    on the full time axis (the layout of sem_driver.cu)."""
    pitch = (nx + 3) // 4 * 4
    NP = nz * pitch
    B = min(spl, nshot)
    lanes = max(1, min(streams, -(-nshot // B)))
    lev = B * NP * 8                                   # one float2 time level of a batch
    if ckpt <= 0 or ckpt >= nt:
        hist = (nt + 2) * lev
    else:
        nseg = -(-nt // ckpt)
        hist = (3 + ckpt + 2 + 1) * lev + nseg * 3 * lev
    per_lane = hist + lev * (1 + 3 + 1) + B * nrec * 2 * nt * 4 + B * 5 * NP * 4
    return lanes * per_lane + nshot * 5 * NP * 4 + 5 * NP * 4 + nshot * nrec * 2 * nt * 4


def tune(nex, nez, h, dt, nt, sources, rec_xz, model, probe_nt=200, repeats=3, tiles=None,
         spl_options=(1, 2, 4, 8, 24), stream_options=(1, 2, 4, 8), ckpt_options=(400,), mem_budget=None,
         use_cache=True):
    """Return (best schedule dict, timings list).  `model` = (rho, vp, vs)
    float32 CUDA tensors on the node grid; nt is the full time axis the
    schedule is for (memory), probe_nt the short axis the probes run."""
    import torch

    dev = model[0].device
    gpu = torch.cuda.get_device_name(dev)
    nshot = len(sources)
    tiles = list(range(num_tiles())) if tiles is None else list(tiles)
    space = f"t{','.join(map(str, tiles))}|s{','.join(map(str, spl_options))}|l{','.join(map(str, stream_options))}" \
            f"|c{','.join(map(str, ckpt_options))}|p{probe_nt}"
    sig = _signature(nex, nez, nshot, len(rec_xz), nt, gpu, space)
    if use_cache and os.path.exists(CACHE):
        try:
            db = json.load(open(CACHE))
            if sig in db:
                return db[sig]["best"], db[sig]["timings"]
        except Exception:
            pass
    if mem_budget is None:
        free, _ = torch.cuda.mem_get_info(dev)
        mem_budget = 0.8 * free
    m = Mesh(nex, nez, h, dt, probe_nt, sources, rec_xz)
    m.set_model(*model)
    ids = list(range(nshot))
    obs = torch.zeros(nshot, len(rec_xz), 2, probe_nt, device=dev)
    grad = torch.zeros(3, m.nz, m.nx, device=dev)
    stream = torch.cuda.current_stream(dev)
    timings, seen = [], {}

    def probe_ckpt(ck):
        if ck <= 0 or ck >= nt:
            return 0
        nseg = -(-nt // ck)
        return max(2, -(-probe_nt // nseg))

    def run(sch):
        key = tuple(sorted(sch.items()))
        if key in seen:
            return seen[key]
        need = schedule_bytes(m.nx, m.nz, nshot, len(rec_xz), nt, sch["shots_per_launch"], sch["streams"],
                              sch["ckpt_every"])
        if need > mem_budget:
            seen[key] = None
            return None
        m.set_schedule(shots_per_launch=sch["shots_per_launch"], tile=sch["tile"], use_graph=sch["use_graph"],
                       ckpt_every=probe_ckpt(sch["ckpt_every"]), streams=sch["streams"])
        m.adjoint_gradient(ids, obs, grad)                  # warm-up, graph capture
        us = []
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.adjoint_gradient(ids, obs, grad)
            e1.record(stream)
            e1.synchronize()
            us.append(1e3 * e0.elapsed_time(e1) / (nshot * probe_nt))
        r = statistics.median(us)
        seen[key] = r
        timings.append(dict(schedule=dict(sch), us_per_shot_step=r, device_bytes=need))
        return r

    def best_of(cands):
        scored = [(run(c), i, c) for i, c in enumerate(cands)]
        scored = [s for s in scored if s[0] is not None]
        return min(scored)[2] if scored else None

    base = dict(shots_per_launch=1, tile=tiles[0], use_graph=1, ckpt_every=0, streams=min(4, nshot))
    # A. tile shape at the default lane schedule (checkpointed if the full
    #    history does not fit)
    cur = best_of([dict(base, tile=t) for t in tiles])
    if cur is None:
        cur = best_of([dict(base, tile=t, ckpt_every=c) for t in tiles for c in ckpt_options])
    if cur is None:
        raise RuntimeError("no schedule fits the device memory budget")
    # B. lanes x shots per launch
    cands = []
    for spl in spl_options:
        for ln in stream_options:
            if spl > nshot or (ln > 1 and spl * ln > nshot):
                continue
            for ck in (0,) + tuple(ckpt_options):
                cands.append(dict(cur, shots_per_launch=spl, streams=ln, ckpt_every=ck))
    cur = best_of(cands + [cur])
    # C. graphs off for the pick
    cur = best_of([cur, dict(cur, use_graph=0)])
    if use_cache:
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            db = json.load(open(CACHE)) if os.path.exists(CACHE) else {}
            db[sig] = {"best": cur, "timings": timings}
            json.dump(db, open(CACHE, "w"), indent=1)
        except Exception:
            pass
    return cur, timings
