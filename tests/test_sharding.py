"""Shot sharding across ranks: the shard blocks partition the shots, and a
world-size-2 gloo run whose ranks each compute the misfit and gradient of
their own shots (FP64 oracle on the CPU) and sum them with
allreduce_gradient reproduces the single-process result."""
import os
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2009_12663_gb300.sharding import allreduce_gradient, shard


@pytest.mark.parametrize("n,w", [(24, 1), (24, 2), (24, 5), (3, 4), (0, 3), (7, 7)])
def test_shard_partitions_shots(n, w):
    parts = [shard(n, r, w) for r in range(w)]
    flat = [s for p in parts for s in p]
    assert flat == list(range(n))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1


def _case():
    import synth
    from oracle import sem
    st = sem.Setup(sem.Mesh(8, 5, 25.0), 5e-4, 200, np.stack([np.linspace(0, 200, 9), np.full(9, 5.0)], 1))
    x, z = st.mesh.coords()
    true = synth.gaussian_anomaly(x, z, seed=1, xrange=(60, 140), zrange=(40, 80))
    start = synth.homogeneous(x, z)
    srcs = [dict(x=xs, z=10.0, type=0, f0=30.0, t0=0.04, amp=1e10) for xs in (30.0, 80.0, 120.0, 170.0)]
    obs = []
    for s in srcs:
        fv, stf = st.source(s)
        obs.append(st.forward(true, fv, stf))
    return st, start, srcs, obs


def _rank(rank, world, path, out):
    from oracle import sem
    dist.init_process_group("gloo", init_method=f"file://{path}", rank=rank, world_size=world)
    st, start, srcs, obs = _case()
    mine = shard(len(srcs), rank, world)
    f, g, _ = sem.misfit_gradient(st, start, [srcs[i] for i in mine], [obs[i] for i in mine])
    gt = torch.tensor(g)
    total = allreduce_gradient(gt, f)
    if rank == 0:
        np.save(out, np.concatenate([[total], gt.numpy().ravel()]))
    dist.destroy_process_group()


def test_two_rank_gloo_gradient_equals_single_process():
    from oracle import sem
    st, start, srcs, obs = _case()
    f, g, _ = sem.misfit_gradient(st, start, srcs, obs)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "r0.npy")
        mp.spawn(_rank, args=(2, os.path.join(d, "pg"), out), nprocs=2, join=True)
        res = np.load(out)
    assert abs(res[0] - f) <= 1e-12 * f
    assert np.allclose(res[1:].reshape(g.shape), g, rtol=1e-12, atol=1e-12 * np.abs(g).max())


def _rank_product(rank, world, path, out, nshot):
    """One rank of sharded_adjoint_gradient, the product's partition and
    reduction, with the oracle standing in for the per-rank CUDA compute."""
    from oracle import sem
    from paper_2009_12663_gb300.sharding import sharded_adjoint_gradient
    dist.init_process_group("gloo", init_method=f"file://{path}", rank=rank, world_size=world)
    st, start, srcs, obs = _case()
    srcs, obs = srcs[:nshot], obs[:nshot]
    ids = list(range(len(srcs)))
    calls = []

    def stand_in(my_ids, d_blk, g):
        calls.append(list(my_ids))
        f, gr, _ = sem.misfit_gradient(st, start, [srcs[i] for i in my_ids], list(d_blk))
        g.copy_(torch.tensor(gr))
        return f

    grad = torch.full((3, st.mesh.nz, st.mesh.nx), float("nan"), dtype=torch.float64)
    total = sharded_adjoint_gradient(None, ids, np.stack(obs), grad, compute=stand_in)
    np.save(out + f".{rank}.npy", np.concatenate([[total], grad.numpy().ravel()]))
    with open(out + f".{rank}.calls", "w") as fh:
        fh.write(repr(calls))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nshot", [(2, 4), (3, 2)])
def test_sharded_adjoint_gradient_equals_single_process(world, nshot):
    """Every rank ends with the single-process misfit and gradient; each
    rank computed only its own block of shots (a rank without shots adds
    zeros)."""
    from oracle import sem
    st, start, srcs, obs = _case()
    f, g, _ = sem.misfit_gradient(st, start, srcs[:nshot], obs[:nshot])
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "res")
        mp.spawn(_rank_product, args=(world, os.path.join(d, "pg"), out, nshot), nprocs=world, join=True)
        for r in range(world):
            res = np.load(out + f".{r}.npy")
            calls = eval(open(out + f".{r}.calls").read())
            mine = shard(nshot, r, world)
            assert calls == ([mine] if mine else [])
            assert abs(res[0] - f) <= 1e-12 * f
            assert np.allclose(res[1:].reshape(g.shape), g, rtol=1e-12, atol=1e-12 * np.abs(g).max())
