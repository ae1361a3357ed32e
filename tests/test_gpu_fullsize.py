"""Parity at the benchmark's sizes.

* The 340 x 70 element Marmousi-shaped mesh (382,441 GLL points) with the
  benchmark's launch configuration: forward seismograms of two shots against
  the FP64 oracle over a shortened time axis (the oracle cannot run 12000
  steps in seconds), the gradient direction on the same truncated workload,
  and the batched / checkpointed schedule against the single-shot one,
  bitwise, with all 24 sources.
* The UQ problem at full size: n = 3 x 382,441, 50 pairs, 60 probes, rank
  50, against Algorithms 2-3 in FP64.
"""
import numpy as np
import pytest

import synth
from oracle import bfgs as ob
from oracle import sem as osem

torch = pytest.importorskip("torch")
import paper_2009_12663_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def cosine(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.fixture(scope="module")
def big():
    nt = 300
    wl = synth.marmousi_like_workload(nt=nt)
    m = gb.Mesh(wl.nex, wl.nez, wl.h, wl.dt, nt, wl.sources(amp=1e12), wl.rec_xz)
    x, z = m.node_coords()
    W, H = wl.nex * wl.h, wl.nez * wl.h
    true = synth.marmousi_like(x, z, 2024, W, H)
    start = synth.marmousi_like_smooth(x, z, 2024, W, H)
    return wl, m, true, start


def _model(m, arrays):
    m.set_model(*[torch.tensor(a, dtype=torch.float32, device=DEV) for a in arrays])


def test_fullsize_forward_two_shots_match_oracle(big):
    wl, m, true, start = big
    ids = [0, 17]
    _model(m, start)
    seis = torch.zeros(2, wl.nrec, 2, wl.nt, device=DEV)
    m.forward(ids, seis)
    st = osem.Setup(osem.Mesh(wl.nex, wl.nez, wl.h), wl.dt, wl.nt, wl.rec_xz)
    srcs = wl.sources(amp=1e12)
    got = seis.cpu().numpy()
    for j, s in enumerate(ids):
        fv, stf = st.source(srcs[s])
        ref = st.forward(start, fv, stf)
        assert rel(got[j], ref) < 1e-4


def test_fullsize_gradient_direction_matches_oracle(big):
    wl, m, true, start = big
    sid = 5
    st = osem.Setup(osem.Mesh(wl.nex, wl.nez, wl.h), wl.dt, wl.nt, wl.rec_xz)
    src = wl.sources(amp=1e12)[sid]
    fv, stf = st.source(src)
    obs_ref = st.forward(true, fv, stf)
    f_ref, g_ref, _ = osem.misfit_gradient(st, start, [src], [obs_ref])
    _model(m, true)
    obs = torch.zeros(1, wl.nrec, 2, wl.nt, device=DEV)
    m.forward([sid], obs)
    _model(m, start)
    grad = torch.zeros(3, m.nz, m.nx, device=DEV)
    f = m.adjoint_gradient([sid], obs, grad)
    g = grad.cpu().numpy()
    assert abs(f - f_ref) / f_ref < 1e-2
    for c in range(3):
        assert cosine(g[c], g_ref[c]) > 1 - 1e-3, c


def test_fullsize_batched_checkpointed_equals_single_shot_bitwise(big):
    wl, m, true, start = big
    ids = list(range(24))
    _model(m, true)
    obs = torch.zeros(24, wl.nrec, 2, wl.nt, device=DEV)
    m.forward(ids, obs)
    _model(m, start)
    out = []
    for sched in (dict(shots_per_launch=1, ckpt_every=0), dict(shots_per_launch=24, ckpt_every=64),
                  dict(shots_per_launch=8, ckpt_every=0, tile=4), dict(shots_per_launch=1, streams=4, use_graph=1),
                  dict(shots_per_launch=2, streams=3, ckpt_every=100)):
        m.set_schedule(**sched)
        grad = torch.zeros(3, m.nz, m.nx, device=DEV)
        f = m.adjoint_gradient(ids, obs, grad)
        out.append((f, grad.cpu().numpy()))
    m.set_schedule(shots_per_launch=1, ckpt_every=0, tile=0)
    for f, g in out[1:]:
        assert f == out[0][0]
        assert np.array_equal(g, out[0][1])


def test_fullsize_uq_matches_algorithm_3():
    n, k, p, rank = 3 * 382441, 50, 60, 50
    S, Y, B0 = synth.synthetic_history(77, n, k)
    b = gb.Bfgs(n, k, torch.tensor(B0, device=DEV))
    for i in range(k):
        b.update(torch.tensor(S[i], device=DEV), torch.tensor(Y[i], device=DEV))
    X = synth.gaussian_block(5, p, n)
    lam = torch.zeros(rank, dtype=torch.float64, device=DEV)
    std = torch.zeros(n, device=DEV)
    V = torch.zeros(rank, n, device=DEV)
    b.lowrank_invhess(p, rank, eps_prior=1.0, X=torch.tensor(X, device=DEV), V=V, lam=lam, std=std)
    S64, Y64, B64 = S.astype(np.float64), Y.astype(np.float64), B0.astype(np.float64)
    E = ob.probe_block(X.astype(np.float64), S64, Y64, B64)
    Vr, lr = ob.rsvd_single_pass(E, X.astype(np.float64), rank)
    assert np.allclose(lam.cpu().numpy(), lr, rtol=1e-4, atol=1e-6 * np.abs(lr).max())
    assert rel(std.cpu().numpy(), ob.posterior_std(Vr, lr, B64, 1.0)) < 1e-4
    # the low-rank part V diag(lam) V^T applied to a probe equals the oracle's
    Vg = V.cpu().numpy().astype(np.float64)
    x = np.random.default_rng(0).standard_normal(n)
    lg = lam.cpu().numpy()
    assert rel(Vg.T @ (lg * (Vg @ x)), Vr.T @ (lr * (Vr @ x))) < 1e-3
