"""Full-length parity at the benchmark's size: one shot of the Marmousi-shaped
340 x 70 element workload (382,441 GLL points, 341 receivers, dt 0.5 ms)
over all 12000 steps, so that the FP32 drift of the whole time axis is
measured, against the FP64 oracle's values stored in
tests/golden/marmousi_shot11_full.npz (written by
tests/golden/make_marmousi_full_length.py, which calls only oracle/).

* records of the true and of the starting model at every 20th receiver and
  every 10th sample: 1e-4 relative L2;
* the misfit (Eq. A1) and the gradient projected on three smooth directions
  (one per parameter), against the oracle's central differences of the
  misfit: the gradient is the exact derivative of the discrete misfit, so
  the projections agree up to FP32 rounding (1e-3);
* checkpointing every 400 steps with recomputation gives bitwise the
  gradient of the full history.
"""
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import paper_2009_12663_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLD = os.path.join(os.path.dirname(__file__), "golden", "marmousi_shot11_full.npz")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_full_length_shot_against_fp64_oracle():
    g = np.load(GOLD)
    wl = synth.marmousi_like_workload()
    assert int(g["nt"]) == wl.nt == 12000
    shot = int(g["shot"])
    srcs = wl.sources(amp=1e12)
    m = gb.Mesh(wl.nex, wl.nez, wl.h, wl.dt, wl.nt, srcs, wl.rec_xz)
    x, z = m.node_coords()
    W, H = wl.nex * wl.h, wl.nez * wl.h
    seed = int(g["seed"])
    true = [torch.tensor(a, dtype=torch.float32, device=DEV) for a in synth.marmousi_like(x, z, seed, W, H)]
    start = [torch.tensor(a, dtype=torch.float32, device=DEV) for a in synth.marmousi_like_smooth(x, z, seed, W, H)]
    ridx, tidx = g["rec_idx"], g["t_idx"]

    d_obs = torch.zeros(1, wl.nrec, 2, wl.nt, device=DEV)
    m.set_model(*true)
    m.forward([shot], d_obs)
    syn = torch.zeros_like(d_obs)
    m.set_model(*start)
    m.forward([shot], syn)
    torch.cuda.synchronize()
    for got, key in ((d_obs, "seis_true"), (syn, "seis_start")):
        sub = got[0].cpu().numpy()[ridx][:, :, tidx]
        err = _rel(sub, g[key].astype(np.float64))
        print(f"{key}: relative L2 {err:.2e} over 12000 steps")
        assert err < 1e-4, (key, err)

    grad = torch.zeros(3, m.nz, m.nx, device=DEV)
    f = m.adjoint_gradient([shot], d_obs, grad, ckpt_every=0)
    f_ref = float(g["misfit"])
    print(f"misfit {f:.9e} oracle {f_ref:.9e} rel {abs(f - f_ref) / f_ref:.2e}")
    assert abs(f - f_ref) <= 1e-4 * f_ref
    G = grad.double().cpu().numpy()
    xs = srcs[shot]["x"]
    bump = np.exp(-((x - xs) ** 2 + (z - float(g["depth"])) ** 2) / (2.0 * float(g["sigma"]) ** 2))
    st = [a.double().cpu().numpy() for a in start]
    for c in range(3):
        proj = float(np.sum(G[c] * st[c] * bump))
        ref = float(g["dfd"][c])
        print(f"parameter {c}: projection {proj:.6e} oracle central difference {ref:.6e} "
              f"rel {abs(proj - ref) / abs(ref):.2e}")
        assert abs(proj - ref) <= 1e-3 * abs(ref), (c, proj, ref)

    grad_ck = torch.zeros_like(grad)
    f_ck = m.adjoint_gradient([shot], d_obs, grad_ck, ckpt_every=400)
    assert f_ck == f
    assert torch.equal(grad_ck, grad)
