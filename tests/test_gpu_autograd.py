"""The misfit as a torch.autograd.Function (forward = forward simulations,
backward = adjoint with checkpoint-every-N recomputation), on the 340 x 70
element mesh with all 24 shots in one launch and a shortened time axis:

* forward() equals gbfwi_misfit, backward() equals gbfwi_adjoint_gradient
  bitwise;
* the gradient against central finite differences of the misfit with a
  relative step of 1e-3 along 20 seeded smooth perturbations (Gaussian bumps
  on all three parameters): median relative error below 1e-2 and every
  error below 1e-2 of the rms directional derivative (the misfit is
  FP64-reduced from FP32 simulations).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import paper_2009_12663_gb300 as gb  # noqa: E402
from paper_2009_12663_gb300.autograd import fwi_misfit  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def setup():
    nt = 400
    wl = synth.marmousi_like_workload(nt=nt)
    m = gb.Mesh(wl.nex, wl.nez, wl.h, wl.dt, nt, wl.sources(amp=1e12), wl.rec_xz)
    m.set_schedule(shots_per_launch=24, tile=0, ckpt_every=64)
    x, z = m.node_coords()
    W, H = wl.nex * wl.h, wl.nez * wl.h
    true = [torch.tensor(a, dtype=torch.float32, device=DEV) for a in synth.marmousi_like(x, z, 7, W, H)]
    start = [torch.tensor(a, dtype=torch.float32, device=DEV) for a in synth.marmousi_like_smooth(x, z, 7, W, H)]
    ids = list(range(24))
    obs = torch.zeros(24, wl.nrec, 2, nt, device=DEV)
    m.set_model(*true)
    m.forward(ids, obs)
    return m, ids, obs, start, x, z


def test_autograd_equals_abi(setup):
    m, ids, obs, start, _, _ = setup
    params = [t.clone().requires_grad_(True) for t in start]
    f = fwi_misfit(*params, m, ids, obs, 64)
    f.backward()
    m.set_model(*start)
    assert f.item() == m.misfit(ids, obs)
    grad = torch.zeros(3, m.nz, m.nx, device=DEV)
    m.adjoint_gradient(ids, obs, grad, 64)
    for c in range(3):
        assert torch.equal(params[c].grad, grad[c])


def test_autograd_gradient_against_finite_differences(setup):
    m, ids, obs, start, x, z = setup
    params = [t.clone().requires_grad_(True) for t in start]
    f = fwi_misfit(*params, m, ids, obs, 64)
    f.backward()
    g = [p.grad.double() for p in params]
    rng = np.random.default_rng(20)
    fds, ans = [], []
    eps = 1e-3
    for _ in range(20):
        dm = []
        for c in range(3):
            cx, cz = rng.uniform(0, x.max()), rng.uniform(0, z.max())
            bump = np.exp(-((x - cx) ** 2 + (z - cz) ** 2) / (2 * 600.0 ** 2))
            dm.append(torch.tensor(bump, dtype=torch.float64, device=DEV) * start[c].double())
        with torch.no_grad():
            fp = fwi_misfit(*[(s.double() + eps * d).float().contiguous() for s, d in zip(start, dm)],
                            m, ids, obs, 64).item()
            fm = fwi_misfit(*[(s.double() - eps * d).float().contiguous() for s, d in zip(start, dm)],
                            m, ids, obs, 64).item()
        fds.append((fp - fm) / (2 * eps))
        ans.append(float(sum((gc * d).sum() for gc, d in zip(g, dm))))
    fds, ans = np.array(fds), np.array(ans)
    rel_err = np.abs(fds - ans) / np.abs(ans)
    # directions whose derivative nearly cancels are compared with the
    # typical derivative size instead of their own
    scaled = np.abs(fds - ans) / np.sqrt(np.mean(ans ** 2))
    print("FD: median relative error %.2e, max error / rms derivative %.2e" % (np.median(rel_err), scaled.max()))
    assert np.median(rel_err) < 1e-2
    assert scaled.max() < 1e-2
