"""gbfwi_misfit_noalloc: the misfit for callers that cannot allocate device
memory during a call (their own pool owns the GPU memory, or they cannot
risk an allocation failure inside a time-critical loop).  Called through the
C ABI and compared with the misfit gbfwi_adjoint_gradient returns, twice in
a row (the shared scratch keeps the previous call's contents)."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import paper_2009_12663_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_misfit_noalloc_matches_adjoint_gradient_misfit_twice():
    nex, nez, h, dt, nt = 12, 6, 50.0, 5e-4, 400
    rec = np.stack([50.0 * np.arange(13), np.zeros(13)], 1)
    srcs = [dict(x=x, z=20.0, type=0, f0=15.0, amp=1e12) for x in (150.0, 300.0, 450.0)]
    m = gb.Mesh(nex, nez, h, dt, nt, srcs, rec)
    x, z = m.node_coords()
    true = [torch.tensor(a, dtype=torch.float32, device=DEV)
            for a in synth.gaussian_anomaly(x, z, seed=2, xrange=(200, 400), zrange=(100, 200))]
    start = [torch.tensor(a, dtype=torch.float32, device=DEV) for a in synth.homogeneous(x, z)]
    ids = [0, 1, 2]
    d_obs = torch.zeros(3, 13, 2, nt, device=DEV)
    m.set_model(*true)
    m.forward(ids, d_obs)
    m.set_model(*start)
    syn = torch.zeros(3, 13, 2, nt, device=DEV)
    m.forward(ids, syn)
    grad = torch.zeros(3, m.nz, m.nx, device=DEV)
    ref_total = m.adjoint_gradient(ids, d_obs, grad)
    ref_shot = [m.adjoint_gradient([s], d_obs[s:s + 1].contiguous(), grad) for s in ids]
    torch.cuda.synchronize()
    L = gb.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    per_shot = 13 * 2 * nt
    for call in range(2):
        out = np.full(3, -1.0)
        rc = L.gbfwi_misfit_noalloc(ctypes.c_void_p(syn.data_ptr()), ctypes.c_void_p(d_obs.data_ptr()), 3,
                                    per_shot, dt, ctypes.c_void_p(out.ctypes.data), stream)
        assert rc == 0, L.gbfwi_strerror(rc)
        assert np.allclose(out, ref_shot, rtol=1e-4), (call, out, ref_shot)
        assert abs(out.sum() - ref_total) <= 1e-4 * ref_total
    # one shot after three: the scratch keeps stale partials of shots 1-2,
    # which must not leak into the result
    out1 = np.zeros(1)
    rc = L.gbfwi_misfit_noalloc(ctypes.c_void_p(syn.data_ptr()), ctypes.c_void_p(d_obs.data_ptr()), 1,
                                per_shot, dt, ctypes.c_void_p(out1.ctypes.data), stream)
    assert rc == 0 and abs(out1[0] - ref_shot[0]) <= 1e-4 * ref_shot[0]


def test_misfit_noalloc_rejects_more_shots_than_its_scratch():
    L = gb.lib()
    a = torch.zeros(4, device=DEV)
    out = np.zeros(300)
    rc = L.gbfwi_misfit_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()), 257, 1, 1e-3,
                                ctypes.c_void_p(out.ctypes.data), None)
    assert rc == -9
    assert b"scratch" in L.gbfwi_strerror(rc)
