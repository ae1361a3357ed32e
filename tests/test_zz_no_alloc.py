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


def _call(L, syn, obs, nshot, per_shot, dt, stream=None):
    out = np.full(nshot, -1.0)
    rc = L.gbfwi_misfit_noalloc(ctypes.c_void_p(syn.data_ptr()), ctypes.c_void_p(obs.data_ptr()), nshot,
                                per_shot, dt, ctypes.c_void_p(out.ctypes.data), stream)
    return rc, out


def test_misfit_noalloc_short_shots_after_long_ones():
    """Every block of every shot rewrites its partial sum, also when the shot
    has fewer samples than one grid stride (64 blocks x 256 threads), so
    most blocks see no sample: a short call after a long one must not pick
    up the long call's partials."""
    L = gb.lib()
    g = torch.Generator(device=DEV).manual_seed(11)
    long_n, short_n, dt = 3 * 64 * 256 + 17, 1000, 1e-3
    syn = torch.randn(4, long_n, device=DEV, generator=g)
    obs = torch.randn(4, long_n, device=DEV, generator=g)
    rc, out = _call(L, syn, obs, 4, long_n, dt)
    # the residual is formed in FP32 and squared and summed in FP64
    ref = 0.5 * dt * ((syn - obs).double() ** 2).sum(1).cpu().numpy()
    assert rc == 0 and np.allclose(out, ref, rtol=1e-9)
    s2, o2 = syn[:, :short_n].contiguous(), obs[:, :short_n].contiguous()
    for _ in range(2):
        rc, out = _call(L, s2, o2, 4, short_n, dt)
        ref = 0.5 * dt * ((s2 - o2).double() ** 2).sum(1).cpu().numpy()
        assert rc == 0 and np.allclose(out, ref, rtol=1e-9), (out, ref)


def test_misfit_noalloc_reserves_no_device_memory():
    """After a first call on the device (which loads the library's device
    code and its fixed scratch array), further calls leave the device's free
    memory unchanged."""
    L = gb.lib()
    syn = torch.ones(8, 5000, device=DEV)
    obs = torch.zeros(8, 5000, device=DEV)
    rc, _ = _call(L, syn, obs, 8, 5000, 1e-3)
    assert rc == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        rc, out = _call(L, syn, obs, 8, 5000, 1e-3)
        assert rc == 0 and np.allclose(out, 0.5 * 1e-3 * 5000)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_misfit_noalloc_refuses_a_capturing_stream():
    """The call synchronises and copies to host memory, which a stream under
    CUDA-graph capture cannot do: it returns EINVAL instead of breaking the
    capture."""
    L = gb.lib()
    syn = torch.ones(2, 100, device=DEV)
    obs = torch.zeros(2, 100, device=DEV)
    graph = torch.cuda.CUDAGraph()
    rcs = []
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rcs.append(_call(L, syn, obs, 2, 100, 1e-3, st)[0])
    assert rcs == [-1]


def test_misfit_noalloc_rejects_more_shots_than_its_scratch():
    L = gb.lib()
    a = torch.zeros(4, device=DEV)
    out = np.zeros(300)
    rc = L.gbfwi_misfit_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()), 257, 1, 1e-3,
                                ctypes.c_void_p(out.ctypes.data), None)
    assert rc == -9
    assert b"scratch" in L.gbfwi_strerror(rc)
