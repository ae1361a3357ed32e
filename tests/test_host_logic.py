"""Host-side logic that runs without a GPU: parameter packing of the FWI
driver, model clamping, the robust first-step scale, and the flat padded
parameter layout of the learned preconditioner."""
import numpy as np
import pytest

from oracle import unet as ou

torch = pytest.importorskip("torch")
from paper_2009_12663_gb300 import fwi, learned  # noqa: E402


def test_pack_unpack_round_trip():
    m = torch.arange(3 * 4 * 5, dtype=torch.float32).reshape(3, 4, 5)
    mask = torch.tensor([False, True, True])
    v = fwi.pack(m, mask)
    assert v.numel() == 2 * 20 and torch.equal(v[:20], m[1].reshape(-1))
    back = fwi.unpack(v, mask, m)
    assert torch.equal(back[1:], m[1:]) and torch.all(back[0] == 0)


def test_clamp_model_bounds():
    m = torch.tensor([[[50.0]], [[9000.0]], [[7000.0]]])
    c = fwi.clamp_model(m)
    assert float(c[0]) == 100.0 and float(c[1]) == 8000.0 and float(c[2]) == pytest.approx(0.7 * 8000.0)


def test_robust_max_ignores_a_spike():
    v = torch.randn(2_000_000, generator=torch.Generator().manual_seed(0))
    v[123] = 1e9
    r = fwi.robust_max(v)
    assert 2.5 < r < 4.0                       # 99.9th percentile of |N(0,1)| is ~3.29
    assert fwi.robust_max(torch.ones(10)) == 1.0


def _layers(levels, base, cin, cout):
    """The library's layout rule: per layer [round8(cout)][round8(cin k k)]
    weights then round8(cout) biases, offsets rounded to 8."""
    r8 = lambda v: (v + 7) // 8 * 8
    out, off = [], 0
    for co, ci, k in ou.layer_shapes(levels, base, cin, cout):
        coutp, kcp = r8(co), r8(ci * k * k)
        wo = off
        bo = wo + coutp * kcp
        off = r8(bo + coutp)
        out.append((co, ci, k, coutp, kcp, wo, bo))
    return out, off


def test_unet_parameter_packing_round_trip():
    layers, total = _layers(3, 8, 5, 3)
    params = ou.init_params(3, 8, 5, 3, seed=2)
    rng = np.random.default_rng(0)
    params = [(W, rng.standard_normal(b.shape)) for W, b in params]
    flat = learned.pack(layers, params)
    assert flat.size == total
    back = learned.unpack(layers, flat)
    for (W, b), (W2, b2) in zip(params, back):
        assert np.allclose(W.astype(np.float32), W2) and np.allclose(b.astype(np.float32), b2)
    # padding stays zero: first layer has cin k k = 45 -> 48 columns, the
    # output layer 3 -> 8 rows
    co, ci, k, coutp, kcp, wo, bo = layers[0]
    blk = flat[wo:wo + coutp * kcp].reshape(coutp, kcp)
    assert kcp == 48 and np.all(blk[:, 45:] == 0)
    co, ci, k, coutp, kcp, wo, bo = layers[-1]
    assert coutp == 8 and np.all(flat[wo + 3 * kcp:wo + coutp * kcp] == 0) and np.all(flat[bo + 3:bo + 8] == 0)
