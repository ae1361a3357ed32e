"""FP64 oracle for the learned diagonal preconditioner: a U-Net that maps
(vp, vs, rho, source-illumination mask, receiver-coverage mask) on an image
grid to the logarithm of the diagonal pseudo-Hessian (the P-maps of
Eqs. 5-8), its exact backward pass, the mean-squared loss, the Adam update
(Kingma & Ba 2015) and the bilinear resampling between the node grid and
the image grid.  The paper has no learned component; this part follows the
standard U-Net (Ronneberger, Fischer & Brox 2015): per level two 3x3
convolutions with ReLU, 2x2 average pooling down, nearest-neighbour 2x
upsampling up, skip connections concatenated after the upsampled features,
and a 1x1 output convolution.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every operation is written from its definition: a convolution is the sum
over input channels and the 3 x 3 taps of shifted inputs times weights, its
adjoints are the same sums with the roles exchanged.  With `bf16=True`
weights, inputs and stored activations are rounded to bfloat16 at the points
where the CUDA path stores them (round to nearest even), while every sum is
FP64.

Parameter shapes: W [cout][cin][3][3] (or [cout][cin][1][1]), b [cout];
order: encoder levels 0..L-1 (two convolutions each), decoder levels L-2..0
(two each, the first on [upsampled, skip] channels), output 1x1.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------- rounding --

def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def _r(a, on: bool):
    return bf16(a) if on else np.asarray(a, np.float64)


# ------------------------------------------------------------- operations --

def conv3x3(X: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[o, y, x] = b[o] + sum_{c, ky, kx} W[o, c, ky, kx] X[c, y + ky - 1, x + kx - 1]
    with X zero outside the image."""
    C, H, Wd = X.shape
    Xp = np.zeros((C, H + 2, Wd + 2))
    Xp[:, 1:-1, 1:-1] = X
    out = np.broadcast_to(np.asarray(b, np.float64)[:, None, None], (W.shape[0], H, Wd)).copy()
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,chw->ohw", W[:, :, ky, kx], Xp[:, ky:ky + H, kx:kx + Wd])
    return out


def conv3x3_backward(X: np.ndarray, W: np.ndarray, dY: np.ndarray):
    """Adjoints of conv3x3: (dX, dW, db) for the output gradient dY."""
    C, H, Wd = X.shape
    Xp = np.zeros((C, H + 2, Wd + 2))
    Xp[:, 1:-1, 1:-1] = X
    dXp = np.zeros_like(Xp)
    dW = np.zeros_like(W, dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("ohw,chw->oc", dY, Xp[:, ky:ky + H, kx:kx + Wd])
            dXp[:, ky:ky + H, kx:kx + Wd] += np.einsum("oc,ohw->chw", W[:, :, ky, kx], dY)
    return dXp[:, 1:-1, 1:-1], dW, dY.sum(axis=(1, 2))


def conv1x1(X, W, b):
    return np.einsum("oc,chw->ohw", W[:, :, 0, 0], X) + np.asarray(b, np.float64)[:, None, None]


def conv1x1_backward(X, W, dY):
    dX = np.einsum("oc,ohw->chw", W[:, :, 0, 0], dY)
    dW = np.einsum("ohw,chw->oc", dY, X)[:, :, None, None]
    return dX, dW, dY.sum(axis=(1, 2))


def avgpool2(X):
    """out[c, y, x] = mean of X[c, 2y:2y+2, 2x:2x+2]."""
    C, H, W = X.shape
    return X.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def avgpool2_backward(dY):
    return np.repeat(np.repeat(dY, 2, axis=1), 2, axis=2) / 4.0


def upsample2(X):
    """Nearest neighbour: out[c, y, x] = X[c, y // 2, x // 2]."""
    return np.repeat(np.repeat(X, 2, axis=1), 2, axis=2)


def upsample2_backward(dY):
    C, H, W = dY.shape
    return dY.reshape(C, H // 2, 2, W // 2, 2).sum(axis=(2, 4))


# ------------------------------------------------------------------ U-Net --

def layer_shapes(levels: int, base: int, cin: int, cout: int):
    """(cout, cin, k) of every convolution in parameter order."""
    ch = [base * 2 ** l for l in range(levels)]
    shapes = []
    for l in range(levels):
        shapes.append((ch[l], cin if l == 0 else ch[l - 1], 3))
        shapes.append((ch[l], ch[l], 3))
    for l in range(levels - 2, -1, -1):
        shapes.append((ch[l], ch[l + 1] + ch[l], 3))
        shapes.append((ch[l], ch[l], 3))
    shapes.append((cout, ch[0], 1))
    return shapes


def init_params(levels, base, cin, cout, seed):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    params = []
    for co, ci, k in layer_shapes(levels, base, cin, cout):
        std = np.sqrt(2.0 / (ci * k * k))
        params.append((rng.standard_normal((co, ci, k, k)) * std, np.zeros(co)))
    return params


def forward(params, x, levels: int, bf16_on: bool = False):
    """Returns (y, cache).  x: [cin][H][W]; y: [cout][H][W] (not rounded)."""
    R = lambda a: _r(a, bf16_on)
    P = [(R(W), np.asarray(b, np.float64)) for W, b in params]
    cache = {"x": R(x)}
    h = cache["x"]
    skips = []
    li = 0
    for l in range(levels):
        if l > 0:
            h = R(avgpool2(h))
            cache[f"p{l}"] = h
        a = R(np.maximum(conv3x3(h, *P[li]), 0.0)); li += 1
        cache[f"e{l}a"] = a
        h = R(np.maximum(conv3x3(a, *P[li]), 0.0)); li += 1
        cache[f"e{l}"] = h
        skips.append(h)
    for l in range(levels - 2, -1, -1):
        cat = np.concatenate([upsample2(h), skips[l]], axis=0)
        cache[f"cat{l}"] = cat
        a = R(np.maximum(conv3x3(cat, *P[li]), 0.0)); li += 1
        cache[f"d{l}a"] = a
        h = R(np.maximum(conv3x3(a, *P[li]), 0.0)); li += 1
        cache[f"d{l}"] = h
    y = conv1x1(h, *P[li])
    cache["params"] = P
    return y, cache


def backward(cache, dy, levels: int, bf16_on: bool = False):
    """Parameter gradients [(dW, db)] in parameter order for the output
    gradient dy, and the input gradient dx."""
    R = lambda a: _r(a, bf16_on)
    P = cache["params"]
    nl = len(P)
    grads = [None] * nl
    li = nl - 1
    top = cache["d0"] if levels > 1 else cache[f"e{levels - 1}"]
    dh, dW, db = conv1x1_backward(top, P[li][0], R(dy))
    grads[li] = (dW, db)
    dskip = {}
    for l in range(0, levels - 1):
        li -= 1
        g = R(dh * (cache[f"d{l}"] > 0))
        da, dW, db = conv3x3_backward(cache[f"d{l}a"], P[li][0], g)
        grads[li] = (dW, db)
        li -= 1
        g = R(da * (cache[f"d{l}a"] > 0))
        dcat, dW, db = conv3x3_backward(cache[f"cat{l}"], P[li][0], g)
        grads[li] = (dW, db)
        cu = P[li][0].shape[1] - cache[f"e{l}"].shape[0]
        dskip[l] = dcat[cu:]
        dh = upsample2_backward(dcat[:cu])
    # encoder, bottleneck first
    for l in range(levels - 1, -1, -1):
        if l in dskip:
            dh = dh + dskip[l]
        li -= 1
        g = R(dh * (cache[f"e{l}"] > 0))
        da, dW, db = conv3x3_backward(cache[f"e{l}a"], P[li][0], g)
        grads[li] = (dW, db)
        li -= 1
        g = R(da * (cache[f"e{l}a"] > 0))
        inp = cache["x"] if l == 0 else cache[f"p{l}"]
        dx, dW, db = conv3x3_backward(inp, P[li][0], g)
        grads[li] = (dW, db)
        if l > 0:
            dh = avgpool2_backward(dx)
    return grads, dx


def mse(y, target, channels=None):
    """L = mean over channels, pixels of (y - target)^2 and dL/dy."""
    c = y.shape[0] if channels is None else channels
    d = y[:c] - target[:c]
    n = d.size
    dy = np.zeros_like(y)
    dy[:c] = 2.0 * d / n
    return float((d * d).sum() / n), dy


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) with bias correction;
    t is the 1-based step count.  Returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------- resampling --

def resample_bilinear(src: np.ndarray, dh: int, dw: int) -> np.ndarray:
    """Bilinear resampling of [C][sh][sw] onto [C][dh][dw] with the corner
    samples of both grids aligned: destination (i, j) sits at source
    coordinates (i (sh-1)/(dh-1), j (sw-1)/(dw-1))."""
    C, sh, sw = src.shape
    out = np.zeros((C, dh, dw))
    for i in range(dh):
        y = i * (sh - 1) / (dh - 1) if dh > 1 else 0.0
        y0 = min(int(np.floor(y)), sh - 1)
        y1 = min(y0 + 1, sh - 1)
        fy = y - y0
        for j in range(dw):
            x = j * (sw - 1) / (dw - 1) if dw > 1 else 0.0
            x0 = min(int(np.floor(x)), sw - 1)
            x1 = min(x0 + 1, sw - 1)
            fx = x - x0
            out[:, i, j] = ((1 - fy) * ((1 - fx) * src[:, y0, x0] + fx * src[:, y0, x1])
                            + fy * ((1 - fx) * src[:, y1, x0] + fx * src[:, y1, x1]))
    return out


def features(rho, vp, vs, x, z, src_xz, rec_xz, sigma):
    """The five input channels on the node grid: vp / 4700, vs / 2700,
    rho / 2500 (fixed scales of the Marmousi-shaped range), and the source
    illumination and receiver coverage masks sum_s exp(-|x - x_s|^2 / 2 sigma^2),
    each divided by its maximum."""
    def mask(pts):
        m = np.zeros_like(np.asarray(x, np.float64))
        for px, pz in pts:
            m += np.exp(-((x - px) ** 2 + (z - pz) ** 2) / (2.0 * sigma ** 2))
        return m / m.max()
    return np.stack([np.asarray(vp, np.float64) / 4700.0, np.asarray(vs, np.float64) / 2700.0,
                     np.asarray(rho, np.float64) / 2500.0, mask(src_xz), mask(rec_xz)])
