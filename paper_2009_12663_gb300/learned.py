"""Learned diagonal preconditioner around the C ABI: a U-Net (gbfwi_unet)
trained on the pseudo-Hessian maps the method itself computes (P4 of
Eqs. 7-8 / A22, gbfwi_precond_diag), used to predict B0 for a new model,
with the computed map as fallback and as the measure of its error.

Argument marshalling and bookkeeping only: features, resampling, the
network's forward / backward / Adam steps and the smoothing-damping-
inversion into B0 all run in the CUDA library.

    X, T = make_pairs(mesh, models, shot_ids, 256, 1024)   # features, log-H targets
    lp = LearnedPreconditioner(Unet(...)); lp.fit(X, T, steps=...)
    B0, info = lp.b0(mesh, model, sigma, damp, computed_H=None)
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import Mesh, Unet, resample

MASK_SIGMA_M = 500.0       # width of the source / receiver masks


def pack(layers, params) -> np.ndarray:
    """[(W [cout][cin][k][k], b [cout])] -> flat FP32 vector in the padded
    layout of gbfwi_unet_layer_info."""
    total = max(l[6] + l[3] for l in layers)
    flat = np.zeros((total + 7) // 8 * 8, np.float32)
    for (cout, cin, k, coutp, kcp, wo, bo), (W, b) in zip(layers, params):
        blk = np.zeros((coutp, kcp), np.float32)
        blk[:cout, :cin * k * k] = np.asarray(W, np.float32).reshape(cout, cin * k * k)
        flat[wo:wo + coutp * kcp] = blk.ravel()
        flat[bo:bo + cout] = np.asarray(b, np.float32)
    return flat


def unpack(layers, flat):
    """Inverse of pack (padding dropped)."""
    flat = np.asarray(flat)
    out = []
    for cout, cin, k, coutp, kcp, wo, bo in layers:
        blk = flat[wo:wo + coutp * kcp].reshape(coutp, kcp)
        out.append((blk[:cout, :cin * k * k].reshape(cout, cin, k, k), flat[bo:bo + cout].copy()))
    return out


def he_init(net: Unet, seed: int) -> np.ndarray:
    """He-normal weights, zero biases (seeded), in the padded flat layout."""
    rng = np.random.default_rng(seed)
    params = []
    for cout, cin, k, *_ in net.layers():
        params.append((rng.standard_normal((cout, cin, k, k)) * np.sqrt(2.0 / (cin * k * k)), np.zeros(cout)))
    flat = pack(net.layers(), params)
    assert flat.size == net.num_params
    return flat


def features(mesh: Mesh, model: torch.Tensor, height: int, width: int) -> torch.Tensor:
    out = torch.zeros(5, height, width, device=model.device)
    return mesh.unet_features(model[0].contiguous(), model[1].contiguous(), model[2].contiguous(),
                              MASK_SIGMA_M, out)


def computed_map(mesh: Mesh, model: torch.Tensor, shot_ids, kind: int = 4, sigma: float = 100.0):
    """Raw pseudo-Hessian map H [3][nz][nx] of the method (P-map `kind`)."""
    mesh.set_model(model[0].contiguous(), model[1].contiguous(), model[2].contiguous())
    H = torch.zeros_like(model)
    B0 = torch.zeros_like(model)
    mesh.precond_diag(shot_ids, kind, sigma, 1.0, H, B0)
    return H


def log_image(H: torch.Tensor, height: int, width: int) -> torch.Tensor:
    out = torch.zeros(3, height, width, device=H.device)
    return resample(H.contiguous(), out, op=1)


def make_pairs(mesh: Mesh, models, shot_ids, height: int, width: int, kind: int = 4):
    """Training pairs (features [5][H][W], log H [3][H][W]) for each model,
    the targets computed by the method (one forward and one receiver-side
    backward simulation per shot for P4)."""
    X, T = [], []
    for mdl in models:
        X.append(features(mesh, mdl, height, width))
        T.append(log_image(computed_map(mesh, mdl, shot_ids, kind), height, width))
    return torch.stack(X).contiguous(), torch.stack(T).contiguous()


class LearnedPreconditioner:
    """U-Net predicting log H minus a per-channel offset (the mean of the
    training targets), so that the network learns the spatial pattern."""

    def __init__(self, net: Unet, seed: int = 0):
        self.net = net
        self.offset = torch.zeros(3, 1, 1)
        net.set_params(he_init(net, seed))
        self.history = []

    def fit(self, X: torch.Tensor, T: torch.Tensor, steps: int, lr: float = 1e-3, batch: int = 4, seed: int = 0,
            lr_decay: float = 1.0):
        self.offset = T.mean(dim=(0, 2, 3), keepdim=False).reshape(3, 1, 1)
        Tn = (T - self.offset.to(T.device)).contiguous()
        rng = np.random.default_rng(seed)
        n = X.shape[0]
        t0 = time.perf_counter()
        for it in range(steps):
            idx = rng.choice(n, size=min(batch, n), replace=False)
            xb, tb = X[idx].contiguous(), Tn[idx].contiguous()
            loss = self.net.train_step(xb, tb, lr * lr_decay ** it)
            self.history.append(loss)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def predict_log(self, x: torch.Tensor) -> torch.Tensor:
        y = torch.zeros(3, x.shape[-2], x.shape[-1], device=x.device)
        self.net.forward(x.contiguous(), y)
        return y + self.offset.to(y.device)

    def predict_map(self, mesh: Mesh, model: torch.Tensor) -> torch.Tensor:
        """Predicted raw map H [3][nz][nx] (exp of the resampled log map)."""
        x = features(mesh, model, self.net.height, self.net.width)
        ly = self.predict_log(x).contiguous()
        H = torch.zeros_like(model)
        return resample(ly, H, op=2)

    def b0(self, mesh: Mesh, model: torch.Tensor, sigma: float, damp: float, computed_H=None, tol: float = 0.2):
        """B0 from the predicted map; when a computed map is given and the
        prediction is off by more than `tol` (relative L2 of log H, worst
        parameter), the computed map is used instead."""
        Hp = self.predict_map(mesh, model)
        info = {"fallback": False, "rel_error": None}
        use = Hp
        if computed_H is not None:
            err = rel_log_error(Hp, computed_H)
            info["rel_error"] = err
            if err > tol:
                info["fallback"] = True
                use = computed_H
        B0 = torch.zeros_like(model)
        mesh.precond_from_hessian(use.contiguous(), sigma, damp, B0)
        return B0, info


def rel_log_error(Hp: torch.Tensor, H: torch.Tensor) -> float:
    """Worst over (rho, vp, vs) of |log Hp - log H|_2 / |log H - mean log H|_2
    (the error of the predicted pattern relative to the pattern's size)."""
    errs = []
    for c in range(3):
        a = torch.log(Hp[c].double().clamp_min(1e-30))
        b = torch.log(H[c].double().clamp_min(1e-30))
        errs.append(float((a - b).norm() / (b - b.mean()).norm()))
    return max(errs)
