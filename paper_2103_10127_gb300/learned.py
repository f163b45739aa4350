"""Learned per-subdomain damping: gather line-search labels from the method's
own runs, train the MLP, and install its predictions in a smoother.

Host orchestration only: features, labels, forward and backward passes and
the Adam updates all run in libravanka (see rav_patch_features,
rav_label_collection, rav_mlp_loss_grad, rav_adam_step, rav_set_learned_omega
in include/ravanka.h).  torch tensors provide device memory.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _capi, inputs
from ._capi import check

NPARAM = 4801
H, F = 64, 8


def _torch():
    import torch
    return torch


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def init_params(seed: int = inputs.BASE_SEED):
    """He-normal weights, zero biases, output bias so that omega starts at 0.5."""
    torch = _torch()
    z = inputs.normal(seed, NPARAM)
    P = np.zeros(NPARAM)
    o = 0
    P[o:o + H * F] = z[o:o + H * F] * math.sqrt(2.0 / F)
    o += H * F + H
    P[o:o + H * H] = z[o:o + H * H] * math.sqrt(2.0 / H)
    o += H * H + H
    P[o:o + H] = z[o:o + H] * math.sqrt(1.0 / H) * 0.1
    P[-1] = math.log(0.5)  # 1.5 sigmoid(b3) = 0.5
    return torch.from_numpy(P.astype(np.float32)).cuda()


def features(sm, level):
    torch = _torch()
    n = sm.mg.counts(level)["n_p"]
    out = torch.empty((n, F), dtype=torch.float32, device="cuda")
    check(_capi.load().rav_patch_features(sm.h, level, _p(out), _s()), "rav_patch_features")
    return out


def collect(mg, sm, x, b, cycles=3, nu=2):
    """Runs `cycles` V(nu,nu) cycles from x while accumulating line-search
    labels; returns (features, mean labels) over every smoothed level."""
    torch = _torch()
    lib = _capi.load()
    check(lib.rav_label_collection(sm.h, 1), "rav_label_collection")
    for _ in range(cycles):
        mg.vcycle(sm, x, b, nu, nu)
    Xs, ys = [], []
    for lev in range(1, mg.nlev):
        n = mg.counts(lev)["n_p"]
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        check(lib.rav_read_labels(sm.h, lev, _p(y), _s()), "rav_read_labels")
        Xs.append(features(sm, lev))
        ys.append(y)
    check(lib.rav_label_collection(sm.h, 0), "rav_label_collection")
    return torch.cat(Xs), torch.cat(ys)


def forward(params, X):
    torch = _torch()
    out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    check(_capi.load().rav_mlp_forward(_p(params), _p(X), X.shape[0], _p(out), _s()), "rav_mlp_forward")
    return out


def loss_grad(params, X, y):
    torch = _torch()
    n = X.shape[0]
    work = torch.empty(((n + 63) // 64) * (NPARAM + 1), dtype=torch.float32, device="cuda")
    g = torch.empty(NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    check(_capi.load().rav_mlp_loss_grad(_p(params), _p(X), _p(y), n, _p(g), _p(loss), _p(work), work.numel(),
                                         _s()), "rav_mlp_loss_grad")
    return loss, g


def train(X, y, steps=1500, lr=3e-3, seed=inputs.BASE_SEED, log_every=100):
    """Full-batch Adam on the mean squared error; returns (params, losses)."""
    torch = _torch()
    lib = _capi.load()
    P = init_params(seed)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    n = X.shape[0]
    work = torch.empty(((n + 63) // 64) * (NPARAM + 1), dtype=torch.float32, device="cuda")
    g = torch.empty(NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    losses = []
    for t in range(1, steps + 1):
        check(lib.rav_mlp_loss_grad(_p(P), _p(X), _p(y), n, _p(g), _p(loss), _p(work), work.numel(), _s()),
              "rav_mlp_loss_grad")
        check(lib.rav_adam_step(_p(P), _p(m), _p(v), _p(g), ctypes.c_float(lr), t, _s()), "rav_adam_step")
        if t == 1 or t % log_every == 0 or t == steps:
            losses.append((t, float(loss.item())))
    return P, losses


def install(sm, params, shrink=0.0):
    """omega_i of every subdomain of every level predicted by the MLP, shrunk
    toward the level's mean prediction by `shrink` (0: one weight per level)."""
    check(_capi.load().rav_set_learned_omega(sm.h, _p(params), float(shrink), _s()), "rav_set_learned_omega")


def reset(sm):
    check(_capi.load().rav_reset_omega(sm.h, _s()), "rav_reset_omega")
