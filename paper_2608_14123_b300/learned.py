"""Learned tensor-product surrogate: training and application through the
C ABI (the network's forward, backward and Adam kernels live in csrc/mlp.cu).

This module only marshals arguments: seeded Glorot initialization of the flat
parameter vector, device buffers, and calls of dgfas_mlp_train /
dgfas_mlp_forward / dgfas_mlp_grad / dgfas_learned_surrogate.  The training
pairs (normalized corners -> log widths and log scalings of the best-fit
Kronecker sum) are inputs supplied by the caller.
"""
import ctypes

import numpy as np

from . import dgfas

SIZES = (24, 64, 64, 6)


def param_count():
    return int(dgfas.load().dgfas_mlp_param_count())


def init_params(seed):
    """Glorot-uniform weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(SIZES) - 1):
        r, c = SIZES[i + 1], SIZES[i]
        lim = np.sqrt(6.0 / (r + c))
        parts += [rng.uniform(-lim, lim, r * c), np.zeros(r)]
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == param_count()
    return th


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def forward(params, X):
    import torch
    out = torch.empty((X.shape[0], 6), dtype=torch.float32, device="cuda")
    dgfas._check(dgfas.load().dgfas_mlp_forward(_p(params), _p(X), X.shape[0], _p(out), _stream()),
                 "mlp_forward")
    return out


def inputs(corners):
    """The network's inputs [n, 24] (device FP32) of elements given by their
    corners [n, 8, 3] (host or device FP64), computed by the library."""
    import torch
    cd = torch.as_tensor(corners, dtype=torch.float64).cuda().contiguous()
    n = cd.shape[0]
    X = torch.empty((n, 24), dtype=torch.float32, device="cuda")
    dgfas._check(dgfas.load().dgfas_mlp_inputs(_p(cd), n, _p(X), _stream()), "mlp_inputs")
    return X


def grad(params, X, Y):
    import torch
    g = torch.empty_like(params)
    dgfas._check(dgfas.load().dgfas_mlp_grad(_p(params), _p(X), _p(Y), X.shape[0], _p(g), _stream()),
                 "mlp_grad")
    return g


def train(X, Y, epochs=200, batch=256, lr=1e-3, seed=1, params=None):
    """Trains on device tensors X [n, 24], Y [n, 6] (FP32); returns (params,
    per-epoch full-data loss)."""
    import torch
    th = torch.from_numpy(init_params(seed)).cuda() if params is None else params
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    loss = np.zeros(epochs, dtype=np.float32)
    dgfas._check(dgfas.load().dgfas_mlp_train(
        _p(th), _p(m), _p(v), _p(X), _p(Y), X.shape[0], epochs, batch, ctypes.c_float(lr),
        ctypes.c_ulonglong(seed), 0, loss.ctypes.data_as(ctypes.c_void_p), _stream()), "mlp_train")
    return th, loss
