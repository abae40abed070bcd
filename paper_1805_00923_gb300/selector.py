"""Learned direction selector (not part of the paper): data, training, weights.

The selector is a 16-64-64-3 ReLU perceptron that predicts, from 16 features
of a traversal level (frontier size, frontier out-degree sum, unvisited
counts, graph size and skew, level, previous direction), the log-time of
SparsePush, DensePush and DensePull; the fused frontier-statistics kernel runs
it and takes the argmin.  Training data are per-level timings of all three
directions produced by gi_selector_profile; training runs the library's
forward/backward/Adam kernels (gi_mlp_*).  Everything here is orchestration
over the C ABI.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _C, _stream, _vp, check, schedule, selector_load

N_PARAM = 5443
D_IN, D_OUT = 16, 3
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.npz")
DIR_NAMES = ("sparse_push", "dense_push", "dense_pull")


def profile(g, kernel_id: int, src: int, sched=None, cap: int = 16384, stream=None):
    """(features[L,16], times_ms[L,3]) of one BFS/SSSP run (gi_selector_profile)."""
    feats = np.zeros((cap, D_IN), np.float32)
    times = np.zeros((cap, D_OUT), np.float32)
    lv = ctypes.c_int32()
    s = sched if sched is not None else schedule()
    check(_C.gi_selector_profile(g.handle, int(kernel_id), int(src), ctypes.byref(s), cap, _vp(feats), _vp(times),
                                 ctypes.byref(lv), _stream(stream)))
    return feats[:lv.value].copy(), times[:lv.value].copy()


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialised weights, zero biases, in the gi_selector_load layout."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2 / 16), 64 * 16), np.zeros(64), rng.normal(0, np.sqrt(2 / 64), 64 * 64),
             np.zeros(64), rng.normal(0, np.sqrt(1 / 64), 3 * 64), np.zeros(3)]
    return np.concatenate(parts).astype(np.float32)


def loss_grad(params: torch.Tensor, X: torch.Tensor, T: torch.Tensor, M: torch.Tensor, stream=None):
    """Masked MSE and its gradient (gi_mlp_loss_grad); all tensors on the GPU."""
    grad = torch.empty(N_PARAM, dtype=torch.float32, device=params.device)
    loss = torch.empty(2, dtype=torch.float32, device=params.device)
    check(_C.gi_mlp_loss_grad(_vp(params), _vp(X), _vp(T), _vp(M), X.shape[0], _vp(grad), _vp(loss),
                              _stream(stream)))
    return loss, grad


def forward(params: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
    Y = torch.empty((X.shape[0], D_OUT), dtype=torch.float32, device=params.device)
    check(_C.gi_mlp_forward(_vp(params), _vp(X), X.shape[0], _vp(Y), _stream(stream)))
    return Y


def adam(params, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    check(_C.gi_mlp_adam(_vp(params), _vp(grad), _vp(m), _vp(v), int(step), float(lr), float(b1), float(b2),
                         float(eps), _stream(stream)))


def normaliser(X: np.ndarray):
    mean = X.mean(axis=0).astype(np.float32)
    std = X.std(axis=0)
    inv_std = (1.0 / np.maximum(std, 1e-3)).astype(np.float32)
    return mean, inv_std


def targets(times_ms: np.ndarray) -> np.ndarray:
    """Natural log of microseconds (what the network predicts)."""
    return np.log(np.maximum(times_ms, 1e-4) * 1e3).astype(np.float32)


def train(X: np.ndarray, T: np.ndarray, M: np.ndarray | None = None, steps: int = 3000, lr: float = 3e-3,
          seed: int = 0, lr_decay: float = 0.999):
    """Full-batch Adam on the GPU.  X raw features, T log-times; returns (params, mean, inv_std, losses)."""
    mean, inv_std = normaliser(X)
    Xn = torch.from_numpy(((X - mean) * inv_std).astype(np.float32)).cuda()
    Tt = torch.from_numpy(T.astype(np.float32)).cuda()
    Mt = torch.from_numpy((np.ones_like(T) if M is None else M).astype(np.float32)).cuda()
    p = torch.from_numpy(init_params(seed)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    losses = []
    for t in range(1, steps + 1):
        loss, grad = loss_grad(p, Xn, Tt, Mt)
        adam(p, grad, m, v, t, lr=lr * (lr_decay ** t))
        if t % 100 == 0 or t == 1:
            losses.append(float(loss[0]))
    return p.cpu().numpy(), mean, inv_std, losses


# |F| + m_f below m / SELECTOR_GATE: the library pushes without consulting
# the network (the same constant as the decision kernels)
SELECTOR_GATE = 200


def gated(X: np.ndarray) -> np.ndarray:
    """Rows of raw features X whose frontier the library pushes without an
    evaluation (features 0, 1, 5 are log2(1 + |F|), log2(1 + m_f), log2(1 + m))."""
    nf = np.rint(np.exp2(X[:, 0].astype(np.float64)) - 1.0)
    mf = np.rint(np.exp2(X[:, 1].astype(np.float64)) - 1.0)
    m = np.rint(np.exp2(X[:, 5].astype(np.float64)) - 1.0)
    return (nf + mf) * SELECTOR_GATE < m


def choose(params: np.ndarray, mean: np.ndarray, inv_std: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Directions (0 SparsePush, 1 DensePush, 2 DensePull) the learned policy
    picks for raw features X: the network's, except SparsePush on gated rows."""
    if X.shape[0] == 0:
        return np.zeros(0, np.int64)
    p = torch.from_numpy(params.astype(np.float32)).cuda()
    Xn = torch.from_numpy(((X - mean) * inv_std).astype(np.float32)).cuda()
    k = forward(p, Xn).argmin(dim=1).cpu().numpy()
    return np.where(gated(X), 0, k)


def save(path: str, params, mean, inv_std, **meta):
    np.savez(path, params=params.astype(np.float32), mean=mean.astype(np.float32),
             inv_std=inv_std.astype(np.float32), **{k: np.asarray(v) for k, v in meta.items()})


def load(path: str = WEIGHTS_PATH):
    z = np.load(path)
    return z["params"], z["mean"], z["inv_std"]


def install(path: str = WEIGHTS_PATH):
    """Load trained weights into the library (used by GI_DIR_LEARNED)."""
    params, mean, inv_std = load(path)
    selector_load(params, mean, inv_std)
    return params, mean, inv_std
