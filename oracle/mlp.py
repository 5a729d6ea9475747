"""FP64 reference of the rho-policy MLP.  TEST INFRASTRUCTURE.

The paper has no learned component; this network (3 layers, width 64,
inputs: log ||r_prim||_inf, log ||r_dual||_inf, log rho and the PCG iteration
count; output: a log-rho multiplier and a log-factor on the PCG tolerance
weight) is an addition.  Parity unpinned against the paper; pinned instead
by central finite differences (tests) and used as the reference for the GPU
BF16 kernels.

    h1 = relu(W1 x + b1)      W1: 64 x 4
    h2 = relu(W2 h1 + b2)     W2: 64 x 64
    o  = W3 h2 + b3           W3: 2 x 64
    loss = sum_k w_k (o_k - t_k)^2 / (2 B)   (masked mean squared error)

Adam (Kingma & Ba 2015) with bias correction updates the parameters.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 4, 64, 2
PARAM_SHAPES = {"W1": (N_HID, N_IN), "b1": (N_HID,), "W2": (N_HID, N_HID), "b2": (N_HID,),
                "W3": (N_OUT, N_HID), "b3": (N_OUT,)}


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))
    r = ((u + bias) & np.uint64(0xFFFF0000)).astype(np.uint32)
    nan = np.isnan(f)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out.reshape(np.shape(a))


def forward(params: dict, X: np.ndarray):
    X = np.asarray(X, np.float64)
    a1 = X @ params["W1"].T + params["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(a2, 0.0)
    out = h2 @ params["W3"].T + params["b3"]
    return out, (X, a1, h1, a2, h2)


def loss_and_grad_out(out, target, weight):
    """Masked MSE: sum_k w_k (o_k - t_k)^2 / (2B); returns (loss, dL/do)."""
    B = out.shape[0]
    diff = (out - target) * weight
    loss = float(np.sum(diff * (out - target)) / (2.0 * B))
    return loss, diff / B


def backward(params: dict, cache, dout):
    X, a1, h1, a2, h2 = cache
    g = {}
    g["W3"] = dout.T @ h2
    g["b3"] = dout.sum(axis=0)
    dh2 = dout @ params["W3"]
    da2 = dh2 * (a2 > 0.0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ params["W2"]
    da1 = dh1 * (a1 > 0.0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return g


def loss_fn(params, X, target, weight) -> float:
    out, _ = forward(params, X)
    return loss_and_grad_out(out, target, weight)[0]


def grads(params, X, target, weight):
    out, cache = forward(params, X)
    loss, dout = loss_and_grad_out(out, target, weight)
    return loss, backward(params, cache, dout)


def adam_step(params, g, state, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); state holds first and second moments."""
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = b1 * m + (1.0 - b1) * g[k]
        v[...] = b2 * v + (1.0 - b2) * g[k] * g[k]
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


def grads_bf16(params: dict, X: np.ndarray, target, weight):
    """The forward and backward pass with the rounding points of the BF16
    kernels: weights, inputs, hidden activations and the back-propagated
    signals (dL/do, and the two pre-activation gradients) rounded to BF16;
    biases unrounded; everything else exact.  X is the normalised input."""
    W1, W2, W3 = (bf16_round(params[k]) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = params["b1"], params["b2"], params["b3"]
    x = bf16_round(X)
    a1 = x @ W1.T + b1
    h1 = bf16_round(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + b2
    h2 = bf16_round(np.maximum(a2, 0.0))
    out = h2 @ W3.T + b3
    loss, dout = loss_and_grad_out(out, target, weight)
    dout = bf16_round(dout)
    g = {"W3": dout.T @ h2, "b3": dout.sum(axis=0)}
    d2 = bf16_round((dout @ W3) * (a2 > 0.0))
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = bf16_round((d2 @ W2) * (a1 > 0.0))
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return loss, g, out


def forward_bf16(params: dict, X: np.ndarray):
    """Inference with the BF16 rounding points of the device code."""
    W1, W2, W3 = (bf16_round(params[k]) for k in ("W1", "W2", "W3"))
    x = bf16_round(X)
    h1 = bf16_round(np.maximum(x @ W1.T + params["b1"], 0.0))
    h2 = bf16_round(np.maximum(h1 @ W2.T + params["b2"], 0.0))
    return h2 @ W3.T + params["b3"]
