"""FP64 forward / backward of the kernel-surrogate MLP (oracle).

The network maps (fractional u offset, fractional v offset, residual w) to the 15 x 15
complex de-gridding tile of a visibility: x in R^3 -> 128 -> GELU -> 128 -> GELU -> 450
(real parts of the 225 taps, then imaginary parts), row a (along u) major.
Inputs are normalised as (2 phi_u - 1, 2 phi_v - 1, w_r / w_scale).

The CUDA path stores the weights in bf16 and feeds the tensor cores bf16 operands with
FP32 accumulation.  With `bf16=True` this oracle rounds the same quantities to bf16
(round to nearest even) at the same points - weights W1, W2, W3, the activations H1, H2
and the backward operands dY, dZ2 - and accumulates in FP64, so a comparison with the
GPU isolates its accumulation order.  GELU is the exact erf form.
This is test infrastructure.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

D_IN, D_H, D_OUT = 3, 128, 450


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int) -> dict:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (the usual default)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (o, i) in (("1", (D_H, D_IN)), ("2", (D_H, D_H)), ("3", (D_OUT, D_H))):
        a = 1.0 / math.sqrt(i)
        p["W" + name] = rng.uniform(-a, a, (o, i))
        p["b" + name] = rng.uniform(-a, a, o)
    return p


def forward(p: dict, x: np.ndarray, bf: bool = False) -> dict:
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    z1 = x @ W1.T + p["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ W2.T + p["b2"]
    h2 = r(gelu(z2))
    y = h2 @ W3.T + p["b3"]
    return dict(z1=z1, h1=h1, z2=z2, h2=h2, y=y, W1=W1, W2=W2, W3=W3)


def loss_and_grads(p: dict, x: np.ndarray, t: np.ndarray, bf: bool = False):
    """Mean squared error over batch and outputs, and its gradients."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    f = forward(p, x, bf)
    B = x.shape[0]
    res = f["y"] - t
    loss = float(np.mean(res * res))
    dy = 2.0 * res / (B * D_OUT)
    dyr = r(dy)
    g = {}
    g["W3"] = dyr.T @ f["h2"]
    g["b3"] = dy.sum(axis=0)
    dh2 = dyr @ f["W3"]
    dz2 = dh2 * gelu_grad(f["z2"])
    dz2r = r(dz2)
    g["W2"] = dz2r.T @ f["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2r @ f["W2"]
    dz1 = dh1 * gelu_grad(f["z1"])
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def inputs(phi_u, phi_v, w_r, w_scale: float) -> np.ndarray:
    return np.stack([2.0 * np.asarray(phi_u) - 1.0, 2.0 * np.asarray(phi_v) - 1.0,
                     np.asarray(w_r) / w_scale], axis=1)


def targets(tiles) -> np.ndarray:
    """Stack 15 x 15 complex tiles as 450 reals (real parts, then imaginary parts)."""
    T = np.stack(tiles).reshape(len(tiles), 225)
    return np.concatenate([T.real, T.imag], axis=1)
