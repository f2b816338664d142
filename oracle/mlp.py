"""FP64 reference of the NCI surrogate network's forward pass and gradients.

TEST INFRASTRUCTURE ONLY.  The network: n_in -> width x depth (tanh) -> 1
(linear), mean-squared-error loss.  With bf16=True the tensor-core operands
are rounded to BF16 (round to nearest even) at the same points as the GPU
kernels: the network input, the weights, the hidden activations and the
backpropagated dH; everything else is exact FP64.  Parameters are laid out
per layer as W[out][in] then b[out].
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(n_in, width, depth):
    dims = [n_in] + [width] * depth + [1]
    return [(dims[i + 1], dims[i]) for i in range(depth + 1)]


def unpack(params, n_in, width, depth):
    out, off = [], 0
    for fo, fi in layer_shapes(n_in, width, depth):
        W = params[off:off + fo * fi].reshape(fo, fi).astype(np.float64)
        off += fo * fi
        b = params[off:off + fo].astype(np.float64)
        off += fo
        out.append((W, b))
    return out


def num_params(n_in, width, depth):
    return sum(fo * fi + fo for fo, fi in layer_shapes(n_in, width, depth))


def forward(params, x, n_in, width, depth, rnd=True):
    q = bf16 if rnd else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params, n_in, width, depth)
    X = [q(x)]
    H = []
    for l, (W, b) in enumerate(layers):
        h = X[-1] @ q(W).T + b
        H.append(h)
        if l < len(layers) - 1:
            X.append(q(np.tanh(h)))
    return H[-1][:, 0], X, H


def gradients(params, x, t, n_in, width, depth, rnd=True):
    q = bf16 if rnd else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params, n_in, width, depth)
    y, X, H = forward(params, x, n_in, width, depth, rnd)
    B = x.shape[0]
    d = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(d * d))
    dH = (2.0 * d / B)[:, None]
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        dHq = q(dH)
        gW = dHq.T @ X[l]
        gb = dH.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dX = dHq @ q(W)
            th = np.tanh(H[l - 1])
            dH = dX * (1.0 - th * th)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in grads])
    return flat, loss
