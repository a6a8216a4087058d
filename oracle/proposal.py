"""FP64 reference of the learned-proposal network (test infrastructure: only
tests/ use it). Plain numpy, following the definition in
include/mp_proposal.h:

    x = scan / in_scale; h1 = relu(x W1 + b1); h2 = relu(h1 W2 + b2);
    h3 = relu(h2 W3 + b3); g = max over points of h3 (first maximum);
    h4 = relu(g W4 + b4); o = h4 W5 + b5 (416 = 32 x (1 + 6 + 6));
    log pi = a - logsumexp(a); s = 3 tanh(r / 3);
    NLL(y) = -log sum_c pi_c prod_d N(y_d; m_cd, exp(2 s_cd)), the yaw
    difference wrapped into (-pi, pi]; the batch loss is the mean.

The gradient is the chain rule written out layer by layer (ReLU passes where
its output is positive, max-pool to the first maximum). Its correctness is
pinned by central finite differences of `loss`, not by itself.

bf16=True gives the network the tensor-core form computes: the per-point
activations h1 and h2 and the weights W2, W3 of the forward products rounded
to BF16 (round to nearest, ties to even, from their FP32 values); the
backward pass uses the FP32 weights and the rounded activations, as the GPU
form does.
"""
from __future__ import annotations

import numpy as np

C1, C2, C3, C4, NOUT, NCOMP = 64, 128, 256, 256, 416, 32
LIM = 3.0
SHAPES = [(3, C1), (C1,), (C1, C2), (C2,), (C2, C3), (C3,), (C3, C4), (C4,), (C4, NOUT), (NOUT,)]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)


def unflatten(p):
    out, k = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(p[k:k + n], np.float64).reshape(s))
        k += n
    return out


def wrap_pi(a):
    a = a - 2 * np.pi * np.floor(a / (2 * np.pi) + 0.5)
    return np.where(a <= -np.pi, a + 2 * np.pi, a)


def bf16(a):
    """The nearest BF16 value (ties to even) of each value's FP32 rounding, as float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, scans, in_scale, bf16_form=False):
    """Layer outputs of B scans (B, P, 3)."""
    W1, b1, W2, b2, W3, b3, W4, b4, W5, b5 = unflatten(p)
    r = bf16 if bf16_form else (lambda a: a)
    x = np.asarray(scans, np.float64) / in_scale
    h1 = r(np.maximum(x @ W1 + b1, 0.0))
    h2 = r(np.maximum(h1 @ r(W2) + b2, 0.0))
    h3 = np.maximum(h2 @ r(W3) + b3, 0.0)
    gi = np.argmax(h3, axis=1)                        # first maximum
    g = np.take_along_axis(h3, gi[:, None, :], axis=1)[:, 0, :]
    h4 = np.maximum(g @ W4 + b4, 0.0)
    o = h4 @ W5 + b5
    return dict(x=x, h1=h1, h2=h2, h3=h3, g=g, gi=gi, h4=h4, o=o)


def _parts(o):
    a = o[:, :NCOMP]
    m = o[:, NCOMP:NCOMP + 6 * NCOMP].reshape(-1, NCOMP, 6)
    r = o[:, NCOMP + 6 * NCOMP:].reshape(-1, NCOMP, 6)
    return a, m, r


def nll(o, y):
    """Per-sample negative log-likelihood of targets y (B, 6) under o (B, 416)."""
    a, m, r = _parts(np.asarray(o, np.float64))
    y = np.asarray(y, np.float64)
    s = LIM * np.tanh(r / LIM)
    d = y[:, None, :] - m
    d[:, :, 3] = wrap_pi(d[:, :, 3])
    logpi = a - np.logaddexp.reduce(a, axis=1, keepdims=True)
    logn = np.sum(-0.5 * (d * np.exp(-s)) ** 2 - s, axis=2) - 3.0 * np.log(2 * np.pi)
    return -np.logaddexp.reduce(logpi + logn, axis=1)


def loss(p, scans, y, in_scale):
    return float(np.mean(nll(forward(p, scans, in_scale)["o"], y)))


def loss_grad(p, scans, y, in_scale, bf16_form=False):
    """(mean loss, gradient w.r.t. the flat parameter array); bf16_form: of the
    tensor-core form (see the module docstring)."""
    W1, b1, W2, b2, W3, b3, W4, b4, W5, b5 = unflatten(p)
    f = forward(p, scans, in_scale, bf16_form)
    o = f["o"]
    B = o.shape[0]
    a, m, r = _parts(o)
    y = np.asarray(y, np.float64)
    s = LIM * np.tanh(r / LIM)
    d = y[:, None, :] - m
    d[:, :, 3] = wrap_pi(d[:, :, 3])
    logpi = a - np.logaddexp.reduce(a, axis=1, keepdims=True)
    logn = np.sum(-0.5 * (d * np.exp(-s)) ** 2 - s, axis=2) - 3.0 * np.log(2 * np.pi)
    lj = logpi + logn
    L = -np.logaddexp.reduce(lj, axis=1)
    resp = np.exp(lj + L[:, None])
    pi = np.exp(logpi)
    iv = np.exp(-2 * s)
    dO = np.zeros_like(o)
    dO[:, :NCOMP] = pi - resp
    dO[:, NCOMP:NCOMP + 6 * NCOMP] = (-resp[:, :, None] * d * iv).reshape(B, -1)
    dr = resp[:, :, None] * (1 - d * d * iv) * (1 - np.tanh(r / LIM) ** 2)
    dO[:, NCOMP + 6 * NCOMP:] = dr.reshape(B, -1)
    dO /= B
    # head
    gW5 = f["h4"].T @ dO
    gb5 = dO.sum(0)
    dz4 = (dO @ W5.T) * (f["h4"] > 0)
    gW4 = f["g"].T @ dz4
    gb4 = dz4.sum(0)
    dg = (dz4 @ W4.T) * (f["g"] > 0)
    # max-pool: to the first maximum of each channel
    dz3 = np.zeros_like(f["h3"])
    bi, ci = np.meshgrid(np.arange(B), np.arange(C3), indexing="ij")
    dz3[bi, f["gi"], ci] = dg
    h2f = f["h2"].reshape(-1, C2)
    gW3 = h2f.T @ dz3.reshape(-1, C3)
    gb3 = dz3.reshape(-1, C3).sum(0)
    dz2 = (dz3 @ W3.T) * (f["h2"] > 0)
    gW2 = f["h1"].reshape(-1, C1).T @ dz2.reshape(-1, C2)
    gb2 = dz2.reshape(-1, C2).sum(0)
    dz1 = (dz2 @ W2.T) * (f["h1"] > 0)
    gW1 = f["x"].reshape(-1, 3).T @ dz1.reshape(-1, C1)
    gb1 = dz1.reshape(-1, C1).sum(0)
    grad = np.concatenate([t.ravel() for t in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4, gW5, gb5)])
    return float(L.mean()), grad


def init_params(seed=0):
    """He-normal weights, zero biases, last layer N(0, 0.01^2) (numpy draws)."""
    rng = np.random.default_rng(seed)
    out = []
    for i, s in enumerate(SHAPES):
        if len(s) == 1:
            out.append(np.zeros(s))
        elif i == 8:
            out.append(rng.normal(0, 0.01, s))
        else:
            out.append(rng.normal(0, np.sqrt(2.0 / s[0]), s))
    return np.concatenate([t.ravel() for t in out])
