"""Coupling-flow proposal oracle -- test infrastructure only.

A plain numpy FP64 restatement of the learned proposal that can stand in for the VEGAS grid.
The flow follows neural importance sampling (Mueller, McWilliams, Rousselle, Gross, Novak,
"Neural Importance Sampling", ACM TOG 2019): a stack of coupling layers on [0,1]^d whose
transformed coordinates go through piecewise-quadratic CDFs. An MLP computes the CDFs from the
untouched coordinates.

Definitions (the GPU library implements the same ones; nothing is shared):
  - Layer l splits the axes into A_l (kept) and B_l (transformed):
      l mod 4 == 0: A = first floor(d/2) axes, B = the rest;
      l mod 4 == 1: the same halves, swapped;
      l mod 4 == 2: A = even axes, B = odd axes;
      l mod 4 == 3: swapped.
  - MLP of layer l: a = h[A]; r1 = relu(W1 a + b1); r2 = relu(W2 r1 + b2); o = W3 r2 + b3. W1 is
    H x |A|, W2 H x H, W3 (|B| (2K+1)) x H. Output slot s (axis B[s]) is
    o[s(2K+1) : s(2K+1)+K] = unnormalised bin widths, then K+1 unnormalised edge values.
  - Piecewise-quadratic CDF of one axis (K bins):
      widths W = softmax(widths);
      edge pdf values V_k = exp(v_k) / Z with Z = sum_k (e^{v_k} + e^{v_{k+1}})/2 W_k;
      the pdf is linear inside each bin, so it integrates to one;
      at x in bin b (left edge X_b, delta = x - X_b):
        CDF(x) = sum_{k<b} (V_k + V_{k+1})/2 W_k + delta V_b + delta^2 (V_{b+1} - V_b)/(2 W_b);
        pdf(x) = V_b + delta (V_{b+1} - V_b)/W_b.
  - Density direction x -> z: h_0 = x, h_l = layer_l(h_{l-1}), z = h_L.
    log q(x) = sum_l sum_{j in B_l} log pdf_{l,j}.
  - Sampling direction z -> x: invert the layers in reverse order. Each transformed coordinate
    solves the bin's quadratic in the cancellation-free form
    delta = 2 (y - Y_b) / (V_b + sqrt(V_b^2 + 2 (y - Y_b)(V_{b+1} - V_b)/W_b)).
  - bf16=True rounds every MLP matmul operand (weights and inputs) to bfloat16, round to
    nearest even, with products summed in FP64. This is the precision the GPU MLP computes in
    (bf16 operands, wide accumulation).
  - Training losses on samples x_i with weights w_i (normalised to sum 1):
      variance (chi^2): L = sum_i w_i / q(x_i), with w_i = f_i^2 J_i from the VEGAS sampler;
        this is the proposal's second moment, E[(f/q)^2];
      KL: L = -sum_i w_i log q(x_i), with w_i = |f_i| J_i.
    Gradients here are central finite differences of these losses (FP64, no bf16).
"""
from __future__ import annotations

import numpy as np


def masks(d: int, layers: int):
    out = []
    h = d // 2
    for l in range(layers):
        kind = l % 4
        if kind in (0, 1):
            A, B = list(range(h)), list(range(h, d))
            if kind == 1:
                A, B = B, A
        else:
            A, B = list(range(0, d, 2)), list(range(1, d, 2))
            if kind == 3:
                A, B = B, A
        out.append((np.array(A, dtype=int), np.array(B, dtype=int)))
    return out


def layer_shapes(d: int, layers: int, hidden: int, bins: int):
    shapes = []
    for A, B in masks(d, layers):
        nout = len(B) * (2 * bins + 1)
        shapes.append([("W1", (hidden, len(A))), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
                       ("W3", (nout, hidden)), ("b3", (nout,))])
    return shapes


def n_params(d, layers, hidden, bins):
    return sum(int(np.prod(s)) for L in layer_shapes(d, layers, hidden, bins) for _, s in L)


def unpack(params, d, layers, hidden, bins):
    params = np.asarray(params, dtype=np.float64)
    out, pos = [], 0
    for L in layer_shapes(d, layers, hidden, bins):
        lay = {}
        for name, s in L:
            n = int(np.prod(s))
            lay[name] = params[pos:pos + n].reshape(s)
            pos += n
        out.append(lay)
    assert pos == params.size, (pos, params.size)
    return out


def bf16(a):
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp(a, lay, use_bf16=False):
    rnd = bf16 if use_bf16 else (lambda v: v)
    r1 = np.maximum(rnd(a) @ rnd(lay["W1"]).T + lay["b1"], 0.0)
    r2 = np.maximum(rnd(r1) @ rnd(lay["W2"]).T + lay["b2"], 0.0)
    return rnd(r2) @ rnd(lay["W3"]).T + lay["b3"]


def _widths_values(raw, bins):
    """raw: (..., 2K+1) -> normalised widths W (..., K), edge values V (..., K+1)."""
    wr = raw[..., :bins]
    vr = raw[..., bins:]
    W = np.exp(wr - wr.max(axis=-1, keepdims=True))
    W = W / W.sum(axis=-1, keepdims=True)
    E = np.exp(vr - vr.max(axis=-1, keepdims=True))
    Z = np.sum((E[..., :-1] + E[..., 1:]) / 2.0 * W, axis=-1, keepdims=True)
    return W, E / Z


def pq_cdf(x, raw, bins):
    """Piecewise-quadratic CDF y(x) and pdf q(x) for elementwise x in [0, 1]."""
    W, V = _widths_values(raw, bins)
    edges = np.concatenate([np.zeros(W.shape[:-1] + (1,)), np.cumsum(W, axis=-1)], axis=-1)
    b = np.sum(edges[..., 1:-1] <= x[..., None], axis=-1)          # bin index, 0..K-1
    take = lambda a, idx: np.take_along_axis(a, idx[..., None], axis=-1)[..., 0]
    Xb, Wb = take(edges, b), take(W, b)
    Vb, Vb1 = take(V, b), take(V, b + 1)
    mass = (V[..., :-1] + V[..., 1:]) / 2.0 * W
    Ycum = np.concatenate([np.zeros(W.shape[:-1] + (1,)), np.cumsum(mass, axis=-1)], axis=-1)
    delta = x - Xb
    y = take(Ycum, b) + delta * Vb + delta * delta * (Vb1 - Vb) / (2.0 * Wb)
    q = Vb + delta * (Vb1 - Vb) / Wb
    return y, q


def pq_inverse(y, raw, bins):
    """Inverse of pq_cdf: x(y) and the pdf at x."""
    W, V = _widths_values(raw, bins)
    edges = np.concatenate([np.zeros(W.shape[:-1] + (1,)), np.cumsum(W, axis=-1)], axis=-1)
    mass = (V[..., :-1] + V[..., 1:]) / 2.0 * W
    Ycum = np.concatenate([np.zeros(W.shape[:-1] + (1,)), np.cumsum(mass, axis=-1)], axis=-1)
    b = np.sum(Ycum[..., 1:-1] <= y[..., None], axis=-1)
    take = lambda a, idx: np.take_along_axis(a, idx[..., None], axis=-1)[..., 0]
    Xb, Wb, Vb, Vb1 = take(edges, b), take(W, b), take(V, b), take(V, b + 1)
    r = np.maximum(y - take(Ycum, b), 0.0)
    delta = 2.0 * r / (Vb + np.sqrt(np.maximum(Vb * Vb + 2.0 * r * (Vb1 - Vb) / Wb, 0.0)))
    delta = np.minimum(delta, Wb)
    x = Xb + delta
    q = Vb + delta * (Vb1 - Vb) / Wb
    return x, q


def forward(params, x, d, layers, hidden, bins, use_bf16=False):
    """x (n x d) -> z (n x d), log q(x) (n)."""
    lays = unpack(params, d, layers, hidden, bins)
    h = np.array(x, dtype=np.float64, copy=True)
    logq = np.zeros(h.shape[0])
    for (A, B), lay in zip(masks(d, layers), lays):
        o = mlp(h[:, A], lay, use_bf16)
        new = h.copy()
        for s, j in enumerate(B):
            raw = o[:, s * (2 * bins + 1):(s + 1) * (2 * bins + 1)]
            y, q = pq_cdf(h[:, j], raw, bins)
            new[:, j] = y
            logq += np.log(q)
        h = new
    return h, logq


def inverse(params, z, d, layers, hidden, bins, use_bf16=False):
    """z (n x d) -> x (n x d), log q(x) (n)."""
    lays = unpack(params, d, layers, hidden, bins)
    h = np.array(z, dtype=np.float64, copy=True)
    logq = np.zeros(h.shape[0])
    for (A, B), lay in reversed(list(zip(masks(d, layers), lays))):
        o = mlp(h[:, A], lay, use_bf16)
        new = h.copy()
        for s, j in enumerate(B):
            raw = o[:, s * (2 * bins + 1):(s + 1) * (2 * bins + 1)]
            xj, q = pq_inverse(h[:, j], raw, bins)
            new[:, j] = xj
            logq += np.log(q)
        h = new
    return h, logq


def loss(params, x, w, d, layers, hidden, bins, kind="variance", use_bf16=False):
    w = np.asarray(w, dtype=np.float64)
    w = w / w.sum()
    _, logq = forward(params, x, d, layers, hidden, bins, use_bf16)
    if kind == "variance":
        return float(np.sum(w * np.exp(-logq)))
    return float(-np.sum(w * logq))


def grad_fd(params, x, w, d, layers, hidden, bins, kind="variance", eps=1e-6, idx=None):
    """Central finite differences of the loss with respect to params[idx] (all if None)."""
    params = np.array(params, dtype=np.float64, copy=True)
    idx = np.arange(params.size) if idx is None else np.asarray(idx)
    g = np.zeros(len(idx))
    for n, i in enumerate(idx):
        p0 = params[i]
        params[i] = p0 + eps
        lp = loss(params, x, w, d, layers, hidden, bins, kind)
        params[i] = p0 - eps
        lm = loss(params, x, w, d, layers, hidden, bins, kind)
        params[i] = p0
        g[n] = (lp - lm) / (2 * eps)
    return g


def grad_x_fd(params, x, d, layers, hidden, bins, eps=1e-7):
    """Jacobian dz/dx (n x d x d) by central differences (for the log-det pin)."""
    n = x.shape[0]
    Jm = np.zeros((n, d, d))
    for k in range(d):
        xp = x.copy()
        xm = x.copy()
        xp[:, k] += eps
        xm[:, k] -= eps
        zp, _ = forward(params, xp, d, layers, hidden, bins)
        zm, _ = forward(params, xm, d, layers, hidden, bins)
        Jm[:, :, k] = (zp - zm) / (2 * eps)
    return Jm
