"""Oracle of the learned blocking -- TEST INFRASTRUCTURE ONLY (imported by
``tests/`` only).  Plain numpy definitions, FP64:

  * ``features``  the 20 matrix statistics the model reads (definitions listed
                  below, written out row by row);
  * ``mlp_*``     the two-hidden-layer ReLU network, its loss (softmax cross
                  entropy on the block-size class + wreg x squared error on
                  the log resolution, averaged over the batch), the gradient
                  by the chain rule, and one Adam step.

Parity pins (tests/test_oracle_learn.py): closed forms of the features on a
tridiagonal and a diagonal matrix; the gradient against central finite
differences; the loss of a zero network (uniform softmax: log ncls).
"""
from __future__ import annotations

import math

import numpy as np

NFEATURES = 20
HIST_EDGES = [2, 4, 6, 8, 12, 20, 40]   # bins [0,2], [3,4], [5,6], [7,8], [9,12], [13,20], [21,40], [41,inf)


def features(n, rowptr, colind, val):
    """20 statistics of a CSR matrix:
    0 log10 n; 1-4 mean, variance, skewness (0 if variance 0), max of the row
    degree (stored entries, diagonal included); 5 log10 nnz; 6-8 mean and min
    of min(d_i, 10) and the fraction with d_i >= 1, d_i = |a_ii| / sum of the
    row's off-diagonal |a_ij| (10 without off-diagonals); 9 max |i-j| / n over
    stored entries; 10 mean |i-j| / n over off-diagonal entries; 11-18
    fractions of rows by off-diagonal count in the bins of HIST_EDGES; 19
    min(log10(max/min |a_ij|) over nonzero off-diagonal values, 6)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    deg = np.diff(rowptr).astype(np.float64)
    f = np.zeros(NFEATURES)
    f[0] = math.log10(n)
    mean = deg.sum() / n
    var = ((deg - mean) ** 2).sum() / n
    f[1], f[2] = mean, var
    f[3] = (((deg - mean) ** 3).sum() / n) / var ** 1.5 if var > 0 else 0.0
    f[4] = deg.max()
    f[5] = math.log10(max(int(rowptr[-1]), 1))
    dsum, dmin, ndom, band, prof, noff_tot = 0.0, 10.0, 0, 0.0, 0.0, 0
    vmax, vmin = 0.0, math.inf
    hist = np.zeros(8)
    for i in range(n):
        diag = off = 0.0
        noff = 0
        for e in range(rowptr[i], rowptr[i + 1]):
            j = int(colind[e])
            a = abs(float(val[e]))
            band = max(band, abs(j - i))
            if j == i:
                diag += a
            else:
                off += a
                noff += 1
                prof += abs(j - i)
                if a > 0:
                    vmax, vmin = max(vmax, a), min(vmin, a)
        d = min(diag / off, 10.0) if off > 0 else 10.0
        dsum += d
        dmin = min(dmin, d)
        ndom += d >= 1.0
        noff_tot += noff
        b = 0
        while b < 7 and noff > HIST_EDGES[b]:
            b += 1
        hist[b] += 1
    f[6], f[7], f[8] = dsum / n, dmin, ndom / n
    f[9] = band / n
    f[10] = prof / noff_tot / n if noff_tot else 0.0
    f[11:19] = hist / n
    f[19] = min(math.log10(vmax / vmin), 6.0) if vmax > 0 else 0.0
    return f


def mlp_offsets(nf, h, c):
    o = {}
    k = 0
    for name, size in (("W1", nf * h), ("b1", h), ("W2", h * h), ("b2", h), ("W3", h * (c + 1)), ("b3", c + 1)):
        o[name] = (k, size)
        k += size
    o["total"] = k
    return o


def mlp_unpack(p, nf, h, c):
    o = mlp_offsets(nf, h, c)
    g = lambda k: np.asarray(p[o[k][0]:o[k][0] + o[k][1]], dtype=np.float64)  # noqa: E731
    return (g("W1").reshape(nf, h), g("b1"), g("W2").reshape(h, h), g("b2"),
            g("W3").reshape(h, c + 1), g("b3"))


def mlp_forward(p, nf, h, c, X):
    """out = (relu(relu(X W1 + b1) W2 + b2)) W3 + b3; returns (out, h1, h2)."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(p, nf, h, c)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ W3 + b3, h1, h2


def mlp_loss(p, nf, h, c, X, ycls, yreg, wreg):
    z, _, _ = mlp_forward(p, nf, h, c, X)
    logits = z[:, :c]
    m = logits.max(axis=1, keepdims=True)
    lse = np.log(np.exp(logits - m).sum(axis=1)) + m[:, 0]
    ce = lse - logits[np.arange(len(ycls)), ycls]
    return float(np.mean(ce + wreg * (z[:, c] - yreg) ** 2))


def mlp_grad(p, nf, h, c, X, ycls, yreg, wreg):
    """Gradient of mlp_loss by the chain rule, flat in the parameter layout."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(p, nf, h, c)
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    z, h1, h2 = mlp_forward(p, nf, h, c, X)
    logits = z[:, :c]
    e = np.exp(logits - logits.max(axis=1, keepdims=True))
    prob = e / e.sum(axis=1, keepdims=True)
    dz = np.zeros_like(z)
    dz[:, :c] = prob
    dz[np.arange(B), ycls] -= 1.0
    dz[:, c] = 2.0 * wreg * (z[:, c] - yreg)
    dz /= B
    gW3, gb3 = h2.T @ dz, dz.sum(axis=0)
    d2 = (dz @ W3.T) * (h2 > 0)
    gW2, gb2 = h1.T @ d2, d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (h1 > 0)
    gW1, gb1 = X.T @ d1, d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam(p, g, m, v, lr, b1, b2, eps, step):
    """One bias-corrected Adam step (Kingma & Ba 2015); returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
