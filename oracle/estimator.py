"""FP64 oracle of the connectivity estimator -- TEST INFRASTRUCTURE (see the
package docstring for who may import it).

The paper names statistical correlation of the activity of two cells as the
common way to map functional connections (Sec. 1) and proposes the mapping
problem on its test networks (Sec. 3.5, Sec. 4).  This build scores two
estimators of "is there an edge i -> j" on candidate pairs of a simulated net:

* plain: the peak normalised cross-correlation over 32 lags of the observed
  traces, starting at the shortest geometric delay d / v_max;
* learned: an MLP 33 -> 256 -> 256 -> 1 on those 32 correlations plus d / r_c,
  trained on nets whose ground-truth topology is known (BCE loss, AdamW).

Everything here is plain numpy in FP64.  The MLP oracle mirrors the points where
the CUDA path rounds to BF16 (inputs, weight copies, hidden activations and
backward activations); with quantise=False it is the exact FP64 network, which the
finite-difference checks pin.
"""
from __future__ import annotations

import numpy as np
from scipy import stats

V_MAX_MM_PER_MS = 0.5   # the fastest conduction speed of the generated nets (0.5 m/s)
N_LAGS = 32


# --------------------------------------------------------------------------- features
def pearson(a: np.ndarray, b: np.ndarray) -> float:
    """Pearson correlation of two equal-length segments (0 if either is constant)."""
    a = a - a.mean()
    b = b - b.mean()
    den = np.sqrt((a * a).sum() * (b * b).sum())
    return float((a * b).sum() / den) if den > 0.0 else 0.0


def first_lag(dist: np.ndarray, sample_ms: float = 1.0) -> np.ndarray:
    """Shortest geometric delay in whole samples: floor(d / v_max / sample)."""
    return np.floor(dist / V_MAX_MM_PER_MS / sample_ms).astype(np.int64)


def ncc_features(Y: np.ndarray, pos: np.ndarray, src: np.ndarray, dst: np.ndarray, radius: float,
                 n_lags: int = N_LAGS, sample_ms: float = 1.0):
    """Features of candidate pairs i -> j of one net.

    Y [T, N] observed traces.  For lag l = l0 + k, k < n_lags, with l0 the first
    geometric lag, f_k = Pearson(y_i[0 : T - l], y_j[l : T]) on the overlap (each
    segment centred on its own mean); f_{n_lags} = d / radius.  Returns the
    features [P, n_lags + 1] and the plain score max_k f_k.
    """
    Y = np.asarray(Y, np.float64)
    T = Y.shape[0]
    d = np.sqrt(((pos[src] - pos[dst]) ** 2).sum(1))
    l0 = first_lag(d, sample_ms)
    P = src.shape[0]
    F = np.zeros((P, n_lags + 1))
    for base in np.unique(l0):
        sel = np.nonzero(l0 == base)[0]
        for k in range(n_lags):
            lag = int(base) + k
            n = T - lag
            if n < 2:
                continue
            A = Y[0:n, src[sel]]
            B = Y[lag:T, dst[sel]]
            A = A - A.mean(0)
            B = B - B.mean(0)
            num = (A * B).sum(0)
            den = np.sqrt((A * A).sum(0) * (B * B).sum(0))
            F[sel, k] = np.where(den > 0.0, num / np.where(den > 0.0, den, 1.0), 0.0)
    F[:, n_lags] = d / radius
    return F, F[:, :n_lags].max(1)


# --------------------------------------------------------------------------- BF16
def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


# --------------------------------------------------------------------------- MLP
def mlp_forward(params: dict, X: np.ndarray, quantise: bool = True):
    """Forward pass; returns the probability p [B] and the cache for backward.

    z1 = X W1 + b1, h1 = relu(z1); z2 = h1 W2 + b2, h2 = relu(z2);
    z = h2 . w3 + b3, p = sigmoid(z).  With quantise, X, W1, W2 and h1 are rounded
    to BF16 where the CUDA path stores them in BF16."""
    q = bf16 if quantise else (lambda a: np.asarray(a, np.float64))
    Xq = q(X)
    W1 = q(params["W1"])
    W2 = q(params["W2"])
    b1 = np.asarray(params["b1"], np.float64)
    b2 = np.asarray(params["b2"], np.float64)
    w3 = np.asarray(params["w3"], np.float64)
    b3 = float(np.asarray(params["b3"], np.float64).reshape(-1)[0])
    z1 = Xq @ W1 + b1
    h1 = q(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    z = h2 @ w3 + b3
    p = 1.0 / (1.0 + np.exp(-z))
    return p, dict(X=Xq, W1=W1, W2=W2, z1=z1, h1=h1, z2=z2, h2=h2, z=z, w3=w3)


def bce(p: np.ndarray, y: np.ndarray) -> float:
    """Mean binary cross-entropy."""
    eps = 1e-12
    return float(-np.mean(y * np.log(p + eps) + (1.0 - y) * np.log(1.0 - p + eps)))


def mlp_backward(params: dict, cache: dict, p: np.ndarray, y: np.ndarray, quantise: bool = True) -> dict:
    """Gradients of the mean BCE with respect to every parameter (chain rule of
    the forward pass; dL/dz = (p - y) / B for a sigmoid output)."""
    q = bf16 if quantise else (lambda a: np.asarray(a, np.float64))
    B = p.shape[0]
    dz = (p - np.asarray(y, np.float64)) / B
    g = {}
    g["w3"] = cache["h2"].T @ dz
    g["b3"] = np.array([dz.sum()])
    dh2 = np.outer(dz, cache["w3"]) * (cache["z2"] > 0.0)
    g["b2"] = dh2.sum(0)
    dh2q = q(dh2)
    g["W2"] = cache["h1"].T @ dh2q
    dh1 = (dh2q @ cache["W2"].T) * (cache["h1"] > 0.0)  # the stored activation gates the gradient
    g["b1"] = dh1.sum(0)
    dh1q = q(dh1)
    g["W1"] = cache["X"].T @ dh1q
    return g


def adamw(params: dict, grads: dict, state: dict, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
          eps: float = 1e-8, weight_decay: float = 0.0) -> dict:
    """One AdamW step (Loshchilov & Hutter: decoupled weight decay) on FP64 copies."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = {}
    for k, w in params.items():
        g = np.asarray(grads[k], np.float64)
        m = state.get("m_" + k, np.zeros_like(g))
        v = state.get("v_" + k, np.zeros_like(g))
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        state["m_" + k] = m
        state["v_" + k] = v
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        w = np.asarray(w, np.float64) * (1.0 - lr * weight_decay)
        out[k] = w - lr * mhat / (np.sqrt(vhat) + eps)
    return out


# --------------------------------------------------------------------------- scoring
def auroc(scores: np.ndarray, labels: np.ndarray) -> float:
    """Area under the ROC curve by the Mann-Whitney U statistic with mid-ranks:
    AUROC = (R_pos - n_pos (n_pos + 1) / 2) / (n_pos n_neg)."""
    labels = np.asarray(labels).astype(bool)
    n_pos = int(labels.sum())
    n_neg = labels.size - n_pos
    if n_pos == 0 or n_neg == 0:
        return float("nan")
    r = stats.rankdata(np.asarray(scores, np.float64))
    return float((r[labels].sum() - n_pos * (n_pos + 1) / 2.0) / (n_pos * n_neg))


def f1_at(scores: np.ndarray, labels: np.ndarray, threshold: float) -> float:
    """F1 of the rule "edge iff score >= threshold"."""
    labels = np.asarray(labels).astype(bool)
    pred = np.asarray(scores) >= threshold
    tp = int((pred & labels).sum())
    fp = int((pred & ~labels).sum())
    fn = int((~pred & labels).sum())
    return 2.0 * tp / (2.0 * tp + fp + fn) if tp + fp + fn else 0.0


def best_threshold(scores: np.ndarray, labels: np.ndarray):
    """The threshold (one of the scores) that maximises F1, and that F1."""
    s = np.asarray(scores, np.float64)
    order = np.argsort(-s, kind="stable")
    lab = np.asarray(labels).astype(bool)[order]
    tp = np.cumsum(lab)
    fp = np.cumsum(~lab)
    fn = lab.sum() - tp
    f1 = 2.0 * tp / np.maximum(2.0 * tp + fp + fn, 1)
    # only thresholds at the last of a run of equal scores are realisable
    ss = s[order]
    last = np.r_[ss[1:] != ss[:-1], True]
    f1 = np.where(last, f1, -1.0)
    i = int(np.argmax(f1))
    return float(ss[i]), float(f1[i])
