"""Rank-predictor MLP: forward, backward and one Adam step in FP64.

No counterpart in the paper (the paper's ranks come from HOSVD only, Sec. IV.A).
Architecture: 7 -> 64 -> 64 -> 64 -> 9, ReLU after the three hidden layers, a
linear output; loss = mean over batch and outputs of (out - target)^2 with
target = log(rank) for the 9 ranks (3 components x 3 modes).  Layer l computes
h_l = W_l h_{l-1} + b_l with W_l stored (out x in).  Adam (Kingma & Ba 2015) with
bias correction.  Parity pinned by central finite differences.
"""
import numpy as np

SIZES = (7, 64, 64, 64, 9)


def init_params(seed: int, sizes=SIZES):
    """He-uniform weights, zero biases (the GPU path receives these as inputs)."""
    rng = np.random.default_rng(seed)
    params = []
    for i in range(len(sizes) - 1):
        fan_in = sizes[i]
        lim = np.sqrt(6.0 / fan_in)
        W = rng.uniform(-lim, lim, size=(sizes[i + 1], sizes[i]))
        b = np.zeros(sizes[i + 1])
        params.append((W, b))
    return params


def forward(params, X):
    """X (B x 7) -> (out (B x 9), cache)."""
    acts = [np.asarray(X, dtype=np.float64)]
    pre = []
    h = acts[0]
    L = len(params)
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if li < L - 1 else z
        acts.append(h)
    return h, (acts, pre)


def loss(out, target):
    d = out - target
    return float(np.mean(d * d))


def backward(params, cache, out, target):
    """Gradients of loss() w.r.t. every (W, b)."""
    acts, pre = cache
    B, O = out.shape
    g = 2.0 * (out - target) / (B * O)
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li < len(params) - 1:
            g = g * (pre[li] > 0.0)
        gW = g.T @ acts[li]
        gb = g.sum(axis=0)
        grads[li] = (gW, gb)
        g = g @ W
    return grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; state = {'t': int, 'm': [...], 'v': [...]} (created if empty)."""
    if not state:
        state.update(t=0, m=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params],
                     v=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
    state["t"] += 1
    t = state["t"]
    new = []
    for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        mW, mb = state["m"][i]
        vW, vb = state["v"][i]
        mW = b1 * mW + (1 - b1) * gW
        mb = b1 * mb + (1 - b1) * gb
        vW = b2 * vW + (1 - b2) * gW * gW
        vb = b2 * vb + (1 - b2) * gb * gb
        state["m"][i] = (mW, mb)
        state["v"][i] = (vW, vb)
        c1 = 1 - b1 ** t
        c2 = 1 - b2 ** t
        W = W - lr * (mW / c1) / (np.sqrt(vW / c2) + eps)
        b = b - lr * (mb / c1) / (np.sqrt(vb / c2) + eps)
        new.append((W, b))
    return new
