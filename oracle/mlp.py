"""FP64 reference of the learned importance-sampling proposal.

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper leaves the optimal bias in the two-dimensional phase space open
(Sec. 5) and uses the diffusion-based bias B = A S (1, tan theta_n) of
Eq. (4.10). The learned proposal replaces the constant amplitude A by
alpha = MLP(x, pi, N) projected on the noise direction:

    h1 = silu(W1 s + b1), h2 = silu(W2 h1 + b2), o = W3 h2 + b3,
    alpha = (o1 + t o2) / sqrt(1 + t^2),   t = tan(theta_n),

clamped to |alpha| <= alpha_max, with s = (state - shift) * scale and alpha
held fixed over segments of ``segment`` steps.

Training objective (log-variance loss towards the exponentially tilted
target): L(theta) = Var_Q[ln w_theta + lambda N] over paths drawn from the
current proposal Q. For a recorded path with segment sums of the noise,
ln w_theta = -sum_s [alpha_s zeta_s - alpha_s^2 m_s dN / 2], zeta_s the
standardised increment of segment s (m_s steps); at the sampling parameters
d ln w / d theta = -sum_s sqrt(dN) (sum of xi over s) d alpha_s / d theta, so
dL/dtheta = (2/n) sum_j (Y_j - mean Y) d ln w_j / d theta, Y = ln w + lambda N.

Full-rank (2-D) noise: the bias is B = S beta with beta = (clamp o1, clamp o2)
(each to +-alpha_max, held per segment), the weight increment of Eq. (4.5) is
beta . (beta dN/2 + xi sqrt(dN)), so ln w_theta = -sum_s [beta_s . zeta_s -
|beta_s|^2 m_s dN / 2] with zeta_s the sums of the standardised increments, and
at the sampling parameters d ln w / d theta = -sum_s sqrt(dN) sum_k
(sum of xi_k over s) d beta_{s,k} / d theta.
"""
from __future__ import annotations

import numpy as np

KEYS = ("W1", "b1", "W2", "b2", "W3", "b3")


def silu(a):
    return a / (1.0 + np.exp(-a))


def dsilu(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def bf16(x):
    """Round float64 values to the nearest bfloat16 (via float32, ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = u.view(np.float32).astype(np.float64)
    bad = ~np.isfinite(f)
    out[bad] = f[bad]
    return out


def forward(p, s, round_bf16=False):
    """s: [n, 3] normalised inputs. Returns (o [n, 2], cache).

    round_bf16: the network as bf16 tensor-core tiles hold it -- the weight
    matrices W1, W2, W3 rounded to bfloat16 (biases stay fp32), and the inputs
    and hidden activations rounded to bfloat16 before each product."""
    W = {k: (bf16(p[k]) if round_bf16 else p[k]) for k in ("W1", "W2", "W3")}
    x = bf16(s) if round_bf16 else s
    a1 = x @ W["W1"].T + p["b1"]
    h1 = silu(a1)
    if round_bf16:
        h1 = bf16(h1)
    a2 = h1 @ W["W2"].T + p["b2"]
    h2 = silu(a2)
    if round_bf16:
        h2 = bf16(h2)
    o = h2 @ W["W3"].T + p["b3"]
    return o, (x, a1, h1, a2, h2)


def alpha_of(o, t, alpha_max):
    a = (o[:, 0] + t * o[:, 1]) / np.sqrt(1.0 + t * t)
    return np.clip(a, -alpha_max, alpha_max)


def backward(p, cache, do):
    """Gradients of sum(do * o) with respect to the parameters."""
    x, a1, h1, a2, h2 = cache
    g = {}
    g["W3"] = do.T @ h2
    g["b3"] = do.sum(axis=0)
    dh2 = do @ p["W3"]
    da2 = dh2 * dsilu(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * dsilu(a1)
    g["W1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    return g


def alpha_grad(p, s, t, alpha_max, dalpha, round_bf16=False):
    """Gradient of sum(dalpha * alpha(s, t)) with respect to the parameters."""
    o, cache = forward(p, s, round_bf16)
    raw = (o[:, 0] + t * o[:, 1]) / np.sqrt(1.0 + t * t)
    live = np.abs(raw) < alpha_max
    c = np.where(live, dalpha, 0.0) / np.sqrt(1.0 + t * t)
    do = np.stack([c, c * t], axis=1)
    return backward(p, cache, do)


def normalise(state, shift, scale):
    return (np.asarray(state) - np.asarray(shift)[None, :]) * np.asarray(scale)[None, :]


def logvar_loss_grad(p, trajs, dN, lam, shift, scale, alpha_max, round_bf16=False):
    """Log-variance loss and its gradient at the sampling parameters.

    ``trajs``: list of dicts with keys state [k,3], tan_theta [k], sum_xi [k],
    logw, nsteps (as returned by oracle.stepper.run_segments).
    """
    Y = np.array([tr["logw"] + lam * tr["nsteps"] * dN for tr in trajs])
    n = len(trajs)
    Ybar = Y.mean()
    loss = float(np.mean((Y - Ybar) ** 2))
    grads = {k: np.zeros_like(p[k]) for k in KEYS}
    for j, tr in enumerate(trajs):
        if len(tr["sum_xi"]) == 0:
            continue
        coef = 2.0 / n * (Y[j] - Ybar)
        dalpha = coef * (-np.sqrt(dN) * tr["sum_xi"])
        s = normalise(tr["state"], shift, scale)
        g = alpha_grad(p, s, tr["tan_theta"], alpha_max, dalpha, round_bf16)
        for k in KEYS:
            grads[k] += g[k]
    return loss, grads


def logw_at(p, tr, dN, shift, scale, alpha_max, segment, round_bf16=False):
    """ln w_theta of a recorded path under parameters p (off-policy), used to
    check the gradient by finite differences. The path's standardised segment
    increments are zeta_s = sqrt(dN) sum_xi_s + alpha_s m_s dN with the
    sampling alpha_s."""
    k = len(tr["sum_xi"])
    m = np.full(k, float(segment))
    m[-1] = tr["nsteps"] - segment * (k - 1)
    zeta = np.sqrt(dN) * tr["sum_xi"] + tr["alpha"] * m * dN
    o, _ = forward(p, normalise(tr["state"], shift, scale), round_bf16)
    a = alpha_of(o, tr["tan_theta"], alpha_max)
    return float(-np.sum(a * zeta - 0.5 * a * a * m * dN))


def beta_of(o, alpha_max):
    """2-D bias: each network output clamped to +-alpha_max."""
    return np.clip(o, -alpha_max, alpha_max)


def beta_grad(p, s, alpha_max, dbeta, round_bf16=False):
    """Gradient of sum(dbeta * beta(s)) with respect to the parameters
    (zero on a clamped component)."""
    o, cache = forward(p, s, round_bf16)
    do = np.where(np.abs(o) < alpha_max, dbeta, 0.0)
    return backward(p, cache, do)


def logvar_loss_grad2(p, trajs, dN, lam, shift, scale, alpha_max, round_bf16=False):
    """Log-variance loss and gradient for 2-D paths (oracle.stepper.run2_segments)."""
    Y = np.array([tr["logw"] + lam * tr["nsteps"] * dN for tr in trajs])
    n = len(trajs)
    Ybar = Y.mean()
    loss = float(np.mean((Y - Ybar) ** 2))
    grads = {k: np.zeros_like(p[k]) for k in KEYS}
    for j, tr in enumerate(trajs):
        if len(tr["sum_xi"]) == 0:
            continue
        coef = 2.0 / n * (Y[j] - Ybar)
        dbeta = coef * (-np.sqrt(dN) * tr["sum_xi"])
        g = beta_grad(p, normalise(tr["state"], shift, scale), alpha_max, dbeta, round_bf16)
        for k in KEYS:
            grads[k] += g[k]
    return loss, grads


def logw_at2(p, tr, dN, shift, scale, alpha_max, segment, round_bf16=False):
    """ln w_theta of a recorded 2-D path under parameters p (off-policy)."""
    k = len(tr["sum_xi"])
    m = np.full(k, float(segment))
    m[-1] = tr["nsteps"] - segment * (k - 1)
    zeta = np.sqrt(dN) * tr["sum_xi"] + tr["beta"] * (m * dN)[:, None]
    o, _ = forward(p, normalise(tr["state"], shift, scale), round_bf16)
    b = beta_of(o, alpha_max)
    return float(-np.sum(b * zeta) + 0.5 * np.sum(b * b * (m * dN)[:, None]))
