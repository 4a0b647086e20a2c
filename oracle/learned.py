"""CPU oracle of the learned walk budget (plain numpy, FP64).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA library.

What it restates:

* the accuracy criterion of Sec. 5.1 (Eq. lengthdelta): the walks from row k
  suffice once Delta Xi'_k sqrt(M_k) / sigma_k exceeds the normal quantile of
  confidence alpha, so M*_k = (z_alpha sigma_k / (Delta Xi'_k))^2.  The label of
  row k is log((sigma_k / Xi'_k)^2 + 1e-6) from pilot walks (walk kind 1 of
  the Philox keying) and the normaliser fixes (z_alpha / Delta)^2 by the
  requested mean walk count, with the lower bound on M_k of Sec. 5.1;
* per-row graph features (definitions below, written out row by row);
* the 12 -> 64 -> 64 -> 1 ReLU network, its loss gradient and an Adam step,
  in FP64, either exactly or rounding to BF16 at the points where the CUDA
  path does (``emulate=True``: inputs, layer-1 activations, W1 and W2, and
  dL/dh2 before its product with W2);
* the integer budget normaliser (largest-remainder apportionment on
  fixed-point quotas; every step exact).
"""
from __future__ import annotations

import math

import numpy as np

from . import build_factor, walk_rows

NUM_FEATURES = 12
FEATURE_STRIDE = 16
H = 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * FEATURE_STRIDE
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NUM_PARAMS = OFF_B3 + 1


# --------------------------------------------------------------------------
# Features
# --------------------------------------------------------------------------
def row_features(A):
    """Features of every row, FP64 arithmetic, returned as float32 [n, 16]."""
    n = A.n
    rp, col, val = A.rowptr, A.col, A.val
    out = np.zeros((n, FEATURE_STRIDE), dtype=np.float32)
    for k in range(n):
        diag = 0.0
        wsum = wup = wmax = 0.0
        up = lo = 0
        for p in range(rp[k], rp[k + 1]):
            c = col[p]
            if c == k:
                diag = float(val[p])
                continue
            w = -float(val[p])
            wsum += w
            wmax = max(wmax, w)
            if c > k:
                up += 1
                wup += w
            else:
                lo += 1
        deg = up + lo
        ent = nex = ndeg = 0.0
        up2 = 0
        for p in range(rp[k], rp[k + 1]):
            c = col[p]
            if c == k:
                continue
            pr = -float(val[p]) / wsum
            if pr > 0.0:
                ent -= pr * math.log(pr)
            cd = csum = 0.0
            for q in range(rp[c], rp[c + 1]):
                if col[q] == c:
                    cd = float(val[q])
                else:
                    csum += float(val[q])
                    if c > k and col[q] > k:
                        up2 += 1
            nex += (cd + csum) / cd
            ndeg += rp[c + 1] - rp[c] - 1
        f = [math.log1p(deg),
             up / deg if deg else 0.0,
             lo / deg if deg else 0.0,
             (diag - wsum) / diag,
             wup / diag,
             ent,
             wmax / wsum if wsum > 0 else 0.0,
             k / (n - 1 if n > 1 else 1),
             nex / deg if deg else 0.0,
             math.log1p(ndeg / deg if deg else 0.0),
             math.log1p(up2),
             math.log(diag)]
        out[k, :NUM_FEATURES] = np.array(f, dtype=np.float64).astype(np.float32)
    return out


# --------------------------------------------------------------------------
# Pilot-walk statistics (labels)
# --------------------------------------------------------------------------
def pilot_stats(A, walks, seed, max_steps=1 << 24, quantity=0):
    """Per row: mean and sample standard deviation of a per-walk quantity of
    `walks` kind-1 walks -- the length in hops (quantity 0) or the visits to
    the start row, 1 + returns (quantity 1 and 2; Sec. 3.1's J'/M', named in
    Sec. 5.1 as an alternative quantity) -- the label log((sd/mean)^2 + 1e-6)
    (quantity 2: half of that label minus log of the mean walk length),
    and has = 1 for rows with walks.  Returns float32 arrays (mean, sd, label,
    has) and the float64 (mean, var) before rounding."""
    F = build_factor(A, walks, seed, 0.0, tag=1, records=True, max_steps=max_steps)
    n = A.n
    mean = np.zeros(n)
    var = np.zeros(n)
    has = np.zeros(n)
    mean_len = np.zeros(n)
    lens = F["rec_len"].astype(np.float64) if quantity == 0 else F["rec_ret"].astype(np.float64) + 1.0
    for i, k in enumerate(F["walk_rows"]):
        x = lens[i * walks:(i + 1) * walks]
        m = x.sum() / walks
        mean[k] = m
        var[k] = ((x - m) ** 2).sum() / (walks - 1)
        has[k] = 1.0
        mean_len[k] = F["rec_len"][i * walks:(i + 1) * walks].astype(np.float64).sum() / walks
    label = np.where(has > 0, np.log(np.divide(var, mean * mean, out=np.zeros(n), where=has > 0) + 1e-6), 0.0)
    if quantity == 2:
        # cost-aware: exp(label) = sqrt(relative variance / mean walk length)
        # (the float32 label of the visits is what both sides combine)
        lab32 = label.astype(np.float32).astype(np.float64)
        ml32 = mean_len.astype(np.float32).astype(np.float64)
        label = np.where(has > 0, 0.5 * (lab32 - np.log(np.where(has > 0, ml32, 1.0))), 0.0)
    f32 = lambda a: a.astype(np.float32)
    return dict(mean=f32(mean), sd=f32(np.sqrt(var)), label=f32(label), has=f32(has),
                mean64=mean, var64=var, lengths=lens, walk_rows=F["walk_rows"])


def exact_length_moments(A, k):
    """Exact mean and variance of the length (hops) of a walk from row k:
    the first step goes to an upper neighbour j with probability
    A_kj / S_k (Sec. 5.2); afterwards the absorbing chain of Sec. 2.1 on the
    transient nodes k..n-1 (homes 0..k-1 and ground absorb).  With Q the
    transient block, t = (I - Q)^-1 1 and s = (I - Q)^-1 (2t - 1) are the first
    and second moments of the remaining steps (absorbing Markov chain)."""
    Ad = A.to_dense()
    n = A.n
    d = np.diag(Ad)
    P = -Ad / d[:, None]
    np.fill_diagonal(P, 0.0)
    idx = np.arange(k, n)
    Q = P[np.ix_(idx, idx)]
    N = np.linalg.inv(np.eye(len(idx)) - Q)
    t = N @ np.ones(len(idx))
    s = N @ (2 * t - 1)
    ups = np.arange(k + 1, n)
    w = -Ad[k, ups]
    p1 = w / w.sum()
    # length = 1 + remaining steps from the landing node j
    tj, sj = t[ups - k], s[ups - k]
    m1 = float(np.sum(p1 * (1 + tj)))
    m2 = float(np.sum(p1 * (1 + 2 * tj + sj)))
    return m1, m2 - m1 * m1


# --------------------------------------------------------------------------
# Network
# --------------------------------------------------------------------------
def bf16_round(x):
    """Round float32 values to the nearest BF16 value (ties to even), as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(np.asarray(x, dtype=np.float32))
    out = r.astype(np.uint32).view(np.float32)
    return np.where(nan, np.float32(np.nan), out)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    W1 = p[OFF_W1:OFF_B1].reshape(H, FEATURE_STRIDE)[:, :NUM_FEATURES]
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(H, H)
    b2 = p[OFF_B2:OFF_W3]
    w3 = p[OFF_W3:OFF_B3]
    b3 = p[OFF_B3]
    return W1, b1, W2, b2, w3, b3


def inputs(norm, feat, emulate=True):
    """x = (f - mu) * inv_sd, in float32 then rounded to BF16 when emulating."""
    f = np.asarray(feat, dtype=np.float32)[:, :NUM_FEATURES]
    mu = np.asarray(norm[:NUM_FEATURES], dtype=np.float32)
    isd = np.asarray(norm[FEATURE_STRIDE:FEATURE_STRIDE + NUM_FEATURES], dtype=np.float32)
    if emulate:
        x = (f - mu) * isd            # float32 arithmetic, like the kernel
        return bf16_round(x).astype(np.float64)
    return (f.astype(np.float64) - mu) * isd.astype(np.float64)


def forward(params, norm, feat, emulate=True):
    """Network output y [rows] and the activations (x, z1, h1, z2, h2)."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    if emulate:
        W1 = bf16_round(W1.astype(np.float32)).astype(np.float64)
        W2 = bf16_round(W2.astype(np.float32)).astype(np.float64)
    x = inputs(norm, feat, emulate)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    if emulate:
        h1 = bf16_round(h1.astype(np.float32)).astype(np.float64)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, dict(x=x, h1=h1, h2=h2, W1=W1, W2=W2, w3=w3)


def gradient(params, norm, feat, label, emulate=True):
    """Gradient of (1/B) sum (y - label)^2 with respect to the parameter
    vector (layout of the flat vector; W1 columns 12..15 get 0) and the loss."""
    y, a = forward(params, norm, feat, emulate)
    B = len(y)
    e = y - np.asarray(label, dtype=np.float64)
    dy = 2.0 * e / B
    dh2 = np.where(a["h2"] > 0, dy[:, None] * a["w3"][None, :], 0.0)
    dh2_in = bf16_round(dh2.astype(np.float32)).astype(np.float64) if emulate else dh2
    dh1 = np.where(a["h1"] > 0, dh2_in @ a["W2"], 0.0)
    g = np.zeros(NUM_PARAMS)
    gW1 = np.zeros((H, FEATURE_STRIDE))
    gW1[:, :NUM_FEATURES] = dh1.T @ a["x"]
    g[OFF_W1:OFF_B1] = gW1.ravel()
    g[OFF_B1:OFF_W2] = dh1.sum(axis=0)
    g[OFF_W2:OFF_B2] = (dh2.T @ a["h1"]).ravel()
    g[OFF_B2:OFF_W3] = dh2.sum(axis=0)
    g[OFF_W3:OFF_B3] = dy @ a["h2"]
    g[OFF_B3] = dy.sum()
    return g, float(np.mean(e * e))


def adam_step(params, m1, m2, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (bias-corrected moments, step number t >= 1)."""
    m1 = beta1 * m1 + (1 - beta1) * grad
    m2 = beta2 * m2 + (1 - beta2) * grad * grad
    mh = m1 / (1 - beta1 ** t)
    vh = m2 / (1 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m1, m2


# --------------------------------------------------------------------------
# Budget normaliser
# --------------------------------------------------------------------------
FRAC_BITS = 20


def _quota_fixed(w64, s, min_b, cap):
    """V_k = round-half-even(min(cap, max(min_b, s w_k)) 2^20) as int64."""
    v = np.minimum(cap, np.maximum(min_b, s * w64))
    return np.rint(np.ldexp(v, FRAC_BITS)).astype(np.int64)


def budget_normalize(A, w, mean_budget, min_budget):
    """Integer budgets [n] (uint32) from relative needs w (float32 [n]).

    Over the walk rows (rows with an upper neighbour; the others get 0) with
    T = floor(mean * walk rows + 1/2): quotas q_k(s) = min(min(T, 2^31),
    max(min_budget, s w_k)) in 2^-20 fixed point; s by doubling from 1 then
    bisection to the largest total not above T 2^20; then largest-remainder
    apportionment of R = T - sum floor: R // nw to every row and one more to
    the R mod nw rows with the largest fractional part (ties: lower k first).
    """
    n = A.n
    wr = walk_rows(A)
    nw = len(wr)
    budget = np.zeros(n, dtype=np.uint32)
    if nw == 0:
        return budget
    w64 = np.asarray(w, dtype=np.float32)[wr].astype(np.float64)
    if np.any(~np.isfinite(w64)) or np.any(w64 < 0):
        raise ValueError("negative or non-finite weight on a walk row")
    T = int(math.floor(mean_budget * nw + 0.5))
    target = T << FRAC_BITS
    cap = min(float(T), 2147483648.0)
    min_b = float(min_budget)

    def total(s):
        # exact integer sum (split in 32-bit halves so that nothing wraps)
        V = _quota_fixed(w64, s, min_b, cap).astype(np.uint64)
        hi = int((V >> np.uint64(32)).sum(dtype=np.uint64))
        lo = int((V & np.uint64(0xFFFFFFFF)).sum(dtype=np.uint64))
        return (hi << 32) + lo

    lo = 0.0
    tsum = total(0.0)
    if tsum < target:
        hi = 1.0
        while True:
            tsum = total(hi)
            if tsum > target:
                break
            lo = hi
            if tsum == target or hi > 1e300:
                break
            hi *= 2.0
        if tsum > target:
            for _ in range(2200):
                mid = 0.5 * (lo + hi)
                if not (lo < mid < hi):
                    break
                if total(mid) <= target:
                    lo = mid
                else:
                    hi = mid
    V = _quota_fixed(w64, lo, min_b, cap)
    fl = V >> FRAC_BITS
    fr = V & ((1 << FRAC_BITS) - 1)
    R = T - int(fl.sum())
    assert R >= 0
    qa, r = divmod(R, nw)
    b = fl + qa
    order = np.lexsort((wr, -fr))        # fractional part descending, row ascending
    b[order[:r]] += 1
    budget[wr] = b.astype(np.uint32)
    return budget
