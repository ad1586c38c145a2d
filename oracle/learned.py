"""fp64 reference of the learned-bounds model (TEST INFRASTRUCTURE ONLY; see oracle/__init__).

Two root kinds are referenced here: the 1 -> H -> 1 monotone MLP below, and the
piecewise-linear root (``pwl_*``): K knots at x = k / K whose heights theta = (h_0 .. h_K)
are the parameters (kept non-decreasing by the optimiser's projection).

The paper accelerates ``A_P.lower_bound`` (Alg. 1) with a static S-tree over the key array
(Sec. 2.1, "Storing P twice").  The GPU path replaces that search structure by a two-stage
learned CDF model whose prediction is only a hint: every predicted position is verified and
falls back to the full binary search, so the positions (and therefore the query results) are
those of ``lower_bound`` by construction.  What needs a reference is the model itself:

  root (a tiny monotone MLP, 1 -> H -> 1), on x = key / 2^60:
      f(x) = c + sum_k exp(alpha_k) * sigmoid(exp(beta_k) * x + b_k)
  trained to the normalised rank y = i / n of the sorted keys with the mean-squared error
      L = (1/N) sum_i (f(x_i) - y_i)^2,
  leaf j = clamp(floor(f(x) * J), 0, J - 1) for J leaves; each leaf is a least-squares line
  of position against key offset; a per-leaf error window is the min and max of
  (position - predicted position) over the leaf's keys.

Each leaf also keeps a fence (``leaf_fence``): the keys at 16 equally spaced positions of its
range; ``fence_bracket`` gives the positions between which lower_bound of a target lies.

Nothing here is fitted to the GPU's fp32 numbers: the gradient is the analytic derivative of
L, pinned by central finite differences in tests/test_oracle_learned.py, and the leaf fit is
the closed-form normal equations, pinned against numpy.polyfit.
"""
from __future__ import annotations

import numpy as np

KEY_SCALE = float(2 ** 60)  # x = key / 2^60 maps the 60-bit key space onto [0, 1)


def unpack(theta: np.ndarray, H: int):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (3 * H + 1,)
    return theta[0:H], theta[H:2 * H], theta[2 * H:3 * H], theta[3 * H]


def pack(alpha, beta, b, c) -> np.ndarray:
    return np.concatenate([np.asarray(alpha, np.float64), np.asarray(beta, np.float64),
                           np.asarray(b, np.float64), np.asarray([c], np.float64)])


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def root_forward(theta, x, H: int):
    """f(x) of the root for fp64 inputs x (already scaled to [0, 1))."""
    alpha, beta, b, c = unpack(theta, H)
    x = np.asarray(x, np.float64)[:, None]
    h = sigmoid(np.exp(beta)[None, :] * x + b[None, :])
    return c + h @ np.exp(alpha)


def root_loss(theta, x, y, H: int) -> float:
    r = root_forward(theta, x, H) - np.asarray(y, np.float64)
    return float(np.mean(r * r))


def root_loss_grad(theta, x, y, H: int):
    """Loss and its analytic gradient dL/dtheta, theta = (alpha, beta, b, c).

    With r_i = 2 (f_i - y_i) / N, h_ik = sigmoid(exp(beta_k) x_i + b_k), A_k = exp(alpha_k):
        dL/dc       = sum_i r_i
        dL/dalpha_k = sum_i r_i A_k h_ik
        dL/db_k     = sum_i r_i A_k h_ik (1 - h_ik)
        dL/dbeta_k  = sum_i r_i A_k h_ik (1 - h_ik) exp(beta_k) x_i
    """
    alpha, beta, b, c = unpack(theta, H)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    N = x.shape[0]
    A = np.exp(alpha)
    B = np.exp(beta)
    h = sigmoid(B[None, :] * x[:, None] + b[None, :])
    f = c + h @ A
    res = f - y
    loss = float(np.mean(res * res))
    r = 2.0 * res / N
    g_alpha = (r @ h) * A
    s = h * (1.0 - h)
    g_b = (r @ s) * A
    g_beta = (r @ (s * x[:, None])) * A * B
    g_c = float(np.sum(r))
    return loss, pack(g_alpha, g_beta, g_b, g_c)


def init_params(H: int) -> np.ndarray:
    """Deterministic start: H logistic steps of equal height 1/H centred at (k + 1/2)/H with
    slope 4H, i.e. close to the CDF of keys spread uniformly over the key space."""
    k = np.arange(H, dtype=np.float64)
    s = 4.0 * H
    alpha = np.full(H, np.log(1.0 / H))
    beta = np.full(H, np.log(s))
    b = -s * (k + 0.5) / H
    return pack(alpha, beta, b, 0.0)


def adam_step(theta, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) with bias correction at step t >= 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


# --------------------------------------------------------------------------------------
# piecewise-linear root
# --------------------------------------------------------------------------------------

def pwl_forward(theta, x, K: int):
    """f(x) = h_k + (h_{k+1} - h_k) t with s = x K, k = min(floor(s), K - 1), t = s - k."""
    h = np.asarray(theta, np.float64)
    assert h.shape == (K + 1,)
    s = np.asarray(x, np.float64) * K
    k = np.clip(np.floor(s).astype(np.int64), 0, K - 1)
    t = s - k
    return h[k] + (h[k + 1] - h[k]) * t


def pwl_loss(theta, x, y, K: int) -> float:
    r = pwl_forward(theta, x, K) - np.asarray(y, np.float64)
    return float(np.mean(r * r))


def pwl_loss_grad(theta, x, y, K: int):
    """Loss and analytic gradient: with r_i = 2 (f_i - y_i) / N, knot k_i receives
    r_i (1 - t_i) and knot k_i + 1 receives r_i t_i."""
    h = np.asarray(theta, np.float64)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    N = x.shape[0]
    s = x * K
    k = np.clip(np.floor(s).astype(np.int64), 0, K - 1)
    t = s - k
    f = h[k] + (h[k + 1] - h[k]) * t
    res = f - y
    r = 2.0 * res / N
    g = np.zeros(K + 1)
    np.add.at(g, k, r * (1.0 - t))
    np.add.at(g, k + 1, r * t)
    return float(np.mean(res * res)), g


def pwl_init(K: int) -> np.ndarray:
    """Heights k / K: f(x) = x."""
    return np.arange(K + 1, dtype=np.float64) / K


def pwl_project(theta) -> np.ndarray:
    """Running maximum: the nearest-above non-decreasing sequence used after each step."""
    return np.maximum.accumulate(np.asarray(theta, np.float64))


def leaf_fit(u: np.ndarray, v: np.ndarray):
    """Least-squares line v ~ slope * u + icpt by the normal equations (fp64).
    Degenerate cases: no points -> (0, 0); all u equal -> (0, mean(v))."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    N = u.shape[0]
    if N == 0:
        return 0.0, 0.0
    su, sv = u.sum(), v.sum()
    suu, suv = (u * u).sum(), (u * v).sum()
    den = N * suu - su * su
    if den <= 0.0:
        return 0.0, sv / N
    slope = (N * suv - su * sv) / den
    icpt = (sv - slope * su) / N
    return float(slope), float(icpt)


def error_window(positions: np.ndarray, predicted: np.ndarray):
    """(min, max) of position - prediction over a leaf's keys: the window that contains the
    true position of every key of the leaf."""
    d = np.asarray(positions, np.int64) - np.asarray(predicted, np.int64)
    return int(d.min()), int(d.max())


FENCE = 16  # fence keys per leaf


def leaf_fence(keys: np.ndarray, first: int, end: int, k: int = FENCE) -> np.ndarray:
    """The fence of a leaf covering sorted positions [first, end): the keys at positions
    first + floor(s * (end - first) / k), s = 0 .. k-1 (all bits set for an empty leaf)."""
    c = int(end) - int(first)
    if c <= 0:
        return np.full(k, np.iinfo(np.uint64).max, np.uint64)
    pos = int(first) + (np.arange(k, dtype=np.int64) * c) // k
    return np.asarray(keys, np.uint64)[pos]


def fence_bracket(fence: np.ndarray, first: int, end: int, t: int, k: int = FENCE):
    """[lo, hi] that holds lower_bound(t) over the leaf's keys when that lies in [first, end]:
    with s fence keys below t, between the positions of fence keys s - 1 (exclusive) and s."""
    c = int(end) - int(first)
    s = int(np.count_nonzero(np.asarray(fence, np.uint64) < np.uint64(t)))
    lo = first if s == 0 else first + ((s - 1) * c) // k + 1
    hi = end if s == k else first + (s * c) // k
    return lo, hi


# --------------------------------------------------------------------------------------
# the query-time predict function, in the precision the queries use (fp32)
# --------------------------------------------------------------------------------------
# The error window of a leaf is an integer decided by fp32 arithmetic: the position predicted
# for key k is first + floor(fma(slope, f32(k - base), icpt)) with every operation rounded to
# nearest (ties to even) in IEEE single precision, the product and sum fused (one rounding).
# The helpers below reproduce that rounding exactly from integer and fp64 arithmetic, so the
# windows can be compared exactly; tests/test_oracle_learned.py pins them against exact
# rational arithmetic.

def _bit_length_u64(v: np.ndarray) -> np.ndarray:
    v = np.asarray(v, np.uint64).copy()
    bl = np.zeros(v.shape, np.int64)
    for s in (32, 16, 8, 4, 2, 1):
        big = v >= np.uint64(1 << s)
        bl += s * big
        v = np.where(big, v >> np.uint64(s), v)
    return bl + (v > 0)


def f32_of_int(v: np.ndarray) -> np.ndarray:
    """int64 values rounded to the nearest float32 (ties to even), returned as float32."""
    v = np.asarray(v, np.int64)
    neg = v < 0
    a = np.where(neg, -v, v).astype(np.uint64)          # |v| < 2^63
    bl = _bit_length_u64(a)
    shift = np.maximum(bl - 24, 0).astype(np.uint64)
    q = a >> shift
    rem = a - (q << shift)
    half = np.where(shift > 0, np.uint64(1) << (np.maximum(shift, np.uint64(1)) - np.uint64(1)), np.uint64(0))
    up = (shift > 0) & ((rem > half) | ((rem == half) & ((q & np.uint64(1)) == 1)))
    q = q + up.astype(np.uint64)
    mag = q.astype(np.float64) * np.exp2(shift.astype(np.float64))   # exact: q <= 2^24
    return np.where(neg, -mag, mag).astype(np.float32)


def fma_f32(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """a * b + c for float32 inputs with a single rounding to float32 (ties to even).

    a * b is exact in fp64 (two 24-bit significands); the fp64 sum s = a*b + c and its exact
    error e come from the TwoSum algorithm (Knuth); s is then moved to round-to-odd (one ulp
    towards e when e != 0 and s's last significand bit is 0), and the round-to-odd fp64 value,
    having at least two more bits than float32, rounds to the correctly rounded float32
    (Boldo and Melquiond, "Emulation of FMA and correctly rounded sums", 2008)."""
    a = np.asarray(a, np.float32).astype(np.float64)
    b = np.asarray(b, np.float32).astype(np.float64)
    c = np.asarray(c, np.float32).astype(np.float64)
    ab = a * b
    s = ab + c
    bb = s - ab
    e = (ab - (s - bb)) + (c - bb)
    s = np.atleast_1d(s).copy()
    e = np.atleast_1d(e)
    even = (s.view(np.int64) & 1) == 0
    fix = (e != 0) & even
    if fix.any():
        s[fix] = np.nextafter(s[fix], np.where(e[fix] > 0, np.inf, -np.inf))
    return s.astype(np.float32)


def predict_positions(slope: float, icpt: float, first: int, base: int, keys: np.ndarray) -> np.ndarray:
    """Predicted positions of keys routed to a leaf: first + floor(p), p = fma(slope,
    f32(key - base), icpt) in float32, clamped to [-2e9, 2e9] (the difference taken as a
    signed 64-bit integer)."""
    d = (np.asarray(keys, np.uint64) - np.uint64(base)).view(np.int64)
    u = f32_of_int(d)
    p = fma_f32(np.full(u.shape, slope, np.float32), u, np.full(u.shape, icpt, np.float32))
    p = np.minimum(np.maximum(p, np.float32(-2.0e9)), np.float32(2.0e9))
    return int(first) + np.floor(p.astype(np.float64)).astype(np.int64)
