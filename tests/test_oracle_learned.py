"""Pins for the fp64 reference of the learned-bounds model: the analytic gradient against
central finite differences, the Adam step against its closed form at t = 1, and the leaf fit
against numpy.polyfit and exact lines."""
import numpy as np
import pytest

from oracle import learned as L


@pytest.mark.parametrize("H", [1, 4, 16])
def test_gradient_vs_finite_differences(H):
    rng = np.random.default_rng(H)
    x = np.sort(rng.uniform(0, 1, 300))
    y = np.linspace(0, 1, 300)
    theta = L.init_params(H) + rng.normal(0, 0.3, 3 * H + 1)
    loss, g = L.root_loss_grad(theta, x, y, H)
    assert loss == pytest.approx(L.root_loss(theta, x, y, H), rel=1e-12)
    eps = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd[i] = (L.root_loss(tp, x, y, H) - L.root_loss(tm, x, y, H)) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9)


def test_zero_loss_at_exact_fit():
    H = 3
    theta = L.init_params(H)
    x = np.linspace(0, 1, 50)
    y = L.root_forward(theta, x, H)
    loss, g = L.root_loss_grad(theta, x, y, H)
    assert loss == 0.0 and np.all(g == 0.0)


def test_root_is_monotone():
    H = 8
    rng = np.random.default_rng(0)
    theta = L.init_params(H) + rng.normal(0, 1.0, 3 * H + 1)
    x = np.linspace(0, 1, 10001)
    assert np.all(np.diff(L.root_forward(theta, x, H)) >= 0)


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so the step is lr*g/(|g|+eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.zeros(4)
    th1, m, v = L.adam_step(th, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(th1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_leaf_fit():
    rng = np.random.default_rng(2)
    u = rng.uniform(0, 1e12, 500)
    v = 3e-9 * u + 17.0 + rng.normal(0, 2.0, 500)
    s, c = L.leaf_fit(u, v)
    ps, pc = np.polyfit(u, v, 1)
    assert s == pytest.approx(ps, rel=1e-9) and c == pytest.approx(pc, rel=1e-9, abs=1e-6)
    s, c = L.leaf_fit(np.arange(10.0), 2.0 * np.arange(10.0) + 5.0)
    assert s == pytest.approx(2.0) and c == pytest.approx(5.0)
    assert L.leaf_fit(np.array([]), np.array([])) == (0.0, 0.0)
    assert L.leaf_fit(np.full(4, 7.0), np.arange(4.0)) == (0.0, 1.5)


def test_error_window_contains_all():
    pos = np.arange(100)
    pred = pos + np.random.default_rng(1).integers(-5, 6, 100)
    lo, hi = L.error_window(pos, pred)
    assert np.all(pos - pred >= lo) and np.all(pos - pred <= hi)
    assert lo == (pos - pred).min() and hi == (pos - pred).max()


@pytest.mark.parametrize("K", [1, 4, 256])
def test_pwl_gradient_vs_finite_differences(K):
    rng = np.random.default_rng(K)
    x = np.sort(rng.uniform(0, 1, 400))
    y = np.linspace(0, 1, 400) ** 1.5
    theta = L.pwl_init(K) + rng.normal(0, 0.01, K + 1)
    loss, g = L.pwl_loss_grad(theta, x, y, K)
    assert loss == pytest.approx(L.pwl_loss(theta, x, y, K), rel=1e-12)
    eps = 1e-6
    idx = range(K + 1) if K <= 8 else rng.choice(K + 1, 24, replace=False)
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (L.pwl_loss(tp, x, y, K) - L.pwl_loss(tm, x, y, K)) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_pwl_init_is_identity_and_projection_monotone():
    K = 256
    x = np.linspace(0, 1, 10001)
    np.testing.assert_allclose(L.pwl_forward(L.pwl_init(K), x, K), x, atol=1e-12)
    rng = np.random.default_rng(3)
    theta = L.pwl_project(L.pwl_init(K) + rng.normal(0, 0.05, K + 1))
    assert np.all(np.diff(theta) >= 0)
    assert np.all(np.diff(L.pwl_forward(theta, x, K)) >= 0)
    # knots are interpolated exactly
    np.testing.assert_allclose(L.pwl_forward(theta, np.arange(K) / K, K), theta[:K], rtol=1e-12)


def test_pwl_least_squares_optimum_is_the_cdf_on_a_line():
    """Data on the line y = 0.3 + 0.5 x: the least-squares heights are the line's values at
    the knots (a closed form), and the analytic gradient vanishes there."""
    K = 8
    x = np.linspace(0, 1, 1001, endpoint=False)
    y = 0.3 + 0.5 * x
    h = 0.3 + 0.5 * np.arange(K + 1) / K
    loss, g = L.pwl_loss_grad(h, x, y, K)
    assert loss < 1e-28 and np.abs(g).max() < 1e-14


def test_fence_bracket_holds_lower_bound():
    """The fence bracket of a leaf (Sec. 2.1's lower_bound, bounded by keys of the array at
    equally spaced positions) always holds the true lower_bound, on duplicates too."""
    from oracle import learned as L
    rng = np.random.default_rng(17)
    keys = np.sort(rng.integers(0, 1 << 40, 5000).astype(np.uint64))
    keys[100:400] = keys[100]                          # a run of duplicates
    for first, end in [(0, 5000), (10, 11), (37, 1237), (100, 420), (4990, 5000)]:
        f = L.leaf_fence(keys, first, end)
        assert np.all(np.diff(f.astype(np.float64)) >= 0)
        for t in list(keys[first:end:7]) + list(rng.integers(int(keys[first]), int(keys[end - 1]) + 1, 300)):
            lb = int(np.searchsorted(keys, np.uint64(t), side="left"))
            lo, hi = L.fence_bracket(f, first, end, int(t))
            if first <= lb <= end:
                assert lo <= lb <= hi, (first, end, t, lb, lo, hi)
            assert hi - lo <= (end - first) // L.FENCE + 1
    e = L.leaf_fence(keys, 5, 5)
    assert np.all(e == np.iinfo(np.uint64).max)


# --------------------------------------------------------------------------------------
# the fp32 predict function (error windows are integers decided in fp32)
# --------------------------------------------------------------------------------------

def _round_f32_exact(x):
    """Nearest float32 (ties to even) of a rational x in the normal range, by integer
    arithmetic on the exact value: scale to a 24-bit significand and round the integer."""
    from fractions import Fraction
    x = Fraction(x)
    if x == 0:
        return 0.0
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    assert Fraction(2) ** e <= a < Fraction(2) ** (e + 1)
    m = a / Fraction(2) ** (e - 23)                 # in [2^23, 2^24)
    q, r = divmod(m.numerator, m.denominator)
    rr = Fraction(r, m.denominator)
    if rr > Fraction(1, 2) or (rr == Fraction(1, 2) and q % 2 == 1):
        q += 1
    return sign * float(Fraction(q) * Fraction(2) ** (e - 23))


def test_f32_of_int_rounds_to_nearest_even():
    rng = np.random.default_rng(7)
    vals = [0, 1, -1, 2 ** 24, 2 ** 24 + 1, 2 ** 24 + 3, 2 ** 25 + 2, 2 ** 25 + 6, 2 ** 53 + 1,
            2 ** 60 - 1, -(2 ** 59 + 2 ** 35), (1 << 62) + (1 << 38)]
    vals += [int(v) for v in rng.integers(-(2 ** 62), 2 ** 62, 3000)]
    vals += [int(v) >> int(s) for v, s in zip(rng.integers(0, 2 ** 62, 3000), rng.integers(0, 62, 3000))]
    got = L.f32_of_int(np.array(vals, np.int64))
    want = np.array([_round_f32_exact(v) for v in vals], np.float64)
    assert np.array_equal(got.astype(np.float64), want)


def test_fma_f32_is_correctly_rounded():
    """fused a*b + c with one rounding, against exact rational arithmetic; includes products
    whose sum with c lands exactly half-way between two floats and cancellations."""
    from fractions import Fraction
    rng = np.random.default_rng(8)
    a = rng.normal(0, 1, 4000).astype(np.float32) * np.float32(2.0) ** rng.integers(-40, 0, 4000).astype(np.float32)
    b = L.f32_of_int(rng.integers(0, 2 ** 50, 4000))
    c = (rng.normal(0, 1, 4000) * 10.0 ** rng.integers(-2, 6, 4000)).astype(np.float32)
    # exact ties: a*b = 2^-24 is half an ulp of c in [1, 2) -> ties to even
    a[:40] = np.float32(1.0)
    b[:40] = np.float32(2.0 ** -24)
    c[:40] = np.where(np.arange(40) % 2 == 0, np.float32(1.0), np.float32(1.0 + 2.0 ** -23))
    # just below a tie: a*b = 2^-24 - k^2 2^-70 with c = 1 + 2^-23 (odd); the fp64 sum rounds
    # onto the tie itself, so rounding that to float32 would go up, while the exact value rounds
    # down
    k = np.arange(1, 41, dtype=np.float64)
    a[40:80] = (1.0 + k * 2.0 ** -23).astype(np.float32)
    b[40:80] = ((1.0 - k * 2.0 ** -23) * 2.0 ** -24).astype(np.float32)
    c[40:80] = np.float32(1.0 + 2.0 ** -23)
    naive = (a[40:80].astype(np.float64) * b[40:80].astype(np.float64) + c[40:80].astype(np.float64)).astype(np.float32)
    assert np.all(naive == np.float32(1.0 + 2.0 ** -22))   # the double rounding this must avoid
    # cancellation
    c[100:150] = -(a[100:150].astype(np.float64) * b[100:150].astype(np.float64)).astype(np.float32)
    got = L.fma_f32(a, b, c)
    want = [_round_f32_exact(Fraction(float(x)) * Fraction(float(y)) + Fraction(float(z)))
            for x, y, z in zip(a, b, c)]
    assert np.array_equal(got.astype(np.float64), np.array(want, np.float64))


def test_predict_positions_small_case():
    """slope 0.5, icpt 1.25: key offsets 0, 1, 2, 3, 5 -> floor(1.25, 1.75, 2.25, 2.75, 3.75)."""
    keys = np.array([100, 101, 102, 103, 105], np.uint64)
    p = L.predict_positions(0.5, 1.25, 10, 100, keys)
    assert p.tolist() == [11, 11, 12, 12, 13]
    # keys below the base give negative offsets (signed difference)
    assert L.predict_positions(1.0, 0.0, 10, 100, np.array([98], np.uint64)).tolist() == [8]
    # the prediction is clamped to [-2e9, 2e9] before the floor
    assert L.predict_positions(1e30, 0.0, 0, 0, np.array([5], np.uint64)).tolist() == [2_000_000_000]
