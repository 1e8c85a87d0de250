"""The FP64-grid rule of the double-float state, checked with NumPy's IEEE FP32 and
FP64 arithmetic on the host (the device code states the same operations with
explicit rounding intrinsics).

Claims: (1) the split of a double, hi = RN32(x) and lo = RZ32(x - hi), is a pair
whose sum is a double and whose split is the pair again; (2) a normalised pair
(the output of a two-sum) moved onto the grid by lo <- RN32(RN64(hi + lo) - hi)
is such a fixed point, the move changes the value by at most 2^-53 of it, and
pairs with lo within 28 binades of hi are not moved at all; (3) the kernels'
FP32-only form of that move (round lo to a multiple of the grid spacing q by
adding and subtracting 2^23 q) gives the same bits."""
import numpy as np

f32, f64 = np.float32, np.float64


def split_rz(x):
    x = np.asarray(x, f64)
    hi = x.astype(f32)
    r = x - hi.astype(f64)                      # exact in FP64
    lo = r.astype(f32)
    over = np.abs(lo.astype(f64)) > np.abs(r)   # RN went away from zero: step back
    lo[over] = np.nextafter(lo[over], f32(0))
    return hi, lo


def to_double(hi, lo):
    return hi.astype(f64) + lo.astype(f64)


def on_grid(hi, lo):
    lo = lo.copy()
    m = np.abs(lo) < np.abs(hi) * f32(2.0 ** -28)
    h = hi[m].astype(f64)
    lo[m] = ((h + lo[m].astype(f64)) - h).astype(f32)
    return hi, lo


def on_grid_fp32(hi, lo):
    """The kernels' form: q = 2^(e - 52) from hi's exponent field (one binade less
    when hi is a power of two and lo points towards zero), lo + M - M with
    M = +-2^23 q when |lo| < 2^23 q, all in FP32."""
    hb = hi.view(np.uint32).astype(np.int64)
    eq = ((hb >> 23) & 0xFF) - 127 - 52
    eq = eq - (((hb & 0x7FFFFF) == 0) & (np.signbit(lo) != np.signbit(hi)) & (lo != 0))
    ok = eq >= -149
    t = np.where(ok, np.clip(eq + 23 + 127, 1, 254) << 23, 0).astype(np.uint32).view(f32)
    m = np.where(np.signbit(lo), -t, t).astype(f32)
    with np.errstate(over="ignore", invalid="ignore"):
        moved = ((lo + m) - m).astype(f32)
    return hi, np.where(ok & (np.abs(lo) < t), moved, lo).astype(f32)


def two_sum(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def is_fixed_point(hi, lo):
    h2, l2 = split_rz(to_double(hi, lo))
    return (h2 == hi) & (l2 == lo)


def sample_doubles(rng, m):
    """Doubles over many binades, with the awkward cases mixed in: values next to
    powers of two, values whose remainder after hi is a tie or just below one,
    zeros and subnormal FP32 magnitudes."""
    e = rng.integers(-120, 60, m)
    x = rng.uniform(1.0, 2.0, m) * np.exp2(e) * rng.choice([-1.0, 1.0], m)
    k = m // 8
    p2 = np.exp2(rng.integers(-100, 40, k).astype(f64))
    x[:k] = p2 * (1.0 + rng.choice([-1, 1], k) * rng.integers(1, 40, k) * 2.0 ** -53)
    hi = x[k:2 * k].astype(f32).astype(f64)
    ulp = np.abs(np.spacing(hi.astype(f32))).astype(f64)
    x[k:2 * k] = hi + 0.5 * ulp * (1.0 - rng.integers(0, 3, k) * 2.0 ** -30)
    x[2 * k:2 * k + 8] = 0.0
    x[2 * k + 8:2 * k + 16] = rng.uniform(1, 2, 8) * 2.0 ** -140
    return x


def test_split_of_a_double_is_a_fixed_point():
    rng = np.random.default_rng(0)
    x = sample_doubles(rng, 400_000)
    hi, lo = split_rz(x)
    assert np.all(is_fixed_point(hi, lo))
    d = to_double(hi, lo)
    # (plus FP32's subnormal step, 2^-149, where lo falls below the normal range)
    assert np.all(np.abs(d - x) <= 2.0 ** -47 * np.abs(x) + 2.0 ** -149)
    assert np.all(np.abs(lo.astype(f64)) <= np.abs(x - hi.astype(f64)))  # lo truncated, never rounded up
    # a double whose remainder fits FP32 is held exactly
    exact = np.abs(x - hi.astype(f64)) == np.abs(lo.astype(f64))
    assert exact.mean() > 0.05
    assert np.array_equal(d[exact], x[exact])


def test_two_sum_outputs_moved_onto_the_grid():
    rng = np.random.default_rng(1)
    m = 400_000
    a = (rng.uniform(-1, 1, m) * np.exp2(rng.integers(-90, 30, m))).astype(f32)
    # increments from a hundredth of a down to far below its last bit
    b = (a.astype(f64) * rng.uniform(-1, 1, m) * np.exp2(-rng.integers(0, 60, m).astype(f64))).astype(f32)
    hi, lo = two_sum(a, b)
    assert np.all(hi.astype(f64) + lo.astype(f64) == a.astype(f64) + b.astype(f64))  # exact
    before = is_fixed_point(hi, lo)
    assert 0.0 < before.mean() < 1.0               # some pairs lie off the grid
    h2, l2 = on_grid(hi, lo)
    assert np.array_equal(h2, hi)
    assert np.all(is_fixed_point(h2, l2))
    old = hi.astype(f64) + lo.astype(f64)          # exact old value (<= 48+ bits, rounded
    new = to_double(h2, l2)                        # only when it spans more than 53)
    assert np.all(np.abs(new - old) <= 2.0 ** -53 * np.abs(old) * (1 + 2.0 ** -20))
    near = np.abs(lo) >= np.abs(hi) * f32(2.0 ** -28)
    assert np.array_equal(l2[near], lo[near])      # lo within 28 binades: untouched
    assert np.all(before[near])
    # the rule is idempotent
    h3, l3 = on_grid(h2, l2)
    assert np.array_equal(h3, h2) and np.array_equal(l3, l2)


def test_fp32_form_gives_the_same_bits():
    rng = np.random.default_rng(2)
    m = 1_000_000
    a = (rng.uniform(-1, 1, m) * np.exp2(rng.integers(-100, 60, m))).astype(f32)
    k = m // 5   # powers of two of either sign, where the grid halves below hi
    a[:k] = (np.exp2(rng.integers(-100, 60, k)) * rng.choice([-1.0, 1.0], k)).astype(f32)
    b = (a.astype(f64) * rng.uniform(-1, 1, m) * np.exp2(-rng.integers(0, 70, m).astype(f64))).astype(f32)
    b[k:k + 1000] = 0.0
    hi, lo = two_sum(a, b)
    h1, l1 = on_grid(hi, lo)
    h2, l2 = on_grid_fp32(hi, lo)
    assert np.array_equal(h1.view(np.uint32), h2.view(np.uint32))
    assert np.array_equal(l1.view(np.uint32), l2.view(np.uint32))   # zeros' signs included
    assert (l1 != lo).sum() > 1000                                   # the move did happen


def test_off_grid_pairs_would_not_survive_the_round_trip():
    """Why the rule is needed: a pair whose lo lies more than 29 binades below hi
    spans more than 53 bits, and its conversion to FP64 and back changes it."""
    hi = np.array([1.0, 3.0, -1.5], f32)
    lo = np.array([2.0 ** -40 * 1.2345, -(2.0 ** -38) * 1.7, 2.0 ** -45 * 1.1], f32)
    assert not np.any(is_fixed_point(hi, lo))
    h2, l2 = on_grid(hi, lo)
    assert np.all(is_fixed_point(h2, l2))
