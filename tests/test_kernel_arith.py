"""Small pieces of the kernels' arithmetic modelled and checked on the CPU.

- The FP64 maps' order-preserving cell keys: a < b as doubles exactly when
  key(a) < key(b) as unsigned integers (so atomicMin on keys keeps the
  lowest height), and their below-the-stock test, key(z) < key(stock with
  both zeros taken as -0), decides as z < stock does -- including z or the
  stock being +0 or -0.
- The FP32 maps' raw cells: a cell starts at -0 and takes only heights
  below the stock (negative floats); among those values, a < b as floats
  exactly when bits(a) > bits(b) as signed integers, so a signed atomicMax
  on the raw bits keeps the lowest height.
- The double-float sums of the FP32 maps' roughness: Knuth's two-sum on the
  high parts is exact and symmetric in its operands (every lane of a
  butterfly reduction ends with the same pair), and a sum of many floats
  kept as a pair is accurate far beyond float precision."""
import numpy as np

f32 = np.float32


def enc64(z):
    b = np.asarray(z, dtype=np.float64).view(np.uint64)
    sign = (b >> np.uint64(63)) == 1
    return np.where(sign, ~b, b | np.uint64(1 << 63))


def stock_key(stock):
    return enc64(np.where(stock == 0.0, -0.0, stock))


def test_keys_preserve_order():
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.normal(0, 1e3, 10**5), [0.0, -0.0, 1e-300, -1e-300, 5e-324, -5e-324]])
    b = np.concatenate([rng.normal(0, 1e3, 10**5), [-0.0, 0.0, -1e-300, 1e-300, -5e-324, 5e-324]])
    lt = a < b
    eq = a == b
    ka, kb = enc64(a), enc64(b)
    # strict order agrees except that -0 and +0 compare equal as floats
    both_zero = (a == 0) & (b == 0)
    assert np.array_equal((ka < kb)[~both_zero], lt[~both_zero])
    assert np.array_equal((ka == kb)[~both_zero], eq[~both_zero])
    # FP32 cells: the values a cell can hold are -0 (its start) and negative
    # floats; their raw bits as int32 order them inversely
    neg = -np.abs(rng.normal(0, 1e3, 10**5)).astype(f32)
    neg = np.concatenate([neg, f32([-1e-45, -1.2e-38, -3.4e38, -1.0, -0.0])])
    neg = neg[(neg < 0) | (np.signbit(neg) & (neg == 0))]
    x, y = neg, rng.permutation(neg)
    ix, iy = x.view(np.int32), y.view(np.int32)
    both_zero = (x == 0) & (y == 0)
    assert np.array_equal((ix > iy)[~both_zero], (x < y)[~both_zero])
    # -0, the start value, is below every other value as int32 (any cut lowers it)
    assert f32(-0.0).view(np.int32) == np.iinfo(np.int32).min
    assert (ix[x < 0] > np.iinfo(np.int32).min).all()


def test_below_the_stock_on_keys_equals_the_fp64_comparison():
    rng = np.random.default_rng(2)
    stocks = np.concatenate([rng.normal(0, 5.0, 200), [0.0, -0.0, 1.25, -0.5]])
    for st in stocks:
        z = np.concatenate([st + rng.normal(0, 1e-3, 2000), [st, 0.0, -0.0, np.nextafter(st, -np.inf),
                                                             np.nextafter(st, np.inf)]])
        assert np.array_equal(enc64(z) < stock_key(np.float64(st)), z < st), st


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def df_add(a, b):
    t, e = two_sum(a[0], b[0])
    e = f32(e + f32(a[1] + b[1]))
    hi = f32(t + e)
    return (hi, f32(e - f32(hi - t)))


def test_two_sum_exact_and_symmetric():
    rng = np.random.default_rng(3)
    for _ in range(20000):
        a = f32(rng.normal(0, 10.0 ** rng.uniform(-6, 3)))
        b = f32(rng.normal(0, 10.0 ** rng.uniform(-6, 3)))
        s, e = two_sum(a, b)
        assert np.float64(s) + np.float64(e) == np.float64(a) + np.float64(b)  # exact
        assert two_sum(b, a) == (s, e)                                         # symmetric
        p, q = (a, f32(0)), (b, f32(a * 1e-8))
        assert df_add(p, q) == df_add(q, p)


def test_double_float_sum_is_accurate():
    rng = np.random.default_rng(4)
    x = (rng.normal(-0.1, 0.002, 100_000)).astype(f32)
    acc = (f32(0), f32(0))
    for v in x:
        acc = df_add(acc, (v, f32(0)))
    got = np.float64(acc[0]) + np.float64(acc[1])
    exact = float(np.sum(x.astype(np.float64)))  # float64 of float32 values: error ~1e-16 relative
    assert abs(got - exact) <= 1e-12 * abs(exact), (got, exact)
    naive = float(np.cumsum(x)[-1])               # plain float32 running sum for contrast
    assert abs(naive - exact) > 1e3 * abs(got - exact)


def test_planner_sinusoids_equal_the_pose():
    """The planner writes each coordinate of an edge point's pose,
    cos(Theta_m) u + sin(Theta_m) v + w with Theta_m = phase0 + sense m dtheta,
    as the sinusoid w + amp cos(dtheta (m - mph)) of the step's phase index,
    amp = |(u, v)|, mph = sense (atan2(v, u) - phase0) / dtheta mod S; the
    enumeration solves for its arcs. Both forms agree at every phase, for both
    spindle senses."""
    rng = np.random.default_rng(5)
    for _ in range(500):
        S = int(rng.choice([360, 720, 3600, 7200]))
        dth = 2.0 * np.pi / S
        sense = 1 if rng.random() < 0.5 else -1
        phase0 = np.deg2rad(rng.uniform(-360.0, 360.0))
        u, v, w = rng.normal(0.0, 3.0, 3)
        amp = np.hypot(u, v)
        mph = np.fmod(sense * (np.arctan2(v, u) - phase0) / dth, S)
        mph = mph + S if mph < 0 else mph
        m = np.arange(S)
        th = phase0 + sense * m * dth
        pose = np.cos(th) * u + np.sin(th) * v + w
        sinus = w + amp * np.cos(dth * (m - mph))
        assert np.abs(pose - sinus).max() <= 1e-9 * max(amp, 1.0)


def split_double(z):
    """Model of the kernels' split of a double into a float pair from its
    bits: hi keeps the top 24 significant bits (truncated), lo the other 29
    rounded to a float; magnitudes outside [2^-60, 2^100] (and zero) use the
    rounded conversions."""
    z = np.asarray(z, dtype=np.float64)
    b = z.view(np.uint64)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023
    sign = (b >> np.uint64(63)).astype(np.uint32) << np.uint32(31)
    m = b & np.uint64(0xFFFFFFFFFFFFF)
    hi_bits = sign | ((np.clip(e, -126, 127) + 127).astype(np.uint32) << np.uint32(23)) | \
        (m >> np.uint64(29)).astype(np.uint32)
    hi = hi_bits.view(np.float32)
    rem = (m & np.uint64(0x1FFFFFFF)).astype(np.float64)
    lo = (rem * np.ldexp(1.0, e - 52)).astype(np.float32) * np.where(sign != 0, -1, 1).astype(np.float32)
    fb = (e < -60) | (e > 100)
    hi_f = z.astype(np.float32)
    lo_f = (z - hi_f.astype(np.float64)).astype(np.float32)
    return np.where(fb, hi_f, hi), np.where(fb, lo_f, lo)


def test_split_double_is_a_faithful_float_pair():
    """FP64 maps' moments run in double-float arithmetic on cells split into
    float pairs: hi + lo must be within 2^-47 |z| of z, with lo small
    against hi (so the pair is normalised), for heights of every scale a
    float can hold."""
    rng = np.random.default_rng(47)
    z = np.concatenate([rng.normal(0.0, 1.0, 10**5) * 10.0 ** rng.uniform(-18, 30, 10**5),
                        [0.0, -0.0, 1.0, -1.0, 2.0 ** -60, 2.0 ** 100, 1e-300, -1e35, 0.1, -0.2]])
    hi, lo = split_double(z)
    back = hi.astype(np.float64) + lo.astype(np.float64)
    err = np.abs(back - z)
    assert np.all(err <= 2.0 ** -47 * np.abs(z) + 1e-300 * (np.abs(z) < 1e-290)), err.max()
    nz = (z != 0) & np.isfinite(hi)
    assert np.all(np.abs(lo[nz]) <= 2.0 ** -22 * np.abs(hi[nz]))
