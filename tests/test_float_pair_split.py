"""The integer float-pair split and widening the propagation kernels use for their observable sums
(no GPU): a numpy restatement of the bit operations on the double's and the float's words, checked
against the bounds their comments state: |h + l - v| <= 2^-48 v + 2^-126 for the split of v >= 0,
|x|^2 as a float pair within 2^-44 relative, exactness of the widening, with infinities and NaN
carried through."""
import numpy as np


def _split(v):
    b = np.asarray(v, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.int64)
    lo = (b & np.uint64(0xffffffff)).astype(np.int64)
    e = (hi >> 20) & 0x7ff
    hb = ((e - 896) << 23) | ((hi & 0xfffff) << 3) | (lo >> 29)
    hb = np.where(e < 897, 0, hb)
    special = e > 1150
    nan = (e == 2047) & (((hi & 0xfffff) | lo) != 0)
    hb = np.where(special, np.where(nan, 0x7fc00000, 0x7f800000), hb)
    m29 = lo & 0x1fffffff
    lz = np.where(m29 == 0, 32, 31 - np.floor(np.log2(np.maximum(m29, 1))).astype(np.int64))
    t = (m29 << (lz + 1)) & 0xffffffff
    fe = e - 917 - lz
    lb = (fe << 23) | (t >> 9)
    lb = lb + ((t >> 8) & 1)
    lb = np.where((m29 == 0) | (fe <= 0) | (e < 897) | special, 0, lb)
    h = (hb & 0xffffffff).astype(np.uint32).view(np.float32)
    l = (lb & 0xffffffff).astype(np.uint32).view(np.float32)
    return h, l


def _widen(f):
    b = np.asarray(f, dtype=np.float32).view(np.uint32).astype(np.int64)
    e = (b >> 23) & 0xff
    sign = b & 0x80000000
    m = b & 0x7fffff
    h = sign | ((e + 896) << 20) | (m >> 3)
    h = np.where(e == 255, sign | 0x7ff00000 | (m >> 3) | np.where(m != 0, 0x80000, 0), h)
    l = np.where(e == 255, 0, (b << 29) & 0xffffffff)
    h = np.where(e == 0, sign, h)
    l = np.where(e == 0, 0, l)
    return ((h.astype(np.uint64) << np.uint64(32)) | l.astype(np.uint64)).view(np.float64)


def test_split_bound_over_the_whole_range():
    rng = np.random.default_rng(17)
    v = np.concatenate([
        np.exp(rng.uniform(np.log(1e-40), np.log(3e38), 200000)),
        rng.uniform(0.0, 1.0, 50000) ** 8,
        [0.0, 1.0, 2.0 ** -126, 2.0 ** -127, 2.0 ** -149, np.nextafter(1.0, 2.0), 3.4e38, 2.0 ** 127 * (2 - 2.0 ** -40)],
    ])
    h, l = _split(v)
    assert np.all(np.isfinite(h)) and np.all(np.isfinite(l)) and np.all(l >= 0)
    # h exact as the leading bits: the split is exact where the remaining bits fit
    err = np.abs(h.astype(np.float64) + l.astype(np.float64) - v)
    assert np.all(err <= 2.0 ** -48 * v + 2.0 ** -126)
    # the bound is nearly reached (so a split that dropped or truncated l would fail)
    assert np.max(err[v > 1e-30] / v[v > 1e-30]) > 2.0 ** -50
    h0, _ = _split(v[v > 1e-30])
    assert np.max(np.abs(h0.astype(np.float64) - v[v > 1e-30]) / v[v > 1e-30]) > 2.0 ** -26


def test_split_carries_infinity_and_nan():
    h, l = _split(np.array([np.inf, np.nan, 1e300, 3.5e38]))
    assert np.isinf(h[0]) and np.isnan(h[1]) and np.isinf(h[2]) and np.isinf(h[3])
    assert np.all(l == 0)


def test_widening_is_exact():
    rng = np.random.default_rng(18)
    f = np.concatenate([
        (rng.standard_normal(100000) * np.exp(rng.uniform(-80, 80, 100000))).astype(np.float32),
        np.array([0.0, -0.0, 1.0, -2.5, np.float32(1.1754944e-38), np.float32(3.4028235e38)], dtype=np.float32),
    ])
    w = _widen(f)
    assert np.array_equal(w, f.astype(np.float64))
    s = _widen(np.array([np.inf, -np.inf, np.nan, np.float32(1e-40)], dtype=np.float32))
    assert s[0] == np.inf and s[1] == -np.inf and np.isnan(s[2]) and s[3] == 0.0


def _split_signed(v):
    v = np.asarray(v, dtype=np.float64)
    h, l = _split(np.abs(v))
    sgn = np.signbit(v)
    return np.where(sgn, -h, h).astype(np.float32), np.where(sgn, -l, l).astype(np.float32)


def _sq_mod(xr, xi):
    """The kernels' |x|^2 as a float pair (sq_mod_ff), restated with float32 operations; the FMA
    residuals are formed exactly in float64 (an FMA rounds once)."""
    f = np.float32
    ah, al = _split_signed(xr)
    bh, bl = _split_signed(xi)
    p1, p2 = (ah * ah).astype(f), (bh * bh).astype(f)
    e1 = (ah.astype(np.float64) ** 2 - p1).astype(f)
    e2 = (bh.astype(np.float64) ** 2 - p2).astype(f)
    s = (p1 + p2).astype(f)
    bp = (s - p1).astype(f)
    t = ((p1 - (s - bp).astype(f)).astype(f) + (p2 - bp).astype(f)).astype(f)
    c = (np.float64((f(2) * ah + al).astype(f)) * al + ((f(2) * bh + bl).astype(f) * bl).astype(f)).astype(f)
    lo = ((t + (e1 + e2).astype(f)).astype(f) + c).astype(f)
    rh = (s + lo).astype(f)
    rl = (lo - (rh - s).astype(f)).astype(f)
    return rh, rl


def test_squared_modulus_pair_bound():
    rng = np.random.default_rng(19)
    scale = np.exp(rng.uniform(np.log(1e-18), np.log(10.0), 200000))
    xr = rng.standard_normal(scale.size) * scale
    xi = rng.standard_normal(scale.size) * scale
    rh, rl = _sq_mod(xr, xi)
    exact = xr.astype(np.longdouble) ** 2 + xi.astype(np.longdouble) ** 2
    err = np.abs(rh.astype(np.longdouble) + rl.astype(np.longdouble) - exact)
    # relative 2^-45, and an absolute floor below float's normal range (squares of parts under 2^-63)
    assert np.all(err < 2.0 ** -44 * exact + 2.0 ** -124)
    assert float(np.max(err[exact > 1e-30] / exact[exact > 1e-30])) < 2.0 ** -44
    # the signed split keeps the sign on both parts
    h, l = _split_signed(np.array([-1.0 / 3.0, 1.0 / 3.0]))
    assert h[0] == -h[1] and l[0] == -l[1] and h[0] < 0 and l[0] <= 0


def _ff_acc(sh, sl, ah, al):
    """The kernels' float-pair accumulation step (two-sum, then a fast two-sum renormalisation)."""
    f = np.float32
    t = f(sh + ah)
    bp = f(t - sh)
    err = f(f(sh - f(t - bp)) + f(ah - bp))
    lo = f(sl + f(err + al))
    nh = f(t + lo)
    return nh, f(lo - f(nh - t))


def _ff_fma_acc(sh, sl, xh, xl, rh, rl):
    f = np.float32
    p = f(xh * rh)
    e = f(np.float64(xh) * np.float64(rh) - np.float64(p))   # the FMA residual, exact
    lo = f(np.float64(xh) * np.float64(rl) + np.float64(f(np.float64(xl) * np.float64(rh) + np.float64(e))))
    return _ff_acc(sh, sl, p, lo)


def test_block_sums_of_float_pairs():
    """A block of 16 terms x_j rho_j summed as the kernels do (x and rho as float pairs) stays within
    2^-44 of the exact sum relative to the sum of magnitudes, for terms of mixed sign."""
    rng = np.random.default_rng(20)
    worst = 0.0
    for _ in range(3000):
        rho = np.abs(rng.standard_normal(16)) * np.exp(rng.uniform(-20, 2))
        x = rng.uniform(-300, 300, 16)
        rh, rl = _split(rho)
        xh = x.astype(np.float32)
        xl = (x - xh.astype(np.float64)).astype(np.float32)
        sh, sl = np.float32(0), np.float32(0)
        for j in range(16):
            sh, sl = _ff_fma_acc(sh, sl, xh[j], xl[j], rh[j], rl[j])
        got = np.float64(sh) + np.float64(sl)
        exact = float(np.sum(x.astype(np.longdouble) * rho.astype(np.longdouble)))
        worst = max(worst, abs(got - exact) / float(np.sum(np.abs(x * rho))))
    assert worst < 2.0 ** -44
    assert worst > 2.0 ** -60      # not exact: the comparison can fail
