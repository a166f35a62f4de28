"""Philox4x32-10 and the Gaussian auxiliary-field draw (oracle side).

Test infrastructure only (see oracle/__init__.py).

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): 10 rounds of two
32x32->64 multiplies with multipliers 0xD2511F53 / 0xCD9E8D57, the Weyl key
increments 0x9E3779B9 / 0xBB67AE85 between rounds.

The fields x_gamma ~ N(0, 1) of Eq. 8 are drawn with the Box-Muller transform
(Box & Muller 1958).  So that a GPU implementation can reproduce them bit for
bit, every floating-point step below is a single IEEE-754 binary64 operation
rounded to nearest (no fused multiply-add), and log / sin / cos are evaluated
by fixed series written out here from the mathematics:

* log u: u = m 2^e with m in [sqrt(1/2), sqrt(2)); log m = 2 atanh(t),
  t = (m-1)/(m+1), summed as the odd series t + t^3/3 + ... + t^23/23 by
  Horner's rule in t^2; log u = e ln2 + 2 t S(t^2).
* sin, cos of phi = 2 pi u2: quarter-turn reduction q = 4 u2 (exact), k =
  floor(q), f = q - k; reflection f -> 1 - f for f > 1/2 so the reduced
  argument r = f pi/2 lies in [0, pi/4]; Taylor series to degree 17 (sin) and
  16 (cos) by Horner's rule in r^2.

Counter layout (a convention of this implementation): for the field pair
(x_{2j}, x_{2j+1}) of walker slot w at step s, stream t:
    counter = (j, w, s mod 2^32, (s >> 32) mod 2^16 | t << 16),  key = (seed lo, seed hi).
Stream 0 draws the fields; stream 1 draws the comb offset xi.
Uniforms use 52 random bits: u = (m + 1/2) 2^-52 with m the top 52 bits of
(r_hi << 32 | r_lo), so u lies strictly inside (0, 1) and is exact.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85

SQRT_HALF = 0.7071067811865476
LN2 = 0.6931471805599453
HALF_PI = 1.5707963267948966
LOG_TERMS = 12          # coefficients 1/1, 1/3, ..., 1/23
TRIG_TERMS = 9          # sin: 1, -1/3!, ..., 1/17!;  cos: 1, -1/2!, ..., 1/16!


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit counters; returns 4 uint64 arrays < 2^32."""
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3)]
    b = np.broadcast_arrays(*c)
    c = [np.array(x, dtype=np.uint64) for x in b]
    key0 = int(k0) & 0xFFFFFFFF
    key1 = int(k1) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            key0 = (key0 + _W0) & 0xFFFFFFFF
            key1 = (key1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(key0), lo1, hi0 ^ c[3] ^ np.uint64(key1), lo0]
    return c


def uniform52(hi, lo):
    """(m + 0.5) * 2^-52 with m = top 52 bits of the 64-bit word hi:lo (exact in binary64)."""
    word = (np.asarray(hi, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo, dtype=np.uint64)
    m = word >> np.uint64(12)
    return (m.astype(np.float64) + 0.5) * (2.0 ** -52)


def _log_coefficients():
    return [1.0 / float(2 * k + 1) for k in range(LOG_TERMS)]


def _sin_coefficients():
    s = [1.0]
    for k in range(1, TRIG_TERMS):
        s.append(s[-1] / (-float((2 * k) * (2 * k + 1))))
    return s


def _cos_coefficients():
    c = [1.0]
    for k in range(1, TRIG_TERMS):
        c.append(c[-1] / (-float((2 * k - 1) * (2 * k))))
    return c


def series_log(u):
    """Natural log of u in (0, 1] by the atanh series (elementwise, no FMA)."""
    u = np.asarray(u, dtype=np.float64)
    m, e = np.frexp(u)
    low = m < SQRT_HALF
    m = np.where(low, m * 2.0, m)
    e = np.where(low, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    a = _log_coefficients()
    s = np.full_like(t, a[-1])
    for k in range(LOG_TERMS - 2, -1, -1):
        s = s * t2 + a[k]
    return e * LN2 + 2.0 * (t * s)


def series_sincos_turn(u2):
    """(cos, sin) of 2 pi u2 for u2 in [0, 1) by quarter-turn reduction and Taylor series."""
    u2 = np.asarray(u2, dtype=np.float64)
    q = 4.0 * u2
    k = np.floor(q)
    f = q - k
    flip = f > 0.5
    r = np.where(flip, 1.0 - f, f) * HALF_PI
    r2 = r * r
    sc, cc = _sin_coefficients(), _cos_coefficients()
    ps = np.full_like(r, sc[-1])
    for j in range(TRIG_TERMS - 2, 0, -1):
        ps = ps * r2 + sc[j]
    sin_r = r + (r * r2) * ps
    pc = np.full_like(r, cc[-1])
    for j in range(TRIG_TERMS - 2, 0, -1):
        pc = pc * r2 + cc[j]
    cos_r = 1.0 + r2 * pc
    ct = np.where(flip, sin_r, cos_r)      # cos(f pi/2)
    st = np.where(flip, cos_r, sin_r)      # sin(f pi/2)
    ki = k.astype(np.int64)
    cos_phi = np.choose(ki, [ct, -st, -ct, st])
    sin_phi = np.choose(ki, [st, ct, -st, -ct])
    return cos_phi, sin_phi


def box_muller(u1, u2):
    rho = np.sqrt(-2.0 * series_log(u1))
    c, s = series_sincos_turn(u2)
    return rho * c, rho * s


def _counter_words(step, stream):
    step = int(step)
    return step & 0xFFFFFFFF, ((step >> 32) & 0xFFFF) | (int(stream) << 16)


def normals(seed, step, nwalkers, naux, stream=0):
    """Fields x[w, gamma] ~ N(0,1), shape [nwalkers, naux] (Eq. 8's p(x))."""
    npairs = (naux + 1) // 2
    j = np.arange(npairs, dtype=np.uint64)[None, :]
    w = np.arange(nwalkers, dtype=np.uint64)[:, None]
    c2, c3 = _counter_words(step, stream)
    r0, r1, r2, r3 = philox4x32_10(j, w, c2, c3, int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
    u1 = uniform52(r0, r1)
    u2 = uniform52(r2, r3)
    z0, z1 = box_muller(u1, u2)
    x = np.empty((nwalkers, 2 * npairs))
    x[:, 0::2] = z0
    x[:, 1::2] = z1
    return np.ascontiguousarray(x[:, :naux])


def comb_uniform(seed, step):
    """The comb offset xi in (0, 1): stream 1, counter (0, 0, step)."""
    c2, c3 = _counter_words(step, 1)
    r0, r1, _, _ = philox4x32_10(0, 0, c2, c3, int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
    return float(uniform52(r0, r1))
