"""The integer arithmetic that the tensor-core BJ_ext apply is built on
(error-free splitting of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59,
2012), written out with Python integers and checked against exact rational
arithmetic: the balanced base-256 digits reproduce every value, every level
sum of digit-plane products stays an exact FP32 integer (below 2^24), and the
recombination rounds the exact digit product once.  The GPU kernel is checked
against the oracle and the FP64 CUDA-core apply by tests/test_gpu_pc_tc.py;
this test pins the exactness bounds and the rounding its design relies on."""
import math
import random
import struct
from fractions import Fraction

import numpy as np

M64 = (1 << 64) - 1
NDIG, NLEV = 8, 9


def biased_exp(v):
    e = (struct.unpack("<Q", struct.pack("<d", v))[0] >> 52) & 0x7FF
    return e if e else 1


def to_int(v, E):
    """v = T 2^(E - 1084), |T| < 2^62 (truncated below 2^-9 of the largest)."""
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    ex, frac = (b >> 52) & 0x7FF, b & ((1 << 52) - 1)
    mant = (frac | (1 << 52)) if ex else frac
    sh = (ex if ex else 1) - E + 9
    T = (mant << sh) if sh >= 0 else (mant >> (-sh) if sh > -64 else 0)
    return -T if b >> 63 else T


def digits(T):
    """Balanced base-256 digits, top first: the seven low bytes after adding
    128 to each, minus 128; the top byte signed."""
    Tp = (T + 0x0080808080808080) & M64
    top = (Tp >> 56) & 0xFF
    d = [top - 256 if top >= 128 else top]
    for b in range(1, NDIG):
        d.append(((Tp >> (8 * (7 - b))) & 0xFF) - 128)
    return d


def recombine(qh, ql, sh):
    """(qh 2^40 + ql) 2^sh rounded once (128-bit integer, leading 64 bits with
    a sticky bit, round to nearest even)."""
    alo = (qh << 40) & M64
    lo = (alo + (ql & M64)) & M64
    hi = (qh >> 24) + (ql >> 63) + (1 if lo < alo else 0)
    neg = hi < 0
    if neg:
        lo = (~lo + 1) & M64
        hi = ~hi + (1 if lo == 0 else 0)
    m = lo
    if hi:
        lz = 64 - hi.bit_length()
        m = ((hi << lz) & M64) | (lo >> (64 - lz)) | (1 if (lo << lz) & M64 else 0)
        sh += 64 - lz
    y = math.ldexp(float(m), sh)       # float(int) rounds to nearest even
    return -y if neg else y


def digit_product(P, x):
    """y = P x through digit planes: per level the exact integer sums (as an
    FP32 tensor-core accumulator would hold them), then one rounding."""
    n = P.shape[1]
    EX = max(biased_exp(v) for v in x)
    xd = [digits(to_int(v, EX)) for v in x]
    y, dmax = [], 0
    for p in range(P.shape[0]):
        EP = max(biased_exp(v) for v in P[p])
        pd = [digits(to_int(v, EP)) for v in P[p]]
        D = []
        for L in range(NLEV):
            s = sum(pd[k][a] * xd[k][L - a] for a in range(max(0, L - 7), min(7, L) + 1) for k in range(n))
            dmax = max(dmax, abs(s))
            D.append(s)
        qh = D[0] * 2 ** 24 + D[1] * 2 ** 16 + D[2] * 2 ** 8 + D[3]
        ql = D[4] * 2 ** 32 + D[5] * 2 ** 24 + D[6] * 2 ** 16 + D[7] * 2 ** 8 + D[8]
        y.append(recombine(qh, ql, EP + EX - 2120))
    return np.array(y), dmax


def test_digits_reproduce_every_value():
    rng = random.Random(5)
    for t in range(20000):
        T = rng.randint(-2 ** 62 + 1, 2 ** 62 - 1) if t > 8 else [0, 1, -1, 127, -128, 128, 255, -255,
                                                                   2 ** 62 - 1][t]
        d = digits(T)
        assert all(-128 <= v <= 127 for v in d[1:]) and -65 <= d[0] <= 65
        assert sum(v * 256 ** (7 - b) for b, v in enumerate(d)) == T


def test_digit_product_is_exact_per_level_and_rounded_once():
    rng = np.random.default_rng(1)
    n2 = 72                                     # 2 n_b for n_b = 36
    for trial in range(3):
        P = rng.standard_normal((n2, n2)) * np.exp(rng.uniform(-8, 8, (n2, 1))) * np.exp(rng.uniform(-3, 3, (1, n2)))
        x = rng.standard_normal(n2) * np.exp(rng.uniform(-3, 3, n2)) * 10.0 ** rng.uniform(-5, 5)
        y, dmax = digit_product(P, x)
        assert dmax < 2 ** 24                    # every level sum is an exact FP32 integer
        exact = np.array([float(sum(Fraction(P[p, k]) * Fraction(x[k]) for k in range(n2))) for p in range(n2)])
        scale = np.abs(P) @ np.abs(x)
        assert np.max(np.abs(y - exact) / scale) <= 2.0 ** -60
        assert np.max(np.abs(P @ x - exact) / scale) > 2.0 ** -60   # FP64's own product is less exact


def test_recombination_rounds_correctly():
    rng = random.Random(3)
    for _ in range(50000):
        qh, ql = rng.randint(-2 ** 43, 2 ** 43), rng.randint(-2 ** 56, 2 ** 56)
        assert recombine(qh, ql, 0) == float(Fraction(qh * 2 ** 40 + ql))
