"""Pins of the oracle's point sets (Sec. 2.4: low-discrepancy points in the MC maps).

Each check rests on something other than the oracle itself: a published generator output, a
number-theoretic count, the binary structure of van der Corput / Pascal matrices, or brute
force counting of points in elementary intervals.
"""
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def test_splitmix64_reference_output(orc):
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        seed, idx, out = line.split()
        state = (int(seed) + (int(idx) + 1) * 0x9E3779B97F4A7C15) % 2 ** 64
        assert orc.mix64(state) == int(out, 16)


def _totient(n):
    r, m, p = n, n, 2
    while p * p <= m:
        if m % p == 0:
            while m % p == 0:
                m //= p
            r -= r // p
        p += 1
    if m > 1:
        r -= r // m
    return r


def _recover_polynomial(col):
    """Smallest degree s and taps a_1..a_{s-1} for which the 32 direction numbers obey the
    Bratley-Fox recurrence V_j = V_{j-s} ^ (V_{j-s} >> s) ^ XOR_k a_k V_{j-k} for all j > s;
    returns the polynomial value x^s + a_1 x^{s-1} + ... + a_{s-1} x + 1."""
    for s in range(1, 12):
        for taps in range(2 ** (s - 1)):
            ok = True
            for j in range(s + 1, 33):
                x = col[j - s - 1] ^ (col[j - s - 1] >> s)
                for k in range(1, s):
                    if (taps >> (s - 1 - k)) & 1:
                        x ^= col[j - k - 1]
                if x != col[j - 1]:
                    ok = False
                    break
            if ok:
                return s, (1 << s) | (taps << 1) | 1
    return None


def _order_of_x(p, s):
    r = 1
    for k in range(1, 2 ** s):
        r <<= 1
        if (r >> s) & 1:
            r ^= p
        if r == 1:
            return k
    return -1


def test_primitive_polynomials(orc):
    # Dimension d >= 1 must use the d-th primitive polynomial over GF(2) in increasing
    # (degree, value) order. Recover each dimension's polynomial from its direction numbers,
    # check it is primitive (x has order 2^s - 1), that the list is increasing, and that every
    # degree contributes phi(2^s - 1)/s polynomials (Euler's totient count).
    V = orc.sobol_table(65)
    polys = []
    for d in range(1, 65):
        col = [int(v) for v in V[d]]
        s, p = _recover_polynomial(col)
        assert _order_of_x(p, s) == 2 ** s - 1
        polys.append((s, p))
    assert polys == sorted(polys) and len(set(polys)) == len(polys)
    for s in range(1, 9):
        assert sum(1 for q in polys if q[0] == s) == _totient(2 ** s - 1) // s
    for d in range(65):
        for b in range(32):
            col = int(V[d, b])
            assert (col >> (31 - b)) & 1 == 1          # unit diagonal: m_j odd
            assert col & ((1 << (31 - b)) - 1) == 0    # upper triangular: m_j < 2^j


def test_dim0_is_van_der_corput(orc):
    n = 4096
    x = orc.points(0, 0, 0, 0, 0, n, 1)[:, 0]
    shift = orc.points(0, 0, 0, 0, 0, 1, 1)[0, 0]     # point 0 = the digital shift itself
    raw = x ^ shift
    rev = np.array([int(f"{i:032b}"[::-1], 2) for i in range(n)], dtype=np.uint64)
    assert np.array_equal(raw.astype(np.uint64), rev)


def test_dim1_is_pascal_matrix(orc):
    # Sobol dimension from x + 1 with m_1 = 1: the generator is Pascal's triangle mod 2,
    # C[r][b] = binom(b, r) mod 2 (row r = bit 31 - r of column b).
    V = orc.sobol_table(2)
    for b in range(32):
        for r in range(32):
            assert ((int(V[1, b]) >> (31 - r)) & 1) == (math.comb(b, r) % 2)


@pytest.mark.parametrize("m", [1, 4, 8, 12])
def test_one_dimensional_stratification(orc, m):
    # The first 2^m points of every dimension put exactly one point in each interval
    # [j 2^-m, (j+1) 2^-m); an XOR digital shift permutes those intervals, so this holds shifted.
    n = 2 ** m
    P = orc.points(12345, 3, 2, 0, 0, n, 65)
    top = P >> np.uint32(32 - m)
    for d in range(65):
        assert np.array_equal(np.sort(top[:, d]), np.arange(n))


def test_pair_nets_brute_force(orc):
    # (dim 0, dim 1) is a (0,2)-sequence: every elementary interval of volume 2^-m of the first
    # 2^m points holds exactly one point, counted by brute force.
    for m in range(1, 11):
        n = 2 ** m
        P = orc.points(7, 1, 1, 0, 0, n, 2).astype(np.uint64)
        for k in range(m + 1):
            a = P[:, 0] >> np.uint64(32 - k) if k else np.zeros(n, np.uint64)
            b = P[:, 1] >> np.uint64(32 - (m - k)) if m - k else np.zeros(n, np.uint64)
            key = a * np.uint64(2 ** (m - k)) + b
            assert len(np.unique(key)) == n


def test_digital_shift_is_xor(orc):
    # Two shifts of one Sobol set differ by a per-dimension constant XOR.
    A = orc.points(1, 5, 2, 0, 0, 1000, 17)
    B = orc.points(2, 9, 3, 0, 0, 1000, 17)
    D = A ^ B
    assert np.all(D == D[0:1, :])
    # random access: a later index range equals the corresponding rows
    C = orc.points(1, 5, 2, 0, 300, 100, 17)
    assert np.array_equal(C, A[300:400])


def test_prng_uniformity(orc):
    P = orc.points(3, 0, 2, 1, 0, 200_000, 4)
    for d in range(4):
        h = np.bincount((P[:, d] >> np.uint32(28)).astype(np.int64), minlength=16)
        chi2 = float(np.sum((h - h.mean()) ** 2 / h.mean()))
        assert chi2 < 50.0            # 15 dof; p ~ 1e-5 tail
    # distinct (i, d) give distinct values (no accidental sharing of the hash)
    assert len(np.unique(P[:1000].ravel())) > 3990


@pytest.mark.parametrize("mode,tol_sc", [(1, 3e-16), (0, 1.2e-15)], ids=["series", "libm"])
def test_direction_and_depth_maps_accuracy(orc, mode, tol_sc):
    # both evaluations of sin/cos(2 pi u) and -log u against 40-digit arithmetic over the point
    # lattice, including the quadrant boundaries and u -> 0, 1. The libm mode rounds the argument
    # 2 pi u first (an absolute error up to half an ulp of 2 pi, 4.4e-16), then libm's own error;
    # the series mode reduces u exactly first.
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    x = np.concatenate([np.arange(0, 2 ** 32, 2 ** 32 // 2003, dtype=np.uint64),
                        np.array([0, 1, 2 ** 30 - 1, 2 ** 30, 2 ** 31, 3 * 2 ** 30, 2 ** 32 - 1], np.uint64)])
    u = (x.astype(np.float64) + 0.5) * 2.0 ** -32
    s, c = orc.sincos_2pi(u, elem=mode)
    t = orc.neg_log(u, elem=mode)
    for i in range(u.size):
        a = 2 * mpmath.pi * mpmath.mpf(float(u[i]))
        assert abs(s[i] - float(mpmath.sin(a))) < tol_sc
        assert abs(c[i] - float(mpmath.cos(a))) < tol_sc
        ref = -mpmath.log(mpmath.mpf(float(u[i])))
        assert abs(t[i] - float(ref)) <= 3e-16 * abs(float(ref))


def test_elementary_modes_are_distinct_evaluations(orc):
    # the two modes evaluate the same maps (agreement to rounding) by different operations (they
    # differ in the last bits somewhere), and the module default is libm
    u = (np.arange(0, 2 ** 32, 2 ** 32 // 4001, dtype=np.uint64).astype(np.float64) + 0.5) * 2.0 ** -32
    s0, c0 = orc.sincos_2pi(u, elem=orc.LIBM)
    s1, c1 = orc.sincos_2pi(u, elem=orc.SERIES)
    t0, t1 = orc.neg_log(u, elem=orc.LIBM), orc.neg_log(u, elem=orc.SERIES)
    assert np.max(np.abs(s0 - s1)) < 2e-15 and np.max(np.abs(c0 - c1)) < 2e-15
    assert np.max(np.abs(t0 - t1) / t0) < 6e-16
    assert np.any(s0 != s1) and np.any(c0 != c1)
    sd, cd = orc.sincos_2pi(u)
    assert np.array_equal(sd, s0) and np.array_equal(cd, c0)


# ---------------------------------------------------------------------------------------------
# Halton points with a shift modulo 1 (sampler 2)
# ---------------------------------------------------------------------------------------------
HALTON = 2


def _primes(n):
    out, c = [], 2
    while len(out) < n:
        if all(c % q for q in range(2, int(math.isqrt(c)) + 1)):
            out.append(c)
        c += 1
    return out


def _unshifted(orc, i0, n, ndims, seed=1, step=0, stream=0):
    """Halton coordinates minus the shift: point 0 is the origin, so its value is the shift."""
    u = orc.points(seed, step, stream, HALTON, i0, n, ndims).astype(np.int64)
    s = orc.points(seed, step, stream, HALTON, 0, 1, ndims).astype(np.int64)[0]
    return (u - s) % 2 ** 32


def test_halton_primes():
    p = _primes(65)
    assert p[:10] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29] and p[64] == 313   # the 65th prime is 313


def test_halton_radical_inverse_exact(orc):
    """floor(2^32 phi_b(i)) against the radical inverse in exact rational arithmetic."""
    from fractions import Fraction
    primes = _primes(65)
    dims = [0, 1, 2, 5, 17, 40, 64]
    idx = list(range(0, 300)) + [4095, 4096, 59049, 12345678, 2 ** 31 - 1, 2 ** 32 - 1]
    for i in idx:
        got = _unshifted(orc, i, 1, 65)[0]
        for d in dims:
            b, n, phi, k = primes[d], i, Fraction(0), 1
            while n:
                phi += Fraction(n % b, b ** k)
                n //= b
                k += 1
            assert got[d] == math.floor(phi * 2 ** 32), (i, d)


def test_halton_matches_scipy_unscrambled(orc):
    """The unscrambled Halton sequence of scipy.stats.qmc (index 0 first) to within FP64 rounding."""
    qmc = pytest.importorskip("scipy.stats.qmc")
    ref = qmc.Halton(d=65, scramble=False).random(2048)
    got = _unshifted(orc, 0, 2048, 65) / 2.0 ** 32
    assert np.max(np.abs(got - ref)) < 2.0 ** -31


@pytest.mark.parametrize("d", [0, 1, 2, 3, 6, 20, 64])
def test_halton_first_b_to_the_k_points_are_a_grid(orc, d):
    """Van der Corput in base b: points 0 .. b^k - 1 are the grid {j / b^k} in some order."""
    b = _primes(65)[d]
    k = 1
    while b ** (k + 1) <= 4096:
        k += 1
    m = b ** k
    u = np.sort(_unshifted(orc, 0, m, 65)[:, d])
    assert np.array_equal(u, [(j << 32) // m for j in range(m)])


def test_halton_shift_is_modular_and_shared(orc):
    """The randomisation adds one 32-bit value per dimension modulo 2^32 (the same value as the
    Sobol set's digital shift of that point set), so differences between points do not depend on
    the seed."""
    a = _unshifted(orc, 0, 512, 65, seed=3)
    b = _unshifted(orc, 0, 512, 65, seed=99, step=7, stream=2)
    assert np.array_equal(a, b)
    for seed, step, stream in ((3, 0, 0), (99, 7, 2)):
        h0 = orc.points(seed, step, stream, HALTON, 0, 1, 65)[0]
        s0 = orc.points(seed, step, stream, 0, 0, 1, 65)[0]
        assert np.array_equal(h0, s0)
    # past the 65 tabulated dimensions both fall back to the counter PRNG
    assert np.array_equal(orc.points(5, 1, 1, HALTON, 10, 50, 70)[:, 65:], orc.points(5, 1, 1, 1, 10, 50, 70)[:, 65:])


def test_halton_planted_mistakes_fail():
    """The exact-rational check separates the radical inverse from its usual slips (digits read in
    the wrong order, a dropped digit, the wrong base)."""
    from fractions import Fraction

    def phi(i, b):
        r, n, k = Fraction(0), i, 1
        while n:
            r += Fraction(n % b, b ** k)
            n //= b
            k += 1
        return r

    def forward_digits(i, b):      # digits not reversed
        ds = []
        while i:
            ds.append(i % b)
            i //= b
        return sum(Fraction(a, b ** (len(ds) - j)) for j, a in enumerate(ds))

    assert any(phi(i, 3) != forward_digits(i, 3) for i in range(1, 30))
    assert any(phi(i, 5) != phi(i, 7) for i in range(1, 30))
    assert any(phi(i, 3) != phi(i // 3, 3) for i in range(1, 30))
