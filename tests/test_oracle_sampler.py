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


def test_direction_and_depth_maps_accuracy(orc):
    # the series evaluations of sin/cos(2 pi u) and -log u against 40-digit arithmetic over the
    # point lattice, including the quadrant boundaries and u -> 0, 1
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    x = np.concatenate([np.arange(0, 2 ** 32, 2 ** 32 // 2003, dtype=np.uint64),
                        np.array([0, 1, 2 ** 30 - 1, 2 ** 30, 2 ** 31, 3 * 2 ** 30, 2 ** 32 - 1], np.uint64)])
    u = (x.astype(np.float64) + 0.5) * 2.0 ** -32
    s, c = orc.sincos_2pi(u)
    t = orc.neg_log(u)
    for i in range(u.size):
        a = 2 * mpmath.pi * mpmath.mpf(float(u[i]))
        assert abs(s[i] - float(mpmath.sin(a))) < 3e-16
        assert abs(c[i] - float(mpmath.cos(a))) < 3e-16
        ref = -mpmath.log(mpmath.mpf(float(u[i])))
        assert abs(t[i] - float(ref)) <= 3e-16 * abs(float(ref))
