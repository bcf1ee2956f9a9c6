"""The tensor-core base conversion's integer encoding, replayed on the CPU.

The kernel computes sum_j y_j T[o][j] mod p_o (Section II-B BConv) with f16
MMA operands: A holds 1024 + byte for the four bytes of every input (built
with two byte permutes against 0x64006400), B holds the bytes of
(2^(8a) T[o][j]) mod p_o, and four extra K slots (A = 1024, B = pieces <= 2048
of 8192 - row sum) make every fp32 accumulator exactly 2^23 + S_b.  This
model checks, in exact integers, every step the exactness argument relies on:
the f16 bit patterns, the nonnegativity of all terms, the 2^24 bound on every
partial sum, the accumulator's bit pattern, and the epilogue's reduction,
against the plain definition of the sum, for random and worst-case inputs.
Digits of 9..12 limbs use a K = 64 shape whose offset pieces may be negative;
`conversion12` checks that every partial sum still stays inside (-2^24, 2^24)."""
import struct

import numpy as np
import pytest

K_DATA, K_TOTAL = 32, 48
# digits of 9..12 limbs: K = 64, 48 data slots, 8 offset slots with signed B pieces
K_DATA12, K_TOTAL12 = 48, 64


def byte_perm(x: int, y: int, s: int) -> int:
    b = [(x >> (8 * i)) & 0xFF for i in range(4)] + [(y >> (8 * i)) & 0xFF for i in range(4)]
    return sum(b[(s >> (4 * i)) & 7] << (8 * i) for i in range(4))


def f16_value(h: int) -> float:
    return float(np.frombuffer(struct.pack("<H", h), dtype=np.float16)[0])


def f16_int(v: int) -> int:
    """f16 bit pattern of an integer -2048 <= v <= 2048 (the table builder's rule)."""
    if v == 0:
        return 0
    sign = 0x8000 if v < 0 else 0
    v = abs(v)
    e = v.bit_length() - 1
    mant = ((v << (10 - e)) & 0x3FF) if e <= 10 else ((v >> (e - 10)) & 0x3FF)
    return sign | ((e + 15) << 10) | mant


def f32_bits(x: int) -> int:
    return struct.unpack("<I", struct.pack("<f", np.float32(x)))[0]


def shoup_lazy(a: int, w: int, ws: int, q: int) -> int:
    return (a * w - ((a * ws) >> 32) * q) & 0xFFFFFFFF


def red2(x: int, q: int) -> int:
    return min(x, (x - q) & 0xFFFFFFFF)


def conversion(y, T, p):
    """One output of the kernel: A row, B rows (4 weights), accumulators, epilogue."""
    n_in = len(y)
    A = [0] * K_TOTAL
    for j in range(8):
        yj = y[j] if j < n_in else 0
        w0, w1 = byte_perm(yj, 0x64006400, 0x7150), byte_perm(yj, 0x64006400, 0x7352)
        for idx, h in enumerate((w0 & 0xFFFF, w0 >> 16, w1 & 0xFFFF, w1 >> 16)):
            A[4 * j + idx] = f16_value(h)
    for e in range(4):
        A[K_DATA + e] = 1024.0
    acc = []
    for b in range(4):
        B = [0.0] * K_TOTAL
        for j in range(n_in):
            for a in range(4):
                ta = (T[j] << (8 * a)) % p
                B[4 * j + a] = f16_value(f16_int((ta >> (8 * b)) & 0xFF))
        rest = 8192 - int(sum(B[:K_DATA]))
        assert rest >= 0  # row sum <= 32 * 255 = 8160
        for e in range(4):
            piece = min(rest, 2048)
            B[K_DATA + e] = f16_value(f16_int(piece))
            rest -= piece
        terms = [int(x) * int(z) for x, z in zip(A, B)]
        assert all(t >= 0 for t in terms)          # every partial sum lies in [0, total]
        total = sum(terms)
        assert total < 2 ** 24                      # so fp32 accumulation is exact in any order
        acc.append(f32_bits(total))
    s_b = [u - 0x4B000000 for u in acc]             # the bits hold 2^23 + S_b
    assert all(0 <= s < 2 ** 21 for s in s_b)
    lo = (acc[1] * 256 + acc[0] - 0x4B000000) & 0xFFFFFFFF
    hi = (acc[3] * 256 + acc[2] - 0x4B000000) & 0xFFFFFFFF
    assert lo < 2 ** 30 and hi < 2 ** 30
    w16s = (65536 << 32) // p
    s = lo + red2(shoup_lazy(hi, 65536, w16s, p), p)
    assert s < 2 ** 32
    return red2(s, p) if p > 2 ** 30 else red2(shoup_lazy(s, 1, (1 << 32) // p, p), p)


def conversion12(y, T, p):
    """The K = 64 shape (up to 12 inputs): the offset pieces may be negative, so the exactness
    argument is that every partial sum, in any order, lies between the sum of the negative
    terms and the sum of the positive ones, both inside (-2^24, 2^24)."""
    n_in = len(y)
    assert n_in <= 12
    A = [0.0] * K_TOTAL12
    for j in range(12):
        yj = y[j] if j < n_in else 0
        w0, w1 = byte_perm(yj, 0x64006400, 0x7150), byte_perm(yj, 0x64006400, 0x7352)
        for idx, h in enumerate((w0 & 0xFFFF, w0 >> 16, w1 & 0xFFFF, w1 >> 16)):
            A[4 * j + idx] = f16_value(h)
    for e in range(8):
        A[K_DATA12 + e] = 1024.0
    acc = []
    for b in range(4):
        B = [0.0] * K_TOTAL12
        for j in range(n_in):
            for a in range(4):
                ta = (T[j] << (8 * a)) % p
                B[4 * j + a] = f16_value(f16_int((ta >> (8 * b)) & 0xFF))
        rest = 8192 - int(sum(B[:K_DATA12]))
        for e in range(4):
            piece = max(-2048, min(rest, 2048))
            B[K_DATA12 + e] = f16_value(f16_int(piece))
            rest -= piece
        assert rest == 0
        terms = [int(x) * int(z) for x, z in zip(A, B)]
        neg = sum(t for t in terms if t < 0)
        pos = sum(t for t in terms if t > 0)
        assert -2 ** 24 < neg and pos < 2 ** 24     # every partial sum is an exact fp32 integer
        total = sum(terms)
        assert 2 ** 23 <= total < 2 ** 24
        acc.append(f32_bits(total))
    s_b = [u - 0x4B000000 for u in acc]
    assert all(0 <= s < 2 ** 22 for s in s_b)
    lo = (acc[1] * 256 + acc[0] - 0x4B000000) & 0xFFFFFFFF
    hi = (acc[3] * 256 + acc[2] - 0x4B000000) & 0xFFFFFFFF
    assert lo < 2 ** 30 + 2 ** 22 and hi < 2 ** 30 + 2 ** 22
    w16s = (65536 << 32) // p
    s = lo + red2(shoup_lazy(hi, 65536, w16s, p), p)
    assert s < 2 ** 32
    big = p > 2 ** 30 + 2 ** 23
    if big:
        assert s < 2 * p                             # one conditional subtraction suffices
    return red2(s, p) if big else red2(shoup_lazy(s, 1, (1 << 32) // p, p), p)


def test_f16_patterns():
    for v in range(-2048, 2049):
        assert f16_value(f16_int(v)) == v
    for b in range(256):
        assert f16_value(0x6400 | b) == 1024 + b
    assert f32_bits(2 ** 23 + 12345) == 0x4B000000 + 12345


# primes of the workloads' sizes: 31-bit NTT-friendly (2^31 - k 2^17 + 1), a 30-bit
# one, and a 22-bit one (the library accepts primes above 2^20)
PRIMES = [2147352577, 2146959361, 2013265921, 1073479681, 2236417]


@pytest.mark.parametrize("p", PRIMES)
def test_random_and_extreme_conversions(p):
    rng = np.random.default_rng(p)
    for trial in range(60):
        n_in = int(rng.integers(1, 9))
        if trial % 3 == 0:
            T = [p - 1] * n_in
        else:
            T = [int(t) for t in rng.integers(0, p, n_in)]
        if trial % 4 == 0:
            y = [2 ** 31 - 1] * n_in      # larger than any residue: the bound still holds
        else:
            y = [int(v) for v in rng.integers(0, p, n_in)]
        assert conversion(y, T, p) == sum(a * b for a, b in zip(y, T)) % p


@pytest.mark.parametrize("p", PRIMES)
def test_wide_digit_conversions(p):
    """9..12 inputs (K = 64): random, all-(p - 1) tables and inputs above every residue."""
    rng = np.random.default_rng(p + 12)
    for trial in range(60):
        n_in = int(rng.integers(9, 13)) if trial % 5 else int(rng.integers(1, 9))
        if trial % 3 == 0:
            T = [p - 1] * n_in
        else:
            T = [int(t) for t in rng.integers(0, p, n_in)]
        if trial % 4 == 0:
            y = [2 ** 31 - 1] * n_in
        else:
            y = [int(v) for v in rng.integers(0, p, n_in)]
        assert conversion12(y, T, p) == sum(a * b for a, b in zip(y, T)) % p


def test_wide_digit_worst_row_sums():
    """Row sums at both extremes: every table byte 255 (rest = 8192 - 12240 < 0) and every byte 0
    (rest = 8192): the offset pieces stay within [-2048, 2048] and the sums stay exact."""
    p = PRIMES[0]
    # T whose shifted residues have all bytes 0xFF is not constructible for every a, so check the
    # offset split and the bound on synthetic byte rows directly
    for row in ([255] * 48, [0] * 48, [255] * 24 + [0] * 24):
        rest = 8192 - sum(row)
        pieces = []
        for _ in range(4):
            piece = max(-2048, min(rest, 2048))
            pieces.append(piece)
            rest -= piece
        assert rest == 0 and all(-2048 <= x <= 2048 for x in pieces)
        A = [1024 + 255] * 48 + [1024] * 4
        terms = [a * b for a, b in zip(A, row + pieces)]
        assert sum(t for t in terms if t > 0) < 2 ** 24 and sum(t for t in terms if t < 0) > -2 ** 24
    assert conversion12([p - 1] * 12, [p - 1] * 12, p) == (12 * (p - 1) * (p - 1)) % p
