"""Pins for the oracle's fast base conversion (Section II-B "BConv",
Section III-C table T[i][j] = (Q*/Q_j) mod P_i).

Fast base conversion is approximate by a known multiple of the input modulus:
for x = CRT(inputs) in [0, Q*), every output equals (x + e Q*) mod p_i with one
integer e in [0, n_in) shared by all output primes of that coefficient.  The
tests recover x and e with Python big integers and check exactly that.
"""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs


def check_bconv(x, q_in, p_out, out):
    Qs = 1
    for q in q_in:
        Qs *= q
    xs = oracle.crt(x, q_in, centered=False)
    n_in = len(q_in)
    for n in range(x.shape[1]):
        e_found = None
        for e in range(n_in):
            if all(int(out[i, n]) == (xs[n] + e * Qs) % p for i, p in enumerate(p_out)):
                e_found = e
                break
        assert e_found is not None, f"column {n}: no e in [0,{n_in}) fits"


@pytest.mark.parametrize("n_in,n_out", [(1, 3), (2, 4), (8, 24), (8, 8), (3, 5)])
def test_bconv_crt_multiple_of_q(n_in, n_out):
    N = 64
    primes = inputs.ntt_primes(1 << 16, 31, n_in + n_out)
    q_in, p_out = primes[:n_in], primes[n_in:]
    g = inputs.rng(10 + n_in)
    x = inputs.uniform_residues(g, q_in, N)
    out = oracle.bconv(x, q_in, p_out)
    check_bconv(x, q_in, p_out, out)


@pytest.mark.parametrize("fill", ["zero", "max", "one"])
def test_bconv_extreme_inputs(fill):
    N = 16
    primes = inputs.ntt_primes(1 << 16, 31, 16)
    q_in, p_out = primes[:8], primes[8:]
    if fill == "zero":
        x = np.zeros((8, N), np.uint32)
    elif fill == "max":
        x = np.array([[q - 1] * N for q in q_in], np.uint32)
    else:
        x = np.ones((8, N), np.uint32)
    out = oracle.bconv(x, q_in, p_out)
    check_bconv(x, q_in, p_out, out)
    if fill == "zero":
        assert not out.any()


def test_bconv_exact_for_small_values():
    # x < min(q) in every residue and equal across limbs -> it is the integer x itself,
    # and x * qhat_inv * qhat sums to x + e Q*;  for x = 0 the result is exactly 0,
    # and for a single input prime the conversion is exact (e = 0): out = x mod p.
    N = 32
    primes = inputs.ntt_primes(1 << 12, 30, 4)
    g = inputs.rng(5)
    x = inputs.uniform_residues(g, primes[:1], N)
    out = oracle.bconv(x, primes[:1], primes[1:])
    for i, p in enumerate(primes[1:]):
        assert np.array_equal(out[i], x[0].astype(np.uint64) % p)


def test_paper_overflow_example():
    # Section III-C: with L_in = 12 word-sized moduli Q_j ~ 2^31 the 64-bit
    # accumulator can reach 3 * 2^64 (12 products of two 2^31 values).
    assert 12 * (2 ** 31) * (2 ** 31) == 3 * 2 ** 64
