"""Pins for the oracle's NTT / INTT (Section II-B) and root-of-unity choice.

The oracle's NTT is the textbook fast transform; these tests pin it to the
O(N^2) sum that defines it, to the convolution theorem (the reason the NTT is
used at all, Section II-B), and to its inverse.
"""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def ntt_definition(a, q, psi):
    """out[i] = sum_n a[n] psi^((2 brv(i) + 1) n) mod q, plain O(N^2) python ints."""
    N = len(a)
    bits = N.bit_length() - 1
    out = []
    for i in range(N):
        w = pow(psi, 2 * brv(i, bits) + 1, q)
        acc, wn = 0, 1
        for n in range(N):
            acc += int(a[n]) * wn
            wn = wn * w % q
        out.append(acc % q)
    return out


def negacyclic_conv(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - N] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


PRIME_CASES = [(16, 31), (64, 31), (256, 30), (256, 31), (1024, 31)]


@pytest.mark.parametrize("N,bits", PRIME_CASES)
def test_psi_is_primitive_2n_root_and_smallest_generator(N, bits):
    for q in inputs.ntt_primes(N, bits, 3):
        psi = oracle.psi(q, N)
        assert pow(psi, N, q) == q - 1          # psi^N = -1  -> order exactly 2N
        assert pow(psi, 2 * N, q) == 1
        # the rule: smallest g >= 2 with g^((q-1)/2N) of order 2N
        for g in range(2, 200):
            cand = pow(g, (q - 1) // (2 * N), q)
            if pow(cand, N, q) == q - 1:
                assert cand == psi
                break


@pytest.mark.parametrize("N,bits", [(16, 31), (64, 31), (256, 30), (256, 31)])
def test_ntt_matches_definition(N, bits):
    g = inputs.rng(1)
    primes = inputs.ntt_primes(N, bits, 2)
    a = inputs.uniform_residues(g, primes, N)
    got = oracle.ntt(a, primes)
    for i, q in enumerate(primes):
        assert list(got[i]) == ntt_definition(a[i], q, oracle.psi(q, N))


def test_ntt_edge_values():
    N = 64
    primes = inputs.ntt_primes(N, 31, 2)
    for q_i, q in enumerate(primes):
        for a in (np.zeros(N), np.full(N, q - 1), np.eye(1, N, 0)[0], np.eye(1, N, N - 1)[0]):
            a = a.astype(np.uint32)[None, :]
            got = oracle.ntt(a, [q])
            assert list(got[0]) == ntt_definition(a[0], q, oracle.psi(q, N))


@pytest.mark.parametrize("N,bits", [(16, 31), (128, 30), (256, 31)])
def test_convolution_theorem(N, bits):
    g = inputs.rng(2)
    primes = inputs.ntt_primes(N, bits, 2)
    a = inputs.uniform_residues(g, primes, N)
    b = inputs.uniform_residues(g, primes, N)
    prod = oracle.intt(oracle.mul(oracle.ntt(a, primes), oracle.ntt(b, primes), primes), primes)
    for i, q in enumerate(primes):
        assert list(prod[i]) == negacyclic_conv(a[i], b[i], q)


@pytest.mark.parametrize("N", [1 << 12, 1 << 16])
def test_intt_inverts_ntt(N):
    g = inputs.rng(3)
    primes = inputs.ntt_primes(N, 31, 3)
    a = inputs.uniform_residues(g, primes, N)
    assert np.array_equal(oracle.intt(oracle.ntt(a, primes), primes), a)
    assert np.array_equal(oracle.ntt(oracle.intt(a, primes), primes), a)


def test_ntt_linear_and_x_monomial():
    # NTT(X) at slot i is psi^(2 brv(i)+1): checks ordering at full size N = 2^12
    N = 1 << 12
    q = inputs.ntt_primes(N, 30, 1)[0]
    psi = oracle.psi(q, N)
    x = np.zeros((1, N), np.uint32)
    x[0, 1] = 1
    got = oracle.ntt(x, [q])[0]
    bits = 12
    for i in range(0, N, 97):
        assert int(got[i]) == pow(psi, 2 * brv(i, bits) + 1, q)


def test_twiddle_runs_factor_for_on_the_fly_generation():
    """The on-the-fly twiddles of the block passes rest on two identities: for a run of
    twiddle indices 2^s + t0 + k (t0 a multiple of 2^m, k < 2^m) the bits are disjoint, so
    psi^brv(2^s + t0 + k) = psi^brv(2^s + t0) psi^brv(k); and the Shoup companion of w is
    floor(w 2^32 / q) = w floor(2^32 / q) + floor(w (2^32 mod q) / q)."""
    g = inputs.rng(41)
    for N in (1 << 12, 1 << 16):
        logn = N.bit_length() - 1
        q = inputs.ntt_primes(N, 31, 2)[1]
        psi = oracle.psi(q, N)

        def brv(x):
            return int(format(x, f"0{logn}b")[::-1], 2)

        for _ in range(200):
            m = int(g.integers(0, 4))
            s = int(g.integers(m + 4, logn))
            t0 = int(g.integers(0, 1 << (s - m))) << m
            k = int(g.integers(0, 1 << m))
            lhs = pow(psi, brv((1 << s) + t0 + k), q)
            rhs = pow(psi, brv((1 << s) + t0), q) * pow(psi, brv(k), q) % q
            assert lhs == rhs
            w = int(g.integers(0, q))
            assert (w << 32) // q == w * ((1 << 32) // q) + (w * ((1 << 32) % q)) // q
