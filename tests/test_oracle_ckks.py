"""CKKS-level pins for the oracle: encoding against the slot definition, and
decryption of rotated / multiplied / transformed ciphertexts against FP64
plaintext arithmetic.

Tolerance for key-switched results: 2^-3 on the max slot error at N = 2^12,
scale 2^25.  The paper gives no bound for these operations, so this is a
heuristic, not a derived bound: most slots land near 2^-10, but the textbook
(non-centred) ModUp output has mean about D_j / 2 per coefficient, so the key
error it multiplies piles up in the lowest-frequency slot (slot 0), which was
observed at 2^-5 .. 2^-4.  Exactness of every residue is pinned elsewhere;
these tests catch gross errors (a wrong automorphism or gadget gives O(1)).
"""
import cmath

import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

TOL = 2.0 ** -3


def cfg1():
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    return oracle.OracleParams.from_params(P)


def test_decode_matches_slot_definition():
    N = 16
    g = inputs.rng(1)
    m = g.integers(-1000, 1000, size=N)
    got = oracle.decode(m, 1.0, N)
    for j in range(N // 2):
        e = pow(5, j, 2 * N)
        z = sum(int(m[n]) * cmath.exp(1j * cmath.pi * e * n / N) for n in range(N))
        assert abs(got[j] - z) < 1e-9 * (1 + abs(z))


def test_encode_decode_roundtrip():
    N = 1 << 12
    g = inputs.rng(2)
    z = inputs.complex_slots(g, N // 2)
    m = oracle.encode(z, 2.0 ** 25, N)
    assert np.abs(oracle.decode(m, 2.0 ** 25, N) - z).max() < 2.0 ** -12


def test_encoding_is_ring_homomorphism():
    N = 64
    g = inputs.rng(3)
    z1, z2 = inputs.complex_slots(g, N // 2), inputs.complex_slots(g, N // 2)
    d = 2.0 ** 20
    m1, m2 = oracle.encode(z1, d, N), oracle.encode(z2, d, N)
    prod = oracle.negacyclic_mul_int(m1, m2)
    assert np.abs(oracle.decode(prod, d * d, N) - z1 * z2).max() < 1e-4


def test_encrypt_decrypt_exact_error():
    P = cfg1()
    g = inputs.rng(4)
    sk = oracle.SecretKey(P, inputs.ternary(g, P.N))
    m = g.integers(-(1 << 40), 1 << 40, size=P.N)
    ct = oracle.encrypt(P, sk, m, 4, g)
    dec = oracle.decrypt(P, sk, ct, 4)
    assert max(abs(a - int(b)) for a, b in zip(dec, m)) <= inputs.ERR_BOUND


def test_automorph_ntt_matches_coefficient_definition():
    N = 1 << 10
    primes = inputs.ntt_primes(N, 31, 2)
    g = inputs.rng(5)
    a = inputs.uniform_residues(g, primes, N)
    for rot in (1, 3, 100, -1):
        k = oracle.galois_elt(rot, N)
        assert k == pow(5, rot % (N // 2), 2 * N)
        via_coef = oracle.ntt(oracle.automorph_coef(a, k, primes), primes)
        assert np.array_equal(oracle.automorph_ntt(oracle.ntt(a, primes), k), via_coef)
    # coefficient definition against an integer polynomial
    m = g.integers(-50, 50, size=N)
    k = oracle.galois_elt(7, N)
    assert np.array_equal(oracle.automorph_coef(oracle.to_rns(m, primes), k, primes),
                          oracle.to_rns(oracle.automorph_int(m, k), primes))


def _fresh(P, seed, level=4, scale=2.0 ** 25):
    g = inputs.rng(seed)
    sk = oracle.SecretKey(P, inputs.ternary(g, P.N))
    z = inputs.complex_slots(g, P.N // 2)
    ct = oracle.encrypt(P, sk, oracle.encode(z, scale, P.N), level, g)
    return g, sk, z, ct


def _dec(P, sk, ct, level, scale):
    return oracle.decode(oracle.decrypt(P, sk, ct, level), scale, P.N)


@pytest.mark.parametrize("rot", [1, 5, 1234])
def test_rotate_decodes_to_rolled_slots(rot):
    P = cfg1()
    g, sk, z, ct = _fresh(P, 10 + rot)
    key = oracle.rotation_key(P, sk, rot, g)
    out = oracle.rotate(P, ct, 4, rot, key)
    assert np.abs(_dec(P, sk, out, 4, 2.0 ** 25) - np.roll(z, -rot)).max() < TOL


def test_rotate_composes():
    P = cfg1()
    g, sk, z, ct = _fresh(P, 20)
    k3, k4 = oracle.rotation_key(P, sk, 3, g), oracle.rotation_key(P, sk, 4, g)
    out = oracle.rotate(P, oracle.rotate(P, ct, 4, 3, k3), 4, 4, k4)
    assert np.abs(_dec(P, sk, out, 4, 2.0 ** 25) - np.roll(z, -7)).max() < TOL


def test_hoisted_rotations():
    P = cfg1()
    g, sk, z, ct = _fresh(P, 30)
    rots = [0, 1, 2, 9]
    keys = [None] + [oracle.rotation_key(P, sk, r, g) for r in rots[1:]]
    outs = oracle.rotate_hoisted(P, ct, 4, rots, keys)
    for r, o in zip(rots, outs):
        assert np.abs(_dec(P, sk, o, 4, 2.0 ** 25) - np.roll(z, -r)).max() < TOL


def test_hmult_relin_rescale():
    P = cfg1()
    g = inputs.rng(40)
    sk = oracle.SecretKey(P, inputs.ternary(g, P.N))
    d = 2.0 ** 25
    z1, z2 = inputs.complex_slots(g, P.N // 2), inputs.complex_slots(g, P.N // 2)
    c1 = oracle.encrypt(P, sk, oracle.encode(z1, d, P.N), 4, g)
    c2 = oracle.encrypt(P, sk, oracle.encode(z2, d, P.N), 4, g)
    rk = oracle.relin_key(P, sk, g)
    m = oracle.hmult(P, c1, c2, 4, rk)
    assert np.abs(_dec(P, sk, m, 4, d * d) - z1 * z2).max() < TOL
    r = oracle.rescale(P, m, 4)
    assert np.abs(_dec(P, sk, r, 3, d * d / P.q[3]) - z1 * z2).max() < TOL


def test_bsgs_linear_transform_small():
    # sum_d diag_d (.) roll(z, d) for d = baby*g + b, diagonals pre-rotated by -baby*g
    P = cfg1()
    g, sk, z, ct = _fresh(P, 50)
    baby, giant = 4, 2
    d_scale = 2.0 ** 20
    nslots = P.N // 2
    diags = [inputs.complex_slots(g, nslots) for _ in range(baby * giant)]
    pdiags = []
    for gi in range(giant):
        for b in range(baby):
            dv = np.roll(diags[gi * baby + b], baby * gi)     # rot_{-baby*g}
            pdiags.append(oracle.ntt(oracle.to_rns(oracle.encode(dv, d_scale, P.N), P.q), P.q))
    pdiags = np.stack(pdiags)
    keys = {r: oracle.rotation_key(P, sk, r, g) for r in list(range(1, baby)) + [baby * gi for gi in range(1, giant)]}
    out = oracle.bsgs_linear_transform(P, ct, 4, pdiags, baby, giant, keys)
    want = sum(diags[k] * np.roll(z, -k) for k in range(baby * giant))
    got = _dec(P, sk, out, 4, 2.0 ** 25 * d_scale)
    assert np.abs(got - want).max() < TOL * 4
