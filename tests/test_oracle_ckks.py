"""CKKS-level pins for the oracle: encoding against the slot definition, and
decryption of rotated / multiplied / transformed ciphertexts against FP64
plaintext arithmetic.

Key-switched and rescaled results are checked against the slot-error model of
oracle/noise.py, derived from the RNS arithmetic: per slot, the decoded error
minus the model's prediction (the key-error term sum_j dt_j e_j / P of key
switching and the mean -(k/2) 1(zeta)(1 + s(zeta)) of each division by k
primes) must lie within the model's bound (the divisions' fluctuation and the
fresh noise).  The prediction reproduces the measured maximum to about three
digits; the bound is tens to hundreds of times smaller than the prediction, so
a change that doubled the error fails.  The composed-rotation test adds two
rotations' terms; the linear-transform test keeps a loose tolerance (its
plaintext products are not modelled).  Exactness of every residue is pinned
elsewhere.
"""
import cmath

import numpy as np
import pytest

import oracle
from oracle import noise
from paper_2512_18345_gb300 import inputs

TOL = 2.0 ** -3  # the linear transform's loose tolerance only


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
    err, pred, ratio = noise.check_rotation(P, sk, ct, 4, rot, key, _dec(P, sk, out, 4, 2.0 ** 25),
                                            np.roll(z, -rot), 2.0 ** 25)
    assert ratio <= 1.0, (err, pred, ratio)


def test_rotate_composes():
    P = cfg1()
    g, sk, z, ct = _fresh(P, 20)
    k3, k4 = oracle.rotation_key(P, sk, 3, g), oracle.rotation_key(P, sk, 4, g)
    mid = oracle.rotate(P, ct, 4, 3, k3)
    out = oracle.rotate(P, mid, 4, 4, k4)
    # the first rotation's error moves with the second rotation (4 slots) and the second adds its own
    p1, b1 = noise.rotation_error(P, sk, ct, 4, 3, k3)
    p2, b2 = noise.rotation_error(P, sk, mid, 4, 4, k4)
    d = 2.0 ** 25
    err, pred, ratio = noise.check(_dec(P, sk, out, 4, d) - np.roll(z, -7), (np.roll(p1, -4) + p2) / d,
                                   (np.roll(b1, -4) + b2) / d)
    assert ratio <= 1.0, (err, pred, ratio)


def test_hoisted_rotations():
    P = cfg1()
    g, sk, z, ct = _fresh(P, 30)
    rots = [0, 1, 2, 9]
    keys = [None] + [oracle.rotation_key(P, sk, r, g) for r in rots[1:]]
    outs = oracle.rotate_hoisted(P, ct, 4, rots, keys)
    for r, k, o in zip(rots, keys, outs):
        dec = _dec(P, sk, o, 4, 2.0 ** 25)
        if r == 0:  # the identity: the input itself
            assert np.abs(dec - z).max() < noise.fresh_noise_bound(P.N) / 2.0 ** 25
            continue
        err, pred, ratio = noise.check_rotation(P, sk, ct, 4, r, k, dec, np.roll(z, -r), 2.0 ** 25, hoisted=True)
        assert ratio <= 1.0, (r, err, pred, ratio)


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
    # before the rescale: fresh-noise products at scale d, the relinearisation at d^2
    ks, kb = noise.keyswitch_error(P, sk, oracle.mul(c1[1], c2[1], P.q), 4, rk, noise.relin_s_from(P, sk))
    bound = (np.abs(z1) + np.abs(z2) + 1.0) * noise.fresh_noise_bound(P.N) / d + (np.abs(ks) + kb) / (d * d)
    assert (np.abs(_dec(P, sk, m, 4, d * d) - z1 * z2) <= bound).all()
    r = oracle.rescale(P, m, 4)
    err, pred, ratio = noise.check_hmult_rescale(P, sk, c1, c2, 4, rk, z1, z2, _dec(P, sk, r, 3, d * d / P.q[3]), d)
    assert ratio <= 1.0, (err, pred, ratio)


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


def test_noise_model_ones_closed_form():
    """1(zeta) = sum_n zeta^n = 2 / (1 - zeta) at every slot, |1(zeta_0)| = 1 / sin(pi / 2N)."""
    N = 1 << 10
    ev = noise.ones_eval(N)
    e = np.array([pow(5, j, 2 * N) for j in range(N // 2)])
    zeta = np.exp(1j * np.pi * e / N)
    assert np.allclose(ev, 2.0 / (1.0 - zeta), rtol=1e-9)
    assert abs(abs(ev[0]) - 1.0 / np.sin(np.pi / (2 * N))) < 1e-6 * N


def test_noise_model_catches_a_rounding_change():
    """Negative control: rescaling with a rounding offset (q_last / 2 added before the floor,
    a plausible mistake) moves the decoded error away from the floor model by its whole mean
    term, far outside the bound."""
    P = cfg1()
    g = inputs.rng(41)
    sk = oracle.SecretKey(P, inputs.ternary(g, P.N))
    d = 2.0 ** 25
    z1, z2 = inputs.complex_slots(g, P.N // 2), inputs.complex_slots(g, P.N // 2)
    c1 = oracle.encrypt(P, sk, oracle.encode(z1, d, P.N), 4, g)
    c2 = oracle.encrypt(P, sk, oracle.encode(z2, d, P.N), 4, g)
    rk = oracle.relin_key(P, sk, g)
    m = oracle.hmult(P, c1, c2, 4, rk)
    half = oracle.ntt(oracle.to_rns(np.full(P.N, P.q[3] // 2, dtype=np.int64), P.q), P.q)
    rounded = np.stack([oracle.add(m[c], half, P.q) for c in range(2)])  # round instead of floor
    r = oracle.rescale(P, rounded, 4)
    err, pred, ratio = noise.check_hmult_rescale(P, sk, c1, c2, 4, rk, z1, z2, _dec(P, sk, r, 3, d * d / P.q[3]), d)
    assert ratio > 3.0, (err, pred, ratio)
