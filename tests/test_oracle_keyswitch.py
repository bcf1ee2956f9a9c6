"""Pins for the oracle's key-switching stages (Section IV, Fig. "keysw").

* ModUp: every converted limb, in coefficient form, equals (x + e D_j) mod its
  prime for one e in [0, alpha_j) per coefficient (big-integer CRT); the
  digit's own limbs are the input limbs.
* ModDown: the output, lifted by CRT over Q_l, equals floor(U / P) - e with
  U the CRT lift of the input over P Q_l and e in [0, K) (floor ModDown).
* Key switching with a noise-free key: out_0 + out_1 s - d s' has every
  coefficient within (K + 1)(1 + h), h the Hamming weight of s (the rounding
  of ModDown plus its e P term, multiplied through by s).  With a real key the
  Gaussian key error adds at most sum_j N (alpha_j + 1) D_j 19 / P.
* Rescale: the output lifted over Q_{l-1} is exactly floor(C / q_last).
"""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

SMALL = dict(N=256, L=5, K=2, dnum=3, bits=31)      # alpha = 2: digits {0,1},{2,3},{4}
CFG1 = dict(N=4096, L=4, K=2, dnum=2, bits=30)


def mkparams(c):
    P = inputs.make_params(c["N"], c["L"], c["K"], c["dnum"], c["bits"])
    return oracle.OracleParams.from_params(P)


def prod(xs):
    r = 1
    for x in xs:
        r *= int(x)
    return r


@pytest.mark.parametrize("level,j", [(5, 0), (5, 1), (5, 2), (4, 1), (3, 1), (1, 0)])
def test_modup_crt(level, j):
    P = mkparams(SMALL)
    g = inputs.rng(100 + level * 7 + j)
    d = inputs.uniform_residues(g, P.q[:level], P.N)
    ext = oracle.modup(P, d, level, j)
    lo, hi = j * P.alpha, min((j + 1) * P.alpha, level)
    assert np.array_equal(ext[lo:hi], d[lo:hi])
    ext_primes = P.ext_primes(level)
    ext_coef = oracle.intt(ext, ext_primes)
    dig_primes = P.q[lo:hi]
    x = oracle.crt(ext_coef[lo:hi], dig_primes, centered=False)
    Dj = prod(dig_primes)
    others = [t for t in range(level + P.K) if not lo <= t < hi]
    for n in range(P.N):
        ok = False
        for e in range(hi - lo):
            if all(int(ext_coef[t, n]) == (x[n] + e * Dj) % ext_primes[t] for t in others):
                ok = True
                break
        assert ok, n


@pytest.mark.parametrize("level", [5, 3, 1])
def test_moddown_floor(level):
    P = mkparams(SMALL)
    g = inputs.rng(200 + level)
    ext_primes = P.ext_primes(level)
    u = inputs.uniform_residues(g, ext_primes, P.N)
    out = oracle.moddown(P, u, level)
    U = oracle.crt(oracle.intt(u, ext_primes), ext_primes, centered=False)
    got = oracle.crt(oracle.intt(out, P.q[:level]), P.q[:level], centered=False)
    Pp, Q = P.P_prod, prod(P.q[:level])
    for n in range(P.N):
        assert any(got[n] == (U[n] // Pp - e) % Q for e in range(P.K)), n


def ks_error(P, sk, d, level, out, s_from_ntt):
    q = P.q[:level]
    lhs = oracle.add(out[0], oracle.mul(out[1], sk.ntt[:level], q), q)
    rhs = oracle.mul(d, s_from_ntt[:level], q)
    diff = oracle.add(lhs, oracle.neg(rhs, q), q)
    return max(abs(x) for x in oracle.crt(oracle.intt(diff, q), q))


@pytest.mark.parametrize("cfg,level", [(SMALL, 5), (SMALL, 4), (SMALL, 3), (SMALL, 1), (CFG1, 4), (CFG1, 3)])
def test_keyswitch_noise_free_key_bound(cfg, level):
    P = mkparams(cfg)
    g = inputs.rng(300 + level)
    sk = oracle.SecretKey(P, inputs.ternary(g, P.N))
    s2 = oracle.mul(sk.ntt, sk.ntt, P.primes)
    key = oracle.switching_key(P, sk, s2, g, noise=False)
    d = inputs.uniform_residues(g, P.q[:level], P.N)
    out = oracle.keyswitch(P, d, level, key)
    err = ks_error(P, sk, d, level, out, s2)
    bound = (P.K + 1) * (1 + sk.hamming_weight)
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("level", [4, 2])
def test_keyswitch_real_key_bound(level):
    P = mkparams(CFG1)
    g = inputs.rng(400 + level)
    sk = oracle.SecretKey(P, inputs.ternary(g, P.N))
    s2 = oracle.mul(sk.ntt, sk.ntt, P.primes)
    key = oracle.switching_key(P, sk, s2, g, noise=True)
    d = inputs.uniform_residues(g, P.q[:level], P.N)
    out = oracle.keyswitch(P, d, level, key)
    err = ks_error(P, sk, d, level, out, s2)
    bound = (P.K + 1) * (1 + sk.hamming_weight)
    for j in range(P.beta(level)):
        lo, hi = j * P.alpha, min((j + 1) * P.alpha, level)
        bound += P.N * (hi - lo + 1) * prod(P.q[lo:hi]) * inputs.ERR_BOUND // P.P_prod + 1
    assert err <= bound, (err, bound)
    # and far below Q: a wrong gadget or sign would give an error of size ~Q
    assert err < prod(P.q[:level]) >> 40


def test_keyswitch_wrong_key_is_detected():
    # negative control: the bound must fail when the key encrypts another secret
    P = mkparams(SMALL)
    g = inputs.rng(500)
    sk = oracle.SecretKey(P, inputs.ternary(g, P.N))
    other = oracle.SecretKey(P, inputs.ternary(g, P.N))
    s2 = oracle.mul(sk.ntt, sk.ntt, P.primes)
    key = oracle.switching_key(P, other, s2, g, noise=False)
    d = inputs.uniform_residues(g, P.q[:5], P.N)
    out = oracle.keyswitch(P, d, 5, key)
    assert ks_error(P, sk, d, 5, out, s2) > (P.K + 1) * (1 + sk.hamming_weight) * 1000


@pytest.mark.parametrize("level", [5, 2])
def test_rescale_exact_floor(level):
    P = mkparams(SMALL)
    g = inputs.rng(600 + level)
    q = P.q[:level]
    ct = np.stack([inputs.uniform_residues(g, q, P.N) for _ in range(2)])
    out = oracle.rescale(P, ct, level)
    ql = q[-1]
    for c in range(2):
        C = oracle.crt(oracle.intt(ct[c], q), q, centered=False)
        got = oracle.crt(oracle.intt(out[c], q[:-1]), q[:-1], centered=False)
        assert got == [x // ql for x in C]


def test_inner_product_definition_small():
    # inner product is a per-limb sum of products: check one coefficient by hand
    P = mkparams(SMALL)
    level = 3
    g = inputs.rng(700)
    beta = P.beta(level)
    ext = np.stack([inputs.uniform_residues(g, P.ext_primes(level), P.N) for _ in range(beta)])
    key = np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)])
                    for _ in range(P.dnum)])
    u = oracle.inner_product(P, ext, level, key)
    for t, row in [(0, 0), (2, 2), (3, P.L), (4, P.L + 1)]:
        pr = P.ext_primes(level)[t]
        for c in range(2):
            n = 17 + t
            want = sum(int(ext[j, t, n]) * int(key[j, c, row, n]) for j in range(beta)) % pr
            assert int(u[c, t, n]) == want
