"""Decoded slot error of the key-switched and rescaled CKKS operations --
TEST INFRASTRUCTURE ONLY (used by tests/ and __graft_entry__.smoke()).

Every residue of every operation is pinned bit for bit elsewhere; this module
predicts the error those exact results carry after decryption and decoding, so
that the decode tests check a bound derived from the arithmetic instead of a
fixed tolerance.

Evaluation at a slot is a ring homomorphism: for zeta_j = exp(i pi 5^j / N),
p -> p(zeta_j) maps the negacyclic product to the pointwise one, and decode(m)_j
= m(zeta_j) / scale.  Every error polynomial below is therefore evaluated slot by
slot (decode with scale 1), and products of polynomials become products of
their evaluations.

Division by D = d_1 ... d_k (rescale: k = 1, D = q_last; ModDown: k = K,
D = P; both floor type, with no rounding offset) of a ciphertext (c0, c1) with
phase c0 + c1 s subtracts r_c = sum_i y_i (D / d_i), y_i = [c_c (D / d_i)^-1]_{d_i},
and divides by D: the fast base conversion of c_c mod D, which equals
[c_c]_D + e' D with the conversion's overflow e' in [0, k).  The result's phase
is (c0 + c1 s) / D - (f0 + f1 s) with f_c = r_c / D = sum_i y_i / d_i per
coefficient: a sum of k terms uniform on [0, 1) (k = 1: plain floor).  So:
  * the mean part -(k/2) 1(zeta) (1 + s(zeta)) is fixed by the secret, with
    1(zeta) = sum_{n < N} zeta^n = 2 / (1 - zeta) (zeta^N = -1), whose size
    |1(zeta_0)| = 1 / sin(pi / 2N) ~ 2N / pi puts it in the lowest-frequency
    slot;
  * the fluctuating part -(g0(zeta) + g1(zeta) s(zeta)), g_c = f_c - k/2: g_c(zeta)
    is a sum of N terms of variance k/12, bounded here by 6 sqrt(N k / 12).

Hybrid key switching (digits j, special modulus P): with dt_j the ModUp output
of digit j as an integer polynomial (the fast base conversion's x + u D_j, not
centred) and the key's b_j = -a_j s + e_j + g_j s' (Section II-A's gadget form),
the inner product's phase is P d s' + sum_j dt_j e_j exactly (the ModUp
exactness invariant), so after ModDown the error is
  sum_j dt_j(zeta) e_j(zeta) / P  plus the floor terms above.
dt_j has mean about D_j per coefficient (x uniform on [0, D_j) plus u D_j), so
this term, too, collects in the lowest-frequency slot.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

from . import ckks


def slot_eval(coeffs: Sequence[int] | np.ndarray, N: int) -> np.ndarray:
    """p(zeta_j) for the N / 2 slots (decode with scale 1)."""
    return ckks.decode(coeffs, 1.0, N)


def ones_eval(N: int) -> np.ndarray:
    return slot_eval(np.ones(N, dtype=np.int64), N)


def floor_division_terms(s_ev: np.ndarray, N: int, k: int = 1) -> Tuple[np.ndarray, np.ndarray]:
    """(mean, bound) of the phase error a division by a product of k primes leaves, per slot:
    mean -(k/2) 1(zeta)(1 + s(zeta)); the rest within 6 sqrt(N k / 12)(1 + |s(zeta)|)."""
    mean = -0.5 * k * ones_eval(N) * (1.0 + s_ev)
    bound = 6.0 * math.sqrt(N * k / 12.0) * (1.0 + np.abs(s_ev))
    return mean, bound


def fresh_noise_bound(N: int, sigma: float = 3.2) -> float:
    """Per-slot bound of a fresh encryption's error plus its encoding rounding:
    6 sigma sqrt(N) + 6 sqrt(N / 12)."""
    return 6.0 * sigma * math.sqrt(N) + 6.0 * math.sqrt(N / 12.0)


def _centered(res: np.ndarray, q: int) -> np.ndarray:
    r = res.astype(np.int64)
    return np.where(r > q // 2, r - q, r)


def key_errors(P: "ckks.OracleParams", sk: "ckks.SecretKey", key: np.ndarray, s_from_ntt: np.ndarray) -> List[np.ndarray]:
    """e_j = b_j + a_j s - g_j s' of each digit, recovered from the key (integer polynomials;
    small, so one prime's centred residues give them)."""
    primes = P.primes
    out = []
    Pp = P.P_prod
    for j in range(P.dnum):
        b, a = key[j, 0], key[j, 1]
        e = ckks.add(b, ckks.mul(a, sk.ntt, primes), primes)
        lo, hi = j * P.alpha, min((j + 1) * P.alpha, P.L)
        for i in range(lo, hi):  # remove g_j s' = [P]_{q_i} s' on the digit's q-limbs
            q = primes[i]
            gs = (np.asarray(s_from_ntt[i], dtype=np.uint64) * (Pp % q)) % q
            e[i] = ((e[i].astype(np.uint64) + q - gs) % q).astype(np.uint32)
        coef = ckks.intt(e, primes)
        e0 = _centered(coef[0], primes[0])
        assert np.array_equal(_centered(coef[-1], primes[-1]), e0), "key error is not small"
        out.append(e0)
    return out


def modup_ints(P: "ckks.OracleParams", d_ntt: np.ndarray, level: int) -> List[List[int]]:
    """dt_j, the ModUp output of each digit of d (NTT form, `level` limbs) as integers in
    [0, Q_level P) (big-integer CRT of its coefficient-form limbs)."""
    prim = P.ext_primes(level)
    out = []
    for j in range(P.beta(level)):
        ext = ckks.modup(P, d_ntt, level, j)
        out.append(ckks.crt(ckks.intt(ext, prim), prim, centered=False))
    return out


def keyswitch_error(P: "ckks.OracleParams", sk: "ckks.SecretKey", d_ntt: np.ndarray, level: int, key: np.ndarray,
                    s_from_ntt: np.ndarray, roll: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """(prediction, bound) of the phase error of KS(d) per slot: prediction
    sum_j dt_j(zeta) e_j(zeta) / P - (K/2) 1(zeta)(1 + s(zeta)); the rest within the ModDown
    division's bound.  roll = r evaluates sigma_{5^r}(dt_j) instead of dt_j (hoisted rotations:
    sigma applied after ModUp), i.e. dt_j at slot j + r."""
    N = P.N
    s_ev = slot_eval(sk.coeffs, N)
    es = key_errors(P, sk, key, s_from_ntt)
    pred = np.zeros(N // 2, dtype=np.complex128)
    for dt, e in zip(modup_ints(P, d_ntt, level), es):
        pred += np.roll(slot_eval(dt, N), -roll) * slot_eval(e, N)
    pred /= float(P.P_prod)
    mean, bound = floor_division_terms(s_ev, N, P.K)  # ModDown divides by the K special primes
    return pred + mean, bound


def rotation_s_from(P: "ckks.OracleParams", sk: "ckks.SecretKey", rot: int) -> np.ndarray:
    """NTT form of sigma_k(s), k = 5^rot mod 2N (the key's source secret)."""
    k = ckks.galois_elt(rot, P.N)
    return ckks.ntt(ckks.to_rns(ckks.automorph_int(sk.coeffs, k), P.primes), P.primes)


def relin_s_from(P: "ckks.OracleParams", sk: "ckks.SecretKey") -> np.ndarray:
    return ckks.mul(sk.ntt, sk.ntt, P.primes)


def rotation_error(P, sk, ct, level, rot, key, hoisted=False) -> Tuple[np.ndarray, np.ndarray]:
    """(prediction, bound) of the phase error of HRotate(ct, rot) per slot: the key switch of
    sigma(c1) (fhe_rotate: sigma before ModUp), or of c1 with sigma applied to its ModUp digits
    (hoisted); the bound adds the input's fresh noise, carried along by sigma."""
    N = P.N
    if hoisted:
        pred, fb = keyswitch_error(P, sk, ct[1], level, key, rotation_s_from(P, sk, rot), roll=rot % (N // 2))
    else:
        c1r = ckks.automorph_ntt(ct[1], ckks.galois_elt(rot, N))
        pred, fb = keyswitch_error(P, sk, c1r, level, key, rotation_s_from(P, sk, rot))
    return pred, fb + fresh_noise_bound(N)


def check(err: np.ndarray, pred: np.ndarray, bound: np.ndarray) -> Tuple[float, float, float]:
    """(max |err|, max |pred|, max |err - pred| / bound) over the slots (all in slot units)."""
    return float(np.abs(err).max()), float(np.abs(pred).max()), float((np.abs(err - pred) / bound).max())


def check_rotation(P, sk, ct, level, rot, key, dec, want, scale, hoisted=False):
    """Decoded rotation against the model: returns check(dec - want, pred / scale, bound / scale)."""
    pred, bound = rotation_error(P, sk, ct, level, rot, key, hoisted)
    return check(dec - want, pred / scale, bound / scale)


def check_hmult_rescale(P, sk, a, b, level, rk, z1, z2, dec, scale):
    """Slot errors of decode(Rescale(HMult(a, b))) at scale^2 / q_last against the model:
    pred = the rescale's floor mean / (scale^2 / q_last); bound = its fluctuation at that scale,
    plus the product's fresh-noise terms (|z1| + |z2| + 1) (fresh bound) / scale and the
    relinearisation's error (prediction plus bound) / scale^2.  Returns (max |err|,
    max |pred|, max |err - pred| / bound)."""
    N = P.N
    s_ev = slot_eval(sk.coeffs, N)
    out_scale = scale * scale / P.q[level - 1]
    mean, fb = floor_division_terms(s_ev, N)
    d2 = ckks.mul(a[1], b[1], P.q[:level])  # the relinearised polynomial (NTT form)
    ks_pred, ks_b = keyswitch_error(P, sk, d2, level, rk, relin_s_from(P, sk))
    bound = fb / out_scale + (np.abs(z1) + np.abs(z2) + 1.0) * fresh_noise_bound(N) / scale \
        + (np.abs(ks_pred) + ks_b) / (scale * scale)
    return check(dec - z1 * z2, mean / out_scale, bound)
