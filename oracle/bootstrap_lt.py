"""Bootstrapping linear transforms (CoeffToSlot / SlotToCoeff) for the CPU
oracle -- TEST INFRASTRUCTURE ONLY.

The paper evaluates bootstrapping, whose linear transforms rely on hoisted
key switching (Section V-C, citing the hoisting literature).  This module
restates, from the CKKS literature, the pieces the key-switching path needs:

  * the homomorphic DFT of the slots as a product of sparse butterfly stages
    (the "special FFT" of CKKS decoding), grouped into radix levels;
  * each level as diagonals (diag_k[r] = M[r][r + k mod n]);
  * the double-hoisted baby-step / giant-step evaluation of one level, as a
    sequence of the oracle's exact RNS steps (ModUp, automorphism, inner
    product, ModDown), in the order that step list defines.

Slot / coefficient relation (the decoding map the oracle's `decode` uses):
with n = N/2 slots, M = 2N and zeta = exp(2 pi i / M), a real polynomial m
decodes to z_j = sum_{k<N} m_k zeta^(5^j k).  Since zeta^(5^j n) = i, this is
z = U a with a_k = m_k + i m_{k+n} and U[j][k] = zeta^(5^j k), j, k < n.
Splitting a into even and odd indices gives z_j = E_j + w_j O_j and
z_{j+n/2} = E_j - w_j O_j with w_j = zeta^(5^j) (5^(n/2) = 1 + M/2 mod M), so
with the input in bit-reversed order U is a product of log2(n) butterfly
stages: stage s (half-width h = 2^(s-1), block length 2h) maps, for each block
and j < h,
    v[i + j]     <- v[i + j] + t_{s,j} v[i + j + h]
    v[i + j + h] <- v[i + j] - t_{s,j} v[i + j + h]
with t_{s,j} = zeta^((5^j mod 4*2h) * M / (4*2h)).  SlotToCoeff applies the
stages s = 1 .. log2(n) (slots <- U bitrev(slots)); CoeffToSlot applies their
inverses in reverse order (slots <- bitrev(U^-1 slots)).  The conjugation
step that separates real and imaginary parts in full bootstrapping is not
part of these transforms (it is outside the key-switching path studied).

Pin status (tests/test_oracle_bootstrap_lt.py):
  stage products   pinned: equal to the dense U bitrev(.) from the definition
  level diagonals  pinned: diagonal-form product equals the dense product
  lt_double_hoisted pinned: decrypts to the FP64 matrix-vector product;
                   CoeffToSlot followed by SlotToCoeff returns the message
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

from . import ckks

Diags = Dict[int, np.ndarray]


# ------------------------------------------------------------------ the special FFT as sparse stages

def _twiddles(N: int, s: int) -> np.ndarray:
    """t_{s,j} for j < 2^(s-1): zeta^((5^j mod 4 len) M / (4 len)), len = 2^s, M = 2N."""
    M = 2 * N
    ln = 1 << s
    lq = 4 * ln
    h = ln // 2
    e = np.empty(h, dtype=np.int64)
    x = 1
    for j in range(h):
        e[j] = (x % lq) * (M // lq)
        x = x * 5 % M
    return np.exp(2j * np.pi * e / M)


def stage_diagonals(N: int, s: int, inverse: bool = False) -> Diags:
    """Diagonal form of butterfly stage s (or its inverse) on n = N/2 slots."""
    n = N // 2
    h = 1 << (s - 1)
    t = _twiddles(N, s)
    r = np.arange(n)
    pos = r % (2 * h)
    upper = pos < h
    w = t[np.where(upper, pos, pos - h)]
    d: Diags = {}

    def put(k, vec):
        k %= n
        d[k] = d[k] + vec if k in d else vec

    if not inverse:
        # upper row: v + w v[+h];  lower row: v[-h] - w v
        put(0, np.where(upper, 1.0 + 0j, -w))
        put(h, np.where(upper, w, 0j))
        put(-h, np.where(upper, 0j, 1.0 + 0j))
    else:
        # upper row: (x + x[+h]) / 2;  lower row: (x[-h] - x) / (2 w)
        put(0, np.where(upper, 0.5 + 0j, -0.5 / w))
        put(h, np.where(upper, 0.5 + 0j, 0j))
        put(-h, np.where(upper, 0j, 0.5 / w))
    return {k: v for k, v in d.items() if np.any(v != 0)}


def compose(A: Diags, B: Diags, n: int) -> Diags:
    """Diagonal form of A B (B applied first): (AB)_{k1+k2} += A_k1 * roll(B_k2, -k1)."""
    C: Diags = {}
    for k1, a in A.items():
        for k2, b in B.items():
            k = (k1 + k2) % n
            term = a * np.roll(b, -k1)
            C[k] = C[k] + term if k in C else term
    return C


def apply_diagonals(D: Diags, z: np.ndarray) -> np.ndarray:
    """M z = sum_k diag_k * rot_k(z), rot_k(z)[r] = z[r + k mod n]."""
    out = np.zeros_like(z, dtype=np.complex128)
    for k, d in D.items():
        out += d * np.roll(z, -k)
    return out


def level_diagonals(N: int, s_lo: int, s_hi: int, inverse: bool) -> Diags:
    """One radix level: stages s_lo..s_hi applied in ascending order (SlotToCoeff), or the
    inverses of stages s_hi..s_lo applied in that order (CoeffToSlot)."""
    n = N // 2
    D: Diags = {0: np.ones(n, dtype=np.complex128)}
    order = range(s_lo, s_hi + 1) if not inverse else range(s_hi, s_lo - 1, -1)
    for s in order:
        D = compose(stage_diagonals(N, s, inverse), D, n)
    return {k: v for k, v in D.items() if np.abs(v).max() > 1e-12}


def bitrev_perm(n: int) -> np.ndarray:
    b = n.bit_length() - 1
    return np.array([int(format(i, f"0{b}b")[::-1], 2) for i in range(n)], dtype=np.int64)


def dft_matrix(N: int) -> np.ndarray:
    """U[j][k] = zeta^(5^j k), j, k < N/2 (the definition; for pins at small N)."""
    n = N // 2
    M = 2 * N
    e = np.empty(n, dtype=np.int64)
    x = 1
    for j in range(n):
        e[j] = x
        x = x * 5 % M
    k = np.arange(n)
    return np.exp(2j * np.pi * ((e[:, None] * k[None, :]) % M) / M)


# ------------------------------------------------------------------ plaintexts of one level

def encode_ext(P: ckks.OracleParams, z: np.ndarray, scale: float, level: int) -> np.ndarray:
    """NTT-form residues of round(scale tau^-1(z)) over q_0..q_{level-1}, p_0..p_{K-1}."""
    primes = P.ext_primes(level)
    return ckks.ntt(ckks.to_rns(ckks.encode(z, scale, P.N), primes), primes)


def level_plaintexts(P: ckks.OracleParams, D: Diags, plan, level: int, scale: float) -> np.ndarray:
    """pt[idx[g][b]] = encode(roll(diag_k, giant[g])) for the offset k = giant[g] + baby[b] of every
    used pair, so that rot_{giant[g]}(pt (.) rot_{baby[b]}(z)) = diag_k (.) rot_k(z)."""
    n = P.N // 2
    out = np.empty((plan.n_diag, len(P.ext_primes(level)), P.N), dtype=np.uint32)
    for g, row in enumerate(plan.idx):
        for b, j in enumerate(row):
            if j < 0:
                continue
            k = plan.offsets[j]
            d = D.get(k, np.zeros(n, dtype=np.complex128))
            out[j] = encode_ext(P, np.roll(d, plan.giant[g]), scale, level)
    return out


# ------------------------------------------------------------------ double-hoisted evaluation

def _lift(P: ckks.OracleParams, x: np.ndarray, level: int) -> np.ndarray:
    """P x on the q-limbs, 0 on the special limbs ([level + K][N])."""
    out = np.zeros((level + P.K, P.N), dtype=np.uint32)
    for i in range(level):
        q = P.q[i]
        out[i] = (x[i].astype(np.uint64) * np.uint64(P.P_prod % q) % np.uint64(q)).astype(np.uint32)
    return out


def lt_double_hoisted(P: ckks.OracleParams, ct: np.ndarray, level: int, baby: Sequence[int],
                      giant: Sequence[int], diags: np.ndarray, idx: Sequence[Sequence[int]],
                      rot_keys: dict) -> np.ndarray:
    """sum_g rot_{giant[g]}( sum_b diags[idx[g][b]] (.) rot_{baby[b]}(ct) ), before rescale, with
    ModUp hoisted over the baby steps and ModDown hoisted over both step kinds:
      1. digits_j = ModUp_j(c1), j < beta;
      2. baby b: (P sigma_b(c0) + u_0, u_1), u = IP(sigma_b(digits), key_b) over Q_l u P
         (the identity: (P c0, P c1) with zero special limbs);
      3. inner_g = sum_b pt (.) baby_b over Q_l u P;
      4. giant g with a rotation: c1' = ModDown(inner_g,1); v = IP(sigma_g(ModUp(c1')), key_g);
         acc += (sigma_g(inner_g,0) + v_0, v_1); without a rotation: acc += inner_g;
      5. out = (ModDown(acc_0), ModDown(acc_1)).
    diags [n_diag][level + K][N] NTT form over the extended basis; idx [n_giant][n_baby]."""
    N, K = P.N, P.K
    xp = P.ext_primes(level)
    beta = P.beta(level)
    c0, c1 = ckks._u32(ct[0]), ckks._u32(ct[1])
    digits = np.stack([ckks.modup(P, c1, level, j) for j in range(beta)])

    babies = []
    for r in baby:
        k = ckks.galois_elt(r, N)
        if k == 1:
            babies.append(np.stack([_lift(P, c0, level), _lift(P, c1, level)]))
            continue
        u = ckks.inner_product(P, np.stack([ckks.automorph_ntt(d, k) for d in digits]), level, rot_keys[r])
        u[0] = ckks.add(u[0], _lift(P, ckks.automorph_ntt(c0, k), level), xp)
        babies.append(u)

    acc = np.zeros((2, level + K, N), dtype=np.uint32)
    for g, r in enumerate(giant):
        inner = np.zeros((2, level + K, N), dtype=np.uint32)
        for b in range(len(baby)):
            j = idx[g][b]
            if j < 0:
                continue
            for c in range(2):
                inner[c] = ckks.add(inner[c], ckks.mul(babies[b][c], diags[j], xp), xp)
        k = ckks.galois_elt(r, N)
        if k == 1:
            for c in range(2):
                acc[c] = ckks.add(acc[c], inner[c], xp)
            continue
        c1d = ckks.moddown(P, inner[1], level)
        dg = np.stack([ckks.automorph_ntt(ckks.modup(P, c1d, level, j), k) for j in range(beta)])
        v = ckks.inner_product(P, dg, level, rot_keys[r])
        acc[0] = ckks.add(acc[0], ckks.add(ckks.automorph_ntt(inner[0], k), v[0], xp), xp)
        acc[1] = ckks.add(acc[1], v[1], xp)
    return np.stack([ckks.moddown(P, acc[0], level), ckks.moddown(P, acc[1], level)])


def radix_transform(P: ckks.OracleParams, ct: np.ndarray, level: int, plans: List, pts: List[np.ndarray],
                    rot_keys: dict) -> np.ndarray:
    """A chain of levels (CoeffToSlot or SlotToCoeff): each double-hoisted level followed by a
    rescale; plans / pts in evaluation order.  Returns the ciphertext at level - len(plans)."""
    for plan, pt in zip(plans, pts):
        ct = lt_double_hoisted(P, ct, level, plan.baby, plan.giant, pt, plan.idx, rot_keys)
        ct = ckks.rescale(P, ct, level)
        level -= 1
    return ct
