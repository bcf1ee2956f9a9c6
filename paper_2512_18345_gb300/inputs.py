"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and picks parameters. It holds none of the
key-switching arithmetic: no NTT, no base conversion, no modular products.
Both the CUDA path and the CPU oracle receive what it produces as plain
inputs, so neither side can leak results into the other through it.

Parameter choice (the paper only says the word-sized moduli sit near 2^31
and are NTT-friendly, Section III-C, "BConv"):
  * q_0 > q_1 > ... are the largest primes below 2^bits with q = 1 mod 2N;
  * the K special primes p_0 > p_1 > ... are the next ones below q_{L-1}.

Random draws (all from numpy's PCG64 seeded with the workload seed):
  * ternary secret: coefficients uniform in {-1, 0, 1};
  * error: rounded Gaussian, sigma = 3.2, redrawn when |e| > 19 (6 sigma);
  * uniform residues: each residue uniform in [0, q_i);
  * messages: complex slots with real and imaginary parts uniform in [-1, 1].
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Sequence

import numpy as np

SIGMA = 3.2
ERR_BOUND = 19  # 6 sigma, rounded down

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (covers every 64-bit value)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(N: int, bits: int, count: int, below: int | None = None) -> List[int]:
    """The `count` largest primes q < min(2^bits, below) with q = 1 mod 2N, descending."""
    two_n = 2 * N
    top = (1 << bits) if below is None else min(1 << bits, below)
    c = ((top - 1 - 1) // two_n) * two_n + 1  # largest value = 1 mod 2N strictly below top
    out: List[int] = []
    while len(out) < count:
        if c <= two_n:
            raise ValueError("not enough NTT-friendly primes")
        if is_prime(c):
            out.append(c)
        c -= two_n
    return out


@dataclasses.dataclass(frozen=True)
class Params:
    """Ring degree, ciphertext primes q, special primes p and the digit count."""
    N: int
    q: tuple
    p: tuple
    dnum: int

    @property
    def L(self) -> int:
        return len(self.q)

    @property
    def K(self) -> int:
        return len(self.p)

    @property
    def alpha(self) -> int:
        return -(-self.L // self.dnum)

    def beta(self, level: int) -> int:
        return -(-level // self.alpha)

    @property
    def primes(self) -> tuple:
        return tuple(self.q) + tuple(self.p)


def make_params(N: int, L: int, K: int, dnum: int, bits: int = 31) -> Params:
    allp = ntt_primes(N, bits, L + K)
    return Params(N=N, q=tuple(allp[:L]), p=tuple(allp[L:]), dnum=dnum)


# The five workloads: shapes from the paper's key-switching study (N = 2^16,
# ~24 limbs, word-sized primes) plus one small case the CPU oracle finishes in
# seconds.  Seeds are fixed: 20251218 + workload number.
WORKLOADS: Dict[str, dict] = {
    "hmult_relin_rescale_N4096_L4": dict(N=1 << 12, L=4, K=2, dnum=2, bits=30, seed=20251219,
                                         scale_bits=25),
    "hrotate_N65536_L24_plain": dict(N=1 << 16, L=24, K=8, dnum=3, bits=31, seed=20251220),
    "hrotate_N65536_L24_tc": dict(N=1 << 16, L=24, K=8, dnum=3, bits=31, seed=20251221),
    "batch64_N65536_L4to24": dict(N=1 << 16, L=24, K=8, dnum=3, bits=31, seed=20251222,
                                  items=64, level_lo=4, level_hi=24),
    "bsgs_lt_N65536_L24": dict(N=1 << 16, L=24, K=8, dnum=3, bits=31, seed=20251223,
                               baby=16, giant=8, scale_bits=31),
    # the paper's own key-switching shapes (Table "ks-param"): alpha = K = 12
    "paper_ks_N65536_L24_a12": dict(N=1 << 16, L=24, K=12, dnum=2, bits=31, seed=20251224),
    "paper_ks_N65536_L48_a12": dict(N=1 << 16, L=48, K=12, dnum=4, bits=31, seed=20251225),
    # bootstrapping linear transforms (CoeffToSlot / SlotToCoeff, radix levels, double
    # hoisting) at the paper's bootstrapping parameters (Table "parameter": N = 2^16,
    # L <= 48, dnum = 4; alpha = K = 12): CoeffToSlot from the top level, SlotToCoeff
    # from `stc_level` (the levels in between belong to EvalMod, which is not modelled)
    "cts_stc_N65536_L48_a12": dict(N=1 << 16, L=48, K=12, dnum=4, bits=31, seed=20251226,
                                   levels=3, cts_level=48, stc_level=33),
    # the same transforms on a ring the oracle finishes in seconds
    "cts_stc_N4096_L8": dict(N=1 << 12, L=8, K=2, dnum=4, bits=30, seed=20251227,
                             levels=3, cts_level=8, stc_level=5, scale_bits=28),
}


def workload_params(name: str) -> Params:
    w = WORKLOADS[name]
    return make_params(w["N"], w["L"], w["K"], w["dnum"], w["bits"])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_residues(g: np.random.Generator, primes: Sequence[int], N: int) -> np.ndarray:
    """[len(primes)][N] uint32, row i uniform in [0, primes[i])."""
    out = np.empty((len(primes), N), dtype=np.uint32)
    for i, q in enumerate(primes):
        out[i] = g.integers(0, q, size=N, dtype=np.uint64).astype(np.uint32)
    return out


def ternary(g: np.random.Generator, N: int) -> np.ndarray:
    """Secret coefficients uniform in {-1, 0, 1} (int64)."""
    return g.integers(-1, 2, size=N, dtype=np.int64)


def gaussian(g: np.random.Generator, N: int, sigma: float = SIGMA, bound: int = ERR_BOUND) -> np.ndarray:
    """Rounded Gaussian coefficients, redrawn until |e| <= bound (int64)."""
    e = np.rint(g.normal(0.0, sigma, size=N)).astype(np.int64)
    bad = np.abs(e) > bound
    while bad.any():
        e[bad] = np.rint(g.normal(0.0, sigma, size=int(bad.sum()))).astype(np.int64)
        bad = np.abs(e) > bound
    return e


def complex_slots(g: np.random.Generator, n: int) -> np.ndarray:
    """n complex slots with real and imaginary parts uniform in [-1, 1]."""
    return g.uniform(-1.0, 1.0, size=n) + 1j * g.uniform(-1.0, 1.0, size=n)


def rotation_index(g: np.random.Generator, lo: int = 1, hi: int = 1 << 15) -> int:
    return int(g.integers(lo, hi))


def batch_items(g: np.random.Generator, items: int, level_lo: int, level_hi: int) -> List[dict]:
    """Mixed batch: each item is a relinearisation or a rotation (p = 1/2),
    level uniform in [level_lo, level_hi], rotation index uniform in [1, 2^15)."""
    out = []
    for _ in range(items):
        op = "rotate" if g.integers(0, 2) else "relin"
        level = int(g.integers(level_lo, level_hi + 1))
        rot = rotation_index(g)
        out.append(dict(op=op, level=level, rot=rot))
    return out


# ------------------------------------------------------------------ bootstrapping transform structure

def radix_levels(log_slots: int, n_levels: int) -> List[tuple]:
    """Split the butterfly stages 1..log_slots (stage s has half-width 2^(s-1)) into n_levels
    consecutive groups, as even as possible, the larger groups first: [(s_lo, s_hi)] ascending."""
    base, extra = divmod(log_slots, n_levels)
    out, s = [], 1
    for i in range(n_levels):
        r = base + (1 if i < extra else 0)
        out.append((s, s + r - 1))
        s += r
    return out


@dataclasses.dataclass(frozen=True)
class BsgsPlan:
    """Baby-step / giant-step split of one radix level: the level's diagonal offsets are
    d * step (mod n) with |d| <= D; offset k = giant[g] + baby[b] is diagonal idx[g][b]
    (-1: that pair covers no new offset); offsets[j] is diagonal j's offset (mod n)."""
    step: int
    baby: tuple
    giant: tuple
    idx: tuple
    offsets: tuple

    @property
    def n_diag(self) -> int:
        return len(self.offsets)

    def rotations(self) -> List[int]:
        return sorted({r for r in self.baby + self.giant if r})


def bsgs_plan(n_slots: int, s_lo: int, s_hi: int, giant_cost: float = 3.0) -> BsgsPlan:
    """Offsets of stages s_lo..s_hi multiplied together are sums of e_s 2^(s-1), e_s in
    {-1, 0, 1}: the multiples d 2^(s_lo - 1), |d| <= D = 2^(s_hi - s_lo + 1) - 1.  Baby steps
    b step (b < n1); giant steps (g n1 - c) step with c = n1 ceil(D / n1), so one giant step is
    the identity; each offset (mod n) goes to the first pair that reaches it, and giant steps
    that reach none are dropped.  n1 is the power of two (at most 32) that minimises
    (n1 - 1) + giant_cost (ceil((2D + 1) / n1) - 1): with double hoisting a baby step costs one
    inner product, a giant step a ModDown, a ModUp and an inner product."""
    step = 1 << (s_lo - 1)
    D = (1 << (s_hi - s_lo + 1)) - 1
    count = min(2 * D + 1, n_slots)
    n1, best = 1, None
    c1 = 1
    while c1 <= min(32, 2 * count):
        cost = (c1 - 1) + giant_cost * (-(-count // c1) - 1)
        if best is None or cost < best:
            n1, best = c1, cost
        c1 *= 2
    c = n1 * (-(-D // n1))
    n2 = (D + c) // n1 + 1
    seen: Dict[int, int] = {}
    rows, giants = [], []
    for g in range(n2):
        row = []
        for b in range(n1):
            d = g * n1 - c + b
            k = (d * step) % n_slots
            if abs(d) <= D and k not in seen:
                seen[k] = len(seen)
                row.append(seen[k])
            else:
                row.append(-1)
        if any(j >= 0 for j in row):
            rows.append(tuple(row))
            giants.append(((g * n1 - c) * step) % n_slots)
    offsets = tuple(sorted(seen, key=seen.get))
    return BsgsPlan(step=step, baby=tuple(b * step for b in range(n1)), giant=tuple(giants), idx=tuple(rows),
                    offsets=offsets)


def transform_plans(N: int, n_levels: int, kind: str) -> List[BsgsPlan]:
    """The levels of CoeffToSlot ("cts": the highest stages first) or SlotToCoeff ("stc":
    the lowest first), in evaluation order, on n = N/2 slots."""
    n = N // 2
    lv = radix_levels(n.bit_length() - 1, n_levels)
    if kind == "cts":
        lv = lv[::-1]
    elif kind != "stc":
        raise ValueError(kind)
    return [bsgs_plan(n, lo, hi) for lo, hi in lv]
