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
