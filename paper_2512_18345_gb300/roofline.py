"""Algorithmic byte model of one hybrid key switch (the L2 roofline numerator).

Every kernel boundary is a round trip through global memory (L2), as in the
paper's traffic model (Section V-B, Table "ks-param"; ideal latency = bytes /
peak L2 bandwidth, Section V-B "Key-switching evaluation").  Counted in limbs
of W = 4N bytes, at level l with K special primes and beta digits, with a
two-pass NTT (read + write per pass):

  stage 1 (ModUp):   INTT of the l input limbs, two passes        4 l
                     BConv reads l, writes beta (l + K) - l        beta (l + K)
                     NTT of the new limbs, two passes              4 (beta (l + K) - l)
                     total                                         5 beta (l + K)
  stage 2 (inner):   ModUp outputs + key (2 beta (l + K)) + the two
                     outputs (2 (l + K)) + the pass-through poly (l)
                                                                   3 beta (l + K) + 2 (l + K) + l
  stage 3 (ModDown): INTT of 2 K limbs two-pass (8 K), BConv reads 2 K,
                     writes 2 l, NTT of 2 l limbs two-pass (8 l), the
                     combine epilogue reads 2 l                    10 K + 12 l

The footprints (stage 1: beta (l + K) limbs, stage 3: 4 l limbs) reproduce
the paper's table exactly, as do stage 2 for every row, every column of
(12,12,1) and stage 3 of (24,12,2).  Stage 1 of (24,12,2) and (48,12,4) sits
below the paper by exactly (beta - 1) l limbs, and stage 3 of (48,12,4) by
about 71 limbs; the paper does not say where those bytes go.
"""
from __future__ import annotations


def limb_bytes(N: int) -> int:
    return 4 * N


def beta_of(level: int, alpha: int) -> int:
    return -(-level // alpha)


def stage_limbs(level: int, K: int, beta: int) -> tuple:
    """(stage1, stage2, stage3) global-memory traffic in limbs."""
    ext = beta * (level + K)
    s1 = 5 * ext
    s2 = 3 * ext + 2 * (level + K) + level
    s3 = 10 * K + 12 * level
    return s1, s2, s3


def footprint_limbs(level: int, K: int, beta: int) -> tuple:
    """(stage1, stage3) maximum memory footprint in limbs."""
    return beta * (level + K), 4 * level


def ks_bytes(N: int, level: int, K: int, alpha: int) -> int:
    """B_KS: algorithmic global-memory bytes of one key switch at `level`."""
    return sum(stage_limbs(level, K, beta_of(level, alpha))) * limb_bytes(N)


def ks_compulsory_hbm_bytes(N: int, level: int, K: int, alpha: int) -> int:
    """Input d (l limbs) + key (2 beta (l + K)) + output (2 l): the DRAM floor."""
    beta = beta_of(level, alpha)
    return (level + 2 * beta * (level + K) + 2 * level) * limb_bytes(N)


def ntt_bytes(N: int, limbs: int) -> int:
    """Compulsory bytes of a one-pass transform of `limbs` limbs: read + write."""
    return 2 * limbs * limb_bytes(N)
