"""The 64-bit accumulation schedules of the streaming kernels, replayed on the CPU
in exact integers.

Both kernels form sums of 62-bit products of residues (primes below 2^31) in one
64-bit word and reduce late:

* the key inner product (Section IV, stage 2) adds the beta <= 4 digits' products
  u_c = sum_j ModUp_j * key_j before one reduction;
* the diagonal pass of the baby-step / giant-step transforms adds one product
  per baby step to each accumulator and, after every third step, folds the word
  as  a = hi 2^34 + lo  ->  hi (2^34 mod q) + lo  (three integer instructions:
  a shift, a mask and one 32 x 32 -> 64 multiply-add), reducing once at the end.

These tests check, at the worst case (every operand q - 1, the largest prime below
2^31) and on random operands, that no intermediate word reaches 2^64, that every
fold keeps the residue and lands below 2^61 + 2^34, and that the final reduction
equals the plain definition of the sum."""
import numpy as np
import pytest

W64 = 1 << 64
LARGEST_31BIT_PRIME = 2147483647  # 2^31 - 1


def fold34(a: int, r34: int) -> int:
    """The kernel's fold: the shift and mask split a 64-bit word at bit 34."""
    return (a >> 34) * r34 + (a & ((1 << 34) - 1))


def diag_schedule(xs, ds, q):
    """One accumulator of the diagonal pass over len(xs) baby steps: a product per step, a
    fold after every third step, one reduction at the end.  Returns the result and the
    largest word seen."""
    r34 = (1 << 34) % q
    acc, peak = 0, 0
    for step, (x, d) in enumerate(zip(xs, ds), start=1):
        acc += x * d
        peak = max(peak, acc)
        assert acc < W64, (step, acc)
        if step % 3 == 0:
            before = acc
            acc = fold34(acc, r34)
            assert acc % q == before % q
            assert acc < (1 << 61) + (1 << 34)
    return acc % q, peak


@pytest.mark.parametrize("q", [LARGEST_31BIT_PRIME, 2147352577, 1073479681, 65537])
@pytest.mark.parametrize("steps", [1, 2, 3, 4, 16, 32])
def test_diagonal_pass_worst_case(q, steps):
    xs = [q - 1] * steps
    got, peak = diag_schedule(xs, xs, q)
    assert got == (steps * (q - 1) * (q - 1)) % q == steps % q
    assert peak < W64


def test_diagonal_pass_fold_bound_is_tight_enough():
    """The bound the kernel relies on: a folded word plus three more maximal products
    stays below 2^64 for every prime below 2^31 (the fold's r34 < q < 2^31)."""
    worst_fold = ((1 << 30) - 1) * (LARGEST_31BIT_PRIME - 1) + ((1 << 34) - 1)
    assert worst_fold < (1 << 61) + (1 << 34)
    assert worst_fold + 3 * (LARGEST_31BIT_PRIME - 1) ** 2 < W64
    # a fourth product would not fit: the fold interval of three steps is the longest safe one
    assert worst_fold + 4 * (LARGEST_31BIT_PRIME - 1) ** 2 >= W64


def test_diagonal_pass_random():
    g = np.random.Generator(np.random.PCG64(7))
    for q in (LARGEST_31BIT_PRIME, 2147352577, 1073479681):
        for steps in (5, 16, 31):
            xs = [int(v) for v in g.integers(0, q, steps)]
            ds = [int(v) for v in g.integers(0, q, steps)]
            got, _ = diag_schedule(xs, ds, q)
            assert got == sum(x * d for x, d in zip(xs, ds)) % q


@pytest.mark.parametrize("beta", [1, 2, 3, 4])
def test_inner_product_worst_case(beta):
    """beta <= 4 digits' products in one word before the reduction, plus nothing else: the
    pass-through term P sigma(c0) is added after the reduction, as a residue."""
    q = LARGEST_31BIT_PRIME
    acc = sum((q - 1) * (q - 1) for _ in range(beta))
    assert acc < W64
    assert acc % q == beta % q
