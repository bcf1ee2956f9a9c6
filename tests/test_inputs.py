"""The seeded input generators: parameters and distributions."""
import numpy as np
import pytest

from paper_2512_18345_gb300 import inputs


@pytest.mark.parametrize("name", list(inputs.WORKLOADS))
def test_workload_primes(name):
    P = inputs.workload_params(name)
    w = inputs.WORKLOADS[name]
    allp = P.primes
    assert len(set(allp)) == len(allp) == w["L"] + w["K"]
    assert list(allp) == sorted(allp, reverse=True)
    for q in allp:
        assert inputs.is_prime(q) and q % (2 * P.N) == 1 and q < 2 ** w["bits"]
    # they are the largest such primes: nothing prime and NTT-friendly is skipped
    c = allp[0] + 2 * P.N
    while c < 2 ** w["bits"]:
        assert not inputs.is_prime(c)
        c += 2 * P.N


def test_is_prime_small():
    small = [n for n in range(2, 2000) if all(n % d for d in range(2, int(n ** 0.5) + 1))]
    assert [n for n in range(2000) if inputs.is_prime(n)] == small


def test_distributions():
    g = inputs.rng(7)
    s = inputs.ternary(g, 1 << 16)
    assert set(np.unique(s)) == {-1, 0, 1}
    e = inputs.gaussian(g, 1 << 16)
    assert np.abs(e).max() <= inputs.ERR_BOUND and abs(e.std() - inputs.SIGMA) < 0.1
    z = inputs.complex_slots(g, 1000)
    assert np.abs(z.real).max() <= 1 and np.abs(z.imag).max() <= 1
    r = inputs.uniform_residues(g, [97, 2 ** 31 - 1], 4096)
    assert r[0].max() < 97 and r.dtype == np.uint32


def test_seeded_reproducible():
    a = inputs.uniform_residues(inputs.rng(5), [2 ** 31 - 1], 8)
    b = inputs.uniform_residues(inputs.rng(5), [2 ** 31 - 1], 8)
    assert np.array_equal(a, b)
    items = inputs.batch_items(inputs.rng(9), 64, 4, 24)
    assert len(items) == 64 and all(4 <= it["level"] <= 24 and 1 <= it["rot"] < 2 ** 15 for it in items)
