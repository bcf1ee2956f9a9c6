"""GPU parity on primes from every part of the accepted range (2^20, 2^31).

The workloads use the largest NTT-friendly primes below 2^31 (or 2^30), whose
2^32 mod q is small.  Constants derived from 2^32 mod q by shifts can wrap for
other primes: for q in (4/3 2^30, 3/2 2^30], 2^32 mod q = 2^32 - 2q is at least
2^30, so 4 (2^32 mod q) no longer fits a 32-bit word.  This file runs every
operation on one context whose primes come from such ranges, in an unsorted
order, and compares each result with the oracle residue by residue:

* the largest prime below 2^31 (2^32 mod q is tiny);
* primes in (4/3 2^30, 3/2 2^30] (2^32 mod q >= 2^30);
* a prime just below 2^30 + 2^23 (the tensor-core epilogue's reduction bound);
* primes just above 2^20 (the smallest accepted), and one near 2^26.
"""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu

N = 1 << 12
LO, HI = (4 << 30) // 3, (3 << 30) // 2


def odd_range_params():
    two_n = 2 * N
    mid = inputs.ntt_primes(N, 31, 3, below=HI + 1)
    assert all(LO < q <= HI for q in mid)
    assert all(((1 << 32) % q) >= (1 << 30) for q in mid)
    top = inputs.ntt_primes(N, 31, 1)
    tc_edge = inputs.ntt_primes(N, 31, 1, below=(1 << 30) + (1 << 23))
    small = []
    c = (1 << 20) + 1
    while len(small) < 2:
        c += two_n
        if inputs.is_prime(c):
            small.append(c)
    near26 = inputs.ntt_primes(N, 26, 1)
    q = (mid[0], small[0], top[0], tc_edge[0], near26[0], mid[1])
    p = (small[1], mid[2])
    return inputs.Params(N=N, q=q, p=p, dnum=3)


@pytest.fixture(scope="module")
def odd(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = odd_range_params()
    ctx = binding.Context.from_params(P)
    yield P, oracle.OracleParams.from_params(P), ctx
    ctx.close()


def dev(a):
    from paper_2512_18345_gb300 import binding
    return binding.to_device(a)


def host(ctx, t):
    from paper_2512_18345_gb300 import binding
    ctx.sync()
    return binding.to_numpy(t)


def rand_key(P, g):
    return np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)]) for _ in range(P.dnum)])


def test_ntt_and_bconv(odd):
    P, OP, ctx = odd
    g = inputs.rng(900)
    idx = list(range(len(P.primes)))
    a = inputs.uniform_residues(g, P.primes, P.N)
    t = dev(a)
    ctx.ntt(t, idx)
    assert np.array_equal(host(ctx, t), oracle.ntt(a, P.primes))
    ctx.intt(t, idx)
    assert np.array_equal(host(ctx, t), a)
    x = inputs.uniform_residues(g, P.q[:3], P.N)
    x[:, :8] = np.array(P.q[:3], dtype=np.uint32)[:, None] - 1
    want = oracle.bconv(x, P.q[:3], P.q[3:] + P.p)
    assert np.array_equal(host(ctx, ctx.bconv(dev(x), [0, 1, 2], [3, 4, 5, 6, 7])), want)


@pytest.mark.parametrize("bconv", [0, 1])
@pytest.mark.parametrize("level", [6, 5, 1])
def test_keyswitch_rotate_hmult_rescale(odd, bconv, level):
    P, OP, ctx = odd
    ctx.set_bconv(bconv)
    g = inputs.rng(910 + level)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    d = inputs.uniform_residues(g, P.q[:level], P.N)
    assert np.array_equal(host(ctx, ctx.keyswitch(dev(d), level)), oracle.keyswitch(OP, d, level, key))
    rot = 1 + level
    rkey = rand_key(P, g)
    ctx.set_rot_key(rot, dev(rkey))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    assert np.array_equal(host(ctx, ctx.rotate(dev(ct), level, rot)), oracle.rotate(OP, ct, level, rot, rkey))
    ct2 = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    m = ctx.hmult(dev(ct), dev(ct2), level)
    want_m = oracle.hmult(OP, ct, ct2, level, key)
    assert np.array_equal(host(ctx, m), want_m)
    if level > 1:
        assert np.array_equal(host(ctx, ctx.rescale(m, level)), oracle.rescale(OP, want_m, level))
    ctx.set_bconv(0)


def test_rotate_hoisted(odd):
    P, OP, ctx = odd
    g = inputs.rng(930)
    rots = [0, 3, 7, 100]
    keys = [None] + [rand_key(P, g) for _ in rots[1:]]
    for r, k in zip(rots[1:], keys[1:]):
        ctx.set_rot_key(r, dev(k))
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    outs = ctx.rotate_hoisted(dev(ct), P.L, rots)
    want = oracle.rotate_hoisted(OP, ct, P.L, rots, keys)
    for i in range(len(rots)):
        assert np.array_equal(host(ctx, outs[i]), want[i]), f"rotation {rots[i]}"


def test_linear_transform_bsgs(odd):
    """The diagonal pass folds its 64-bit accumulators with 2^34 mod q: the constant that
    wraps in 32 bits for the middle primes here."""
    P, OP, ctx = odd
    g = inputs.rng(940)
    baby, giant, level = 8, 3, P.L
    keys = {}
    for r in list(range(1, baby)) + [baby * gg for gg in range(1, giant)]:
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    qm1 = np.array([q - 1 for q in P.q], dtype=np.uint32)[:, None] * np.ones((1, P.N), dtype=np.uint32)
    ct = np.stack([qm1, inputs.uniform_residues(g, P.q, P.N)])
    diags = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(baby * giant)])
    diags[: baby] = qm1
    got = host(ctx, ctx.linear_transform(dev(ct), level, dev(diags), baby, giant))
    assert np.array_equal(got, oracle.bsgs_linear_transform(OP, ct, level, diags, baby, giant, keys))


def test_linear_transform_double_hoisted(odd):
    from oracle import bootstrap_lt
    P, OP, ctx = odd
    g = inputs.rng(950)
    plan = inputs.transform_plans(P.N, 3, "cts")[1]
    lv = P.L
    keys = {}
    for r in plan.rotations():
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    diags = np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(plan.n_diag)])
    got = host(ctx, ctx.linear_transform_dh(dev(ct), lv, plan.baby, plan.giant, dev(diags), plan.idx))
    want = bootstrap_lt.lt_double_hoisted(OP, ct, lv, plan.baby, plan.giant, diags, plan.idx, keys)
    assert np.array_equal(got, want)
