"""Baby-step / giant-step linear transform (the fifth workload's shape):
bit-exact against the oracle's composition of hoisted baby rotations,
diagonal multiply-accumulate and giant rotations, and decoded against the
FP64 matrix-vector product."""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu


def dev(a):
    from paper_2512_18345_gb300 import binding
    return binding.to_device(a)


def host(ctx, t):
    from paper_2512_18345_gb300 import binding
    ctx.sync()
    return binding.to_numpy(t)


def rand_key(P, g):
    return np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)]) for _ in range(P.dnum)])


@pytest.mark.parametrize("name,level,baby,giant", [("hmult_relin_rescale_N4096_L4", 4, 4, 2),
                                                   ("hmult_relin_rescale_N4096_L4", 3, 5, 3),
                                                   ("bsgs_lt_N65536_L24", 8, 16, 8)])
def test_linear_transform_parity(fhe_lib, name, level, baby, giant):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    g = inputs.rng(500 + baby)
    keys = {}
    for r in list(range(1, baby)) + [baby * gg for gg in range(1, giant)]:
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    diags = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(baby * giant)])
    got = host(ctx, ctx.linear_transform(dev(ct), level, dev(diags), baby, giant))
    want = oracle.bsgs_linear_transform(OP, ct, level, diags, baby, giant, keys)
    assert np.array_equal(got, want)
    ctx.close()


@pytest.mark.parametrize("name,level,baby,giant", [("hmult_relin_rescale_N4096_L4", 4, 32, 5),
                                                   ("bsgs_lt_N65536_L24", 8, 16, 8)])
def test_linear_transform_extreme_products(fhe_lib, name, level, baby, giant):
    """Every c0 product of the diagonal pass at its maximum.  Zero rotation keys make each
    rotation exactly (sigma(c0), 0); with c0 = q - 1 on every coefficient (a constant, which
    every automorphism keeps) and every diagonal q - 1, each c0 product is (q - 1)^2, just
    below 2^62, so the pass's 64-bit accumulators run at the bound their folds are sized for.
    (q - 1)^2 = 1 mod q, so the output's c0 is the constant baby * giant mod q; its c1 comes
    from the identity pair alone: (q - 1) c1 = -c1 mod q."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    g = inputs.rng(520 + baby)
    zero = np.zeros((P.dnum, 2, len(P.primes), P.N), dtype=np.uint32)
    keys = {}
    for r in list(range(1, baby)) + [baby * gg for gg in range(1, giant)]:
        keys[r] = zero
        ctx.set_rot_key(r, dev(zero))
    qm1 = np.array([q - 1 for q in P.q[:level]], dtype=np.uint32)[:, None] * np.ones((1, P.N), dtype=np.uint32)
    ct = np.stack([qm1, inputs.uniform_residues(g, P.q[:level], P.N)])
    diags = np.broadcast_to(qm1, (baby * giant, level, P.N)).copy()
    got = host(ctx, ctx.linear_transform(dev(ct), level, dev(diags), baby, giant))
    want = oracle.bsgs_linear_transform(OP, ct, level, diags, baby, giant, keys)
    assert np.array_equal(got, want)
    closed = np.array([(baby * giant) % q for q in P.q[:level]], dtype=np.uint32)[:, None]
    assert np.array_equal(got[0], np.broadcast_to(closed, (level, P.N)))
    qs = np.array(P.q[:level], dtype=np.int64)[:, None]
    assert np.array_equal(got[1].astype(np.int64), (qs - ct[1].astype(np.int64)) % qs)
    ctx.close()


def test_linear_transform_decodes_to_matvec(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    g = inputs.rng(510)
    sk = oracle.SecretKey(OP, inputs.ternary(g, P.N))
    z = inputs.complex_slots(g, P.N // 2)
    scale, dscale = 2.0 ** 25, 2.0 ** 20
    ct = oracle.encrypt(OP, sk, oracle.encode(z, scale, P.N), P.L, g)
    baby, giant = 4, 2
    for r in list(range(1, baby)) + [baby * gg for gg in range(1, giant)]:
        ctx.set_rot_key(r, dev(oracle.rotation_key(OP, sk, r, g)))
    diag_slots = [inputs.complex_slots(g, P.N // 2) for _ in range(baby * giant)]
    pd = []
    for gg in range(giant):
        for b in range(baby):
            dv = np.roll(diag_slots[gg * baby + b], baby * gg)
            pd.append(oracle.ntt(oracle.to_rns(oracle.encode(dv, dscale, P.N), P.q), P.q))
    out = host(ctx, ctx.linear_transform(dev(ct), P.L, dev(np.stack(pd)), baby, giant))
    dec = oracle.decode(oracle.decrypt(OP, sk, out, P.L), scale * dscale, P.N)
    want = sum(diag_slots[k] * np.roll(z, -k) for k in range(baby * giant))
    assert np.abs(dec - want).max() < 2.0 ** -1
    ctx.close()
