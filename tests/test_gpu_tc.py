"""Tensor-core base conversion (tcgen05, bf16 byte digits, fp32 accumulation in
tensor memory): bit-exact against the CPU oracle and against the CUDA-core
path, alone and inside full key switches (the N = 2^16, L = 24 rotation with
tensor-core BConv is the third workload)."""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hrotate_N65536_L24_tc")
    ctx = binding.Context.from_params(P)
    ctx.set_bconv(binding.FHE_BCONV_TC)
    yield P, oracle.OracleParams.from_params(P), ctx
    ctx.close()


@pytest.fixture(scope="module")
def tc_small(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    ctx = binding.Context.from_params(P)
    ctx.set_bconv(binding.FHE_BCONV_TC)
    yield P, oracle.OracleParams.from_params(P), ctx
    ctx.close()


def dev(a):
    from paper_2512_18345_gb300 import binding
    return binding.to_device(a)


def host(ctx, t):
    from paper_2512_18345_gb300 import binding
    ctx.sync()  # raises if a bounded tensor-core wait expired
    return binding.to_numpy(t)


def rand_key(P, g):
    return np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)]) for _ in range(P.dnum)])


@pytest.mark.parametrize("n_in,n_out", [(1, 5), (3, 29), (8, 24), (4, 16), (2, 30), (9, 20), (12, 24), (11, 21),
                                         (12, 1)])
def test_bconv_tc_parity(tc, n_in, n_out):
    P, OP, ctx = tc
    g = inputs.rng(300 + n_in)
    in_idx = list(range(32 - n_in, 32))
    out_idx = list(range(n_out))
    pin = [P.primes[i] for i in in_idx]
    pout = [P.primes[i] for i in out_idx]
    x = inputs.uniform_residues(g, pin, P.N)
    got = host(ctx, ctx.bconv(dev(x), in_idx, out_idx))
    assert np.array_equal(got, oracle.bconv(x, pin, pout))


@pytest.mark.parametrize("fill", ["max", "zero", "ones"])
@pytest.mark.parametrize("n_in", [8, 12])
def test_bconv_tc_extremes(tc, fill, n_in):
    P, OP, ctx = tc
    in_idx, out_idx = list(range(32 - n_in, 32)), list(range(24))
    pin = [P.primes[i] for i in in_idx]
    pout = [P.primes[i] for i in out_idx]
    if fill == "max":
        x = np.array([[q - 1] * P.N for q in pin], np.uint32)
    elif fill == "zero":
        x = np.zeros((n_in, P.N), np.uint32)
    else:
        x = np.ones((n_in, P.N), np.uint32)
    got = host(ctx, ctx.bconv(dev(x), in_idx, out_idx))
    assert np.array_equal(got, oracle.bconv(x, pin, pout))


@pytest.mark.parametrize("level", [24, 17, 8, 1])
def test_keyswitch_tc_equals_scalar_and_oracle(tc, level):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = tc
    g = inputs.rng(310 + level)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    d = inputs.uniform_residues(g, P.q[:level], P.N)
    got_tc = host(ctx, ctx.keyswitch(dev(d), level, binding.FHE_RELIN_KEY))
    ctx.set_bconv(binding.FHE_BCONV_SCALAR)
    got_sc = host(ctx, ctx.keyswitch(dev(d), level, binding.FHE_RELIN_KEY))
    ctx.set_bconv(binding.FHE_BCONV_TC)
    assert np.array_equal(got_tc, got_sc)
    assert np.array_equal(got_tc, oracle.keyswitch(OP, d, level, key))


def test_rotate_tc_full_size(tc):
    P, OP, ctx = tc
    g = inputs.rng(320)
    rot = inputs.rotation_index(g)
    key = rand_key(P, g)
    ctx.set_rot_key(rot, dev(key))
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    got = host(ctx, ctx.rotate(dev(ct), P.L, rot))
    assert np.array_equal(got, oracle.rotate(OP, ct, P.L, rot, key))


def test_hmult_tc_small_ring(tc_small):
    P, OP, ctx = tc_small
    g = inputs.rng(330)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    a = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    b = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    got = host(ctx, ctx.hmult(dev(a), dev(b), P.L))
    assert np.array_equal(got, oracle.hmult(OP, a, b, P.L, key))


def test_batch_plan_tc(tc):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = tc
    g = inputs.rng(340)
    items, want = [], []
    for lv, rot in [(24, 5), (13, 900), (4, 31000)]:
        k = rand_key(P, g)
        ctx.set_rot_key(rot, dev(k))
        a = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
        items.append(dict(op=binding.FHE_OP_ROTATE, level=lv, rot=rot, **{"in": dev(a)}, out=binding.empty((2, lv, P.N))))
        want.append(oracle.rotate(OP, a, lv, rot, k))
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    plan.launch()
    for it, w in zip(items, want):
        assert np.array_equal(host(ctx, it["out"]), w)
    plan.close()
