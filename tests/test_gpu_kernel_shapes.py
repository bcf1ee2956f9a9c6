"""Kernel shapes (fhe_ctx_set_kernel_shape) and the fused special-limb inner
product + first ModDown pass: every shape gives the oracle's residues bit for
bit, alone and with the NTT variants, in single operations and batched plans;
the autotuner's shape search applies a valid shape and records it in its cache."""
import itertools

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


@pytest.fixture(scope="module")
def big(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hrotate_N65536_L24_tc")
    ctx = binding.Context.from_params(P)
    yield P, oracle.OracleParams.from_params(P), ctx
    ctx.close()


@pytest.mark.parametrize("bconv", [0, 1])
@pytest.mark.parametrize("pipe", [True, False])
@pytest.mark.parametrize("level", [24, 17, 9, 1])
def test_fused_ip_moddown_single_ops(big, bconv, pipe, level):
    """Key switch, rotation and HMult with the fused kernel, digits 1..3 (level 1: one limb)."""
    P, OP, ctx = big
    ctx.set_kernel_shape(fuse_ip_moddown=1)
    ctx.set_bconv(bconv)
    ctx.set_pipelining(pipe)
    g = inputs.rng(3000 + 4 * level + 2 * bconv + int(pipe))
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    d = inputs.uniform_residues(g, P.q[:level], P.N)
    d[:, :5] = np.array(P.q[:level], dtype=np.uint32)[:, None] - 1
    assert np.array_equal(host(ctx, ctx.keyswitch(dev(d), level)), oracle.keyswitch(OP, d, level, key))
    rot = 11 + level
    rk = rand_key(P, g)
    ctx.set_rot_key(rot, dev(rk))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    assert np.array_equal(host(ctx, ctx.rotate(dev(ct), level, rot)), oracle.rotate(OP, ct, level, rot, rk))
    ct2 = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    assert np.array_equal(host(ctx, ctx.hmult(dev(ct), dev(ct2), level)), oracle.hmult(OP, ct, ct2, level, key))
    ctx.set_kernel_shape(fuse_ip_moddown=0)
    ctx.set_bconv(0)
    ctx.set_pipelining(True)


@pytest.mark.parametrize("ntt_mode", [0, 2, 4, 6])
def test_fused_in_batched_plan_with_hoisted_items(big, ntt_mode):
    """A graph plan mixing fused key switches with hoisted rotations (their digits go through
    the automorphism, so they keep the unfused pair), under each NTT mode."""
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = big
    ctx.set_kernel_shape(fuse_ip_moddown=1)
    ctx.set_ntt(ntt_mode)
    g = inputs.rng(3100 + ntt_mode)
    rk = rand_key(P, g)
    ctx.set_relin_key(dev(rk))
    items, want = [], []
    for lv, rot in [(24, 5), (13, 0), (24, 0), (7, 900), (2, 0)]:
        a = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
        if rot:
            k = rand_key(P, g)
            ctx.set_rot_key(rot, dev(k))
            items.append(dict(op=binding.FHE_OP_ROTATE, level=lv, rot=rot, **{"in": dev(a)},
                              out=binding.empty((2, lv, P.N))))
            want.append(oracle.rotate(OP, a, lv, rot, k))
        else:
            b = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
            items.append(dict(op=binding.FHE_OP_RELIN, level=lv, **{"in": dev(a)}, in2=dev(b),
                              out=binding.empty((2, lv, P.N))))
            want.append(oracle.hmult(OP, a, b, lv, rk))
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    for _ in range(2):
        plan.launch()
        for it, w in zip(items, want):
            assert np.array_equal(host(ctx, it["out"]), w)
    plan.close()
    # hoisted rotations with the fused shape set: their ModDown halves stay unfused
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    rots = [0, 3, 77]
    keys = [None] + [rand_key(P, g) for _ in rots[1:]]
    for r, k in zip(rots[1:], keys[1:]):
        ctx.set_rot_key(r, dev(k))
    outs = ctx.rotate_hoisted(dev(ct), P.L, rots)
    ref = oracle.rotate_hoisted(OP, ct, P.L, rots, keys)
    for o, w in zip(outs, ref):
        assert np.array_equal(host(ctx, o), w)
    ctx.set_ntt(0)
    ctx.set_kernel_shape(fuse_ip_moddown=0)


def test_fused_at_four_digits(fhe_lib):
    """The paper's (48, 12, 4) shape: four digits of twelve limbs, K = 12."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("paper_ks_N65536_L48_a12")
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    ctx.set_kernel_shape(fuse_ip_moddown=1)
    g = inputs.rng(3200)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    for level in (48, 37):
        d = inputs.uniform_residues(g, P.q[:level], P.N)
        assert np.array_equal(host(ctx, ctx.keyswitch(dev(d), level)), oracle.keyswitch(OP, d, level, key))
    ctx.close()


def test_every_shape_candidate_bit_exact(big):
    """Each value the autotuner may pick (alone and in combination) on a two-item plan."""
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = big
    g = inputs.rng(3300)
    rk = rand_key(P, g)
    ctx.set_relin_key(dev(rk))
    a = [np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)]) for _ in range(2)]
    want = [oracle.hmult(OP, a[0], a[1], P.L, rk), oracle.hmult(OP, a[1], a[0], P.L, rk)]
    ctx.set_bconv(binding.FHE_BCONV_TC)
    ctx.set_ntt(binding.FHE_NTT_STREAM)
    for fuse, pipe, tc, st, nc in itertools.product([0, 1], [0, 1], [1, 2, 3, 4], [2, 3], [1, 2, 3]):
        if (tc, st, nc) not in [(4, 3, 3), (1, 2, 1), (2, 3, 2), (3, 2, 3)]:
            continue
        ctx.set_kernel_shape(fuse_ip_moddown=fuse, bconv_tc_ctas=tc, ntt_stream_stages=st, ntt_stream_ctas=nc,
                             bconv_tc_pipeline=pipe)
        items = [dict(op=binding.FHE_OP_RELIN, level=P.L, **{"in": dev(a[i])}, in2=dev(a[1 - i]),
                      out=binding.empty((2, P.L, P.N))) for i in range(2)]
        plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
        plan.launch()
        for it, w in zip(items, want):
            assert np.array_equal(host(ctx, it["out"]), w), (fuse, pipe, tc, st, nc)
        plan.close()
    ctx.set_kernel_shape(fuse_ip_moddown=0, bconv_tc_ctas=4, ntt_stream_stages=3, ntt_stream_ctas=3,
                         bconv_tc_pipeline=0)
    ctx.set_ntt(0)
    ctx.set_bconv(0)


def test_kernel_shape_validation(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    ctx = binding.Context.from_params(P)
    assert ctx.kernel_shape() == {"fuse_ip_moddown": 0, "bconv_tc_ctas": 4, "ntt_stream_stages": 3,
                                  "ntt_stream_ctas": 3, "bconv_tc_pipeline": 0, "ip_staged_gather": 1,
                                  "ip_staged_ctas": 2, "ip_staged_depth": 0}
    with pytest.raises(binding.FheError) as e:
        ctx.set_kernel_shape(fuse_ip_moddown=1)  # the fused kernel is 2^16-only
    assert e.value.code == binding.FHE_EUNSUPPORTED
    for bad in ({"bconv_tc_ctas": 0}, {"bconv_tc_ctas": 5}, {"ntt_stream_stages": 1}, {"ntt_stream_ctas": 4},
                {"fuse_ip_moddown": 2}, {"bconv_tc_pipeline": 2}, {"ip_staged_gather": 2},
                {"ip_staged_gather": -1}, {"ip_staged_ctas": 0}, {"ip_staged_ctas": 3},
                {"ip_staged_depth": 1}, {"ip_staged_depth": 5}, {"ip_staged_depth": -1}):
        with pytest.raises(binding.FheError) as e:
            ctx.set_kernel_shape(**bad)
        assert e.value.code == binding.FHE_EINVAL
    assert ctx.kernel_shape()["bconv_tc_ctas"] == 4  # rejected calls change nothing
    ctx.close()


def test_autotune_shape_search_applies_and_records(fhe_lib, tmp_path):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hrotate_N65536_L24_tc")
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    ctx.set_bconv(binding.FHE_BCONV_TC)
    path = tmp_path / "tune.txt"
    r = ctx.autotune(P.L, 4, binding.FHE_TUNE_SHAPE, cache=str(path))
    assert r["candidates"] >= 3
    assert ctx.kernel_shape() == r["shape"]
    assert "fuse=" in path.read_text()
    g = inputs.rng(3400)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    d = inputs.uniform_residues(g, P.q, P.N)
    assert np.array_equal(host(ctx, ctx.keyswitch(dev(d), P.L)), oracle.keyswitch(OP, d, P.L, key))
    ctx.close()
    ctx2 = binding.Context.from_params(P)
    ctx2.set_bconv(binding.FHE_BCONV_TC)
    r2 = ctx2.autotune(P.L, 4, binding.FHE_TUNE_SHAPE, cache=str(path))
    assert r2["candidates"] == 0 and r2["shape"] == r["shape"] and ctx2.kernel_shape() == r["shape"]
    ctx2.close()


@pytest.mark.parametrize("n_in,n_out", [(1, 5), (3, 24), (8, 24), (2, 30), (5, 27)])
@pytest.mark.parametrize("ctas", [1, 2])
def test_pipelined_tc_bconv_parity(big, n_in, n_out, ctas):
    """The two-accumulator tensor-core BConv against the oracle, with random and all-(q - 1)
    inputs, output counts that take one or two tensor-memory buffers per CTA."""
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = big
    ctx.set_bconv(binding.FHE_BCONV_TC)
    ctx.set_kernel_shape(bconv_tc_pipeline=1, bconv_tc_ctas=ctas)
    g = inputs.rng(3500 + 7 * n_in + n_out)
    in_idx = list(range(n_in))
    out_idx = [n_in + i for i in range(n_out)]
    pin = [P.primes[i] for i in in_idx]
    pout = [P.primes[i] for i in out_idx]
    x = inputs.uniform_residues(g, pin, P.N)
    x[:, : P.N // 4] = np.array(pin, dtype=np.uint32)[:, None] - 1
    got = host(ctx, ctx.bconv(dev(x), in_idx, out_idx))
    assert np.array_equal(got, oracle.bconv(x, pin, pout))
    ctx.set_kernel_shape(bconv_tc_pipeline=0, bconv_tc_ctas=4)
    ctx.set_bconv(0)


def test_pipelined_tc_bconv_twelve_limb_digits(fhe_lib):
    """The K = 64 contraction (digits of 12 limbs) in the pipelined kernel: a key switch at
    the paper's (48, 12, 4) shape."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("paper_ks_N65536_L48_a12")
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    ctx.set_bconv(binding.FHE_BCONV_TC)
    ctx.set_kernel_shape(bconv_tc_pipeline=1, fuse_ip_moddown=1)
    g = inputs.rng(3600)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    d = inputs.uniform_residues(g, P.q, P.N)
    assert np.array_equal(host(ctx, ctx.keyswitch(dev(d), P.L)), oracle.keyswitch(OP, d, P.L, key))
    ctx.close()


SHAPES_HOISTED = [dict(ip_staged_gather=1, ip_staged_ctas=2), dict(ip_staged_gather=1, ip_staged_ctas=1),
                  dict(ip_staged_gather=1, ip_staged_ctas=2, ip_staged_depth=3),
                  dict(ip_staged_gather=1, ip_staged_ctas=1, ip_staged_depth=4), dict(ip_staged_gather=0)]


@pytest.mark.parametrize("staged", range(len(SHAPES_HOISTED)))
@pytest.mark.parametrize("name,level,rots", [("hmult_relin_rescale_N4096_L4", 4, [0, 1, 2, 5, 15, -1]),
                                             ("hmult_relin_rescale_N4096_L4", 1, [3, 2047]),
                                             ("hrotate_N65536_L24_tc", 24, [0, 1, 7, 100]),
                                             ("hrotate_N65536_L24_tc", 11, [1, -3])])
def test_hoisted_inner_product_both_gathers(fhe_lib, staged, name, level, rots):
    """Hoisted rotations (sigma applied to the extended digits) through the staged-block kernel
    (one or two CTAs per SM) and through the gathering one: each equals the oracle bit for bit, at digit counts 1..3 and
    with the identity rotation in the batch (sigma_1 beside proper automorphisms)."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    ctx.set_kernel_shape(**SHAPES_HOISTED[staged])
    g = inputs.rng(3700 + level + 17 * staged)
    keys = [None if r % (P.N // 2) == 0 else rand_key(P, g) for r in rots]
    for r, k in zip(rots, keys):
        if k is not None:
            ctx.set_rot_key(r, dev(k))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    ct[:, :, : P.N // 8] = np.array(P.q[:level], dtype=np.uint32)[None, :, None] - 1  # the largest residues
    outs = ctx.rotate_hoisted(dev(ct), level, rots)
    want = oracle.rotate_hoisted(OP, ct, level, rots, keys)
    for i, r in enumerate(rots):
        assert np.array_equal(host(ctx, outs[i]), want[i]), f"rotation {r}"
    ctx.close()


@pytest.mark.parametrize("staged", range(len(SHAPES_HOISTED)))
def test_double_hoisted_level_both_gathers(fhe_lib, staged):
    """A double-hoisted CoeffToSlot level (baby-step inner products over the extended basis,
    giant steps on the extended sums) with either hoisted inner product."""
    from oracle import bootstrap_lt as blt
    from paper_2512_18345_gb300 import binding
    name = "cts_stc_N4096_L8"
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    W = inputs.WORKLOADS[name]
    plan = inputs.transform_plans(P.N, W["levels"], "cts")[1]
    level = W["cts_level"] - 1
    g = inputs.rng(3800 + staged)
    ctx = binding.Context.from_params(P)
    ctx.set_kernel_shape(**SHAPES_HOISTED[staged])
    keys = {}
    for r in plan.rotations():
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    xp = tuple(P.q[:level]) + tuple(P.p)
    diags = np.stack([inputs.uniform_residues(g, xp, P.N) for _ in range(plan.n_diag)])
    got = host(ctx, ctx.linear_transform_dh(dev(ct), level, plan.baby, plan.giant, dev(diags), plan.idx))
    assert np.array_equal(got, blt.lt_double_hoisted(OP, ct, level, plan.baby, plan.giant, diags, plan.idx, keys))
    ctx.close()
