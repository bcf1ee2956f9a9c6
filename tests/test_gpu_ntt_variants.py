"""NTT kernel variants (fhe_ctx_set_ntt): on-the-fly register twiddles in the
block passes, the single-pass cluster transform, the streaming passes and the
persistent cooperative two-pass transform.  Every mode must give the
oracle's residues bit for bit: the stage entry points, a batched graph plan of
mixed key switches, hoisted rotations, HMult + rescale and the double-hoisted
transform."""
import numpy as np
import pytest

import oracle
from oracle import bootstrap_lt as blt
from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu

# 0, FHE_NTT_OTF, FHE_NTT_SINGLE_PASS, both; FHE_NTT_STREAM alone, with OTF, with SINGLE_PASS;
# FHE_NTT_PERSIST
MODES = [0, 1, 2, 3, 4, 5, 6, 8]


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


@pytest.mark.parametrize("mode", MODES)
def test_stage_transforms_each_mode(big, mode):
    P, OP, ctx = big
    ctx.set_ntt(mode)
    g = inputs.rng(1500 + mode)
    idx = [0, 5, 23, P.L, P.L + 7]  # q and p primes
    primes = [P.primes[i] for i in idx]
    a = np.stack([inputs.uniform_residues(g, [p], P.N)[0] for p in primes])
    t = dev(a)
    ctx.ntt(t, idx)
    fwd = host(ctx, t)
    assert np.array_equal(fwd, oracle.ntt(a, primes))
    ctx.intt(t, idx)
    assert np.array_equal(host(ctx, t), a)
    ctx.set_ntt(0)


@pytest.mark.parametrize("mode", MODES)
def test_batched_plan_each_mode(big, mode):
    """A graph plan of 6 mixed items (rotations and relinearisations, levels 3..24) per mode."""
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = big
    ctx.set_ntt(mode)
    g = inputs.rng(1600 + mode)
    rk = rand_key(P, g)
    ctx.set_relin_key(dev(rk))
    items, want = [], []
    for lv, rot in [(24, 3), (17, 0), (24, 1000), (3, 0), (9, 77), (24, 0)]:
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
    ctx.set_ntt(0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("fused", [True, False])
def test_single_ops_each_mode(big, mode, fused):
    """Hoisted rotations, HMult + rescale, one plain-pipeline rotation."""
    P, OP, ctx = big
    ctx.set_ntt(mode)
    ctx.set_fused(fused)
    g = inputs.rng(1700 + 2 * mode + int(fused))
    level = 20
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    keys = {}
    for r in (1, 5):
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    outs = ctx.rotate_hoisted(dev(ct), level, [1, 5])
    want = oracle.rotate_hoisted(OP, ct, level, [1, 5], [keys[1], keys[5]])
    for o, w in zip(outs, want):
        assert np.array_equal(host(ctx, o), w)
    assert np.array_equal(host(ctx, ctx.rotate(dev(ct), level, 5)), oracle.rotate(OP, ct, level, 5, keys[5]))
    rk = rand_key(P, g)
    ctx.set_relin_key(dev(rk))
    b = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    m = ctx.hmult(dev(ct), dev(b), level)
    r = ctx.rescale(m, level)
    wm = oracle.hmult(OP, ct, b, level, rk)
    assert np.array_equal(host(ctx, r), oracle.rescale(OP, wm, level))
    ctx.set_fused(True)
    ctx.set_ntt(0)


@pytest.mark.parametrize("mode", [1, 2, 3, 4, 6, 8])
def test_double_hoisted_level_each_mode(fhe_lib, mode):
    from paper_2512_18345_gb300 import binding
    name = "cts_stc_N65536_L48_a12"
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    W = inputs.WORKLOADS[name]
    plan = inputs.transform_plans(P.N, W["levels"], "stc")[2]
    level = W["stc_level"]
    g = inputs.rng(1800 + mode)
    ctx = binding.Context.from_params(P)
    ctx.set_ntt(mode)
    keys = {}
    for r in plan.rotations():
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    diags = np.stack([inputs.uniform_residues(g, tuple(P.q[:level]) + tuple(P.p), P.N) for _ in range(plan.n_diag)])
    got = host(ctx, ctx.linear_transform_dh(dev(ct), level, plan.baby, plan.giant, dev(diags), plan.idx))
    assert np.array_equal(got, blt.lt_double_hoisted(OP, ct, level, plan.baby, plan.giant, diags, plan.idx, keys))
    ctx.close()


def test_small_ring_modes(fhe_lib):
    """N = 2^12: on-the-fly twiddles apply; the single-pass and streaming transforms are 2^16-only."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    with pytest.raises(binding.FheError) as e:
        ctx.set_ntt(binding.FHE_NTT_SINGLE_PASS)
    assert e.value.code == binding.FHE_EUNSUPPORTED
    with pytest.raises(binding.FheError) as e:
        ctx.set_ntt(binding.FHE_NTT_STREAM)
    assert e.value.code == binding.FHE_EUNSUPPORTED
    with pytest.raises(binding.FheError) as e:
        ctx.set_ntt(binding.FHE_NTT_PERSIST)
    assert e.value.code == binding.FHE_EUNSUPPORTED
    with pytest.raises(binding.FheError) as e:
        ctx.set_ntt(16)
    assert e.value.code == binding.FHE_EINVAL
    ctx.set_ntt(binding.FHE_NTT_OTF)
    g = inputs.rng(1900)
    key = rand_key(P, g)
    ctx.set_rot_key(3, dev(key))
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    assert np.array_equal(host(ctx, ctx.rotate(dev(ct), P.L, 3)), oracle.rotate(OP, ct, P.L, 3, key))
    ctx.close()


def test_autotune_measures_ntt_modes(big):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = big
    r = ctx.autotune(P.L, 4, binding.FHE_TUNE_NTT)
    assert r["ntt_mode"] in MODES and r["candidates"] >= 3
    g = inputs.rng(2000)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    d = inputs.uniform_residues(g, P.q, P.N)
    assert np.array_equal(host(ctx, ctx.keyswitch(dev(d), P.L)), oracle.keyswitch(OP, d, P.L, key))
    ctx.set_ntt(0)


@pytest.mark.parametrize("n_limbs", [1, 7, 33, 130])
def test_streaming_passes_ragged_unit_counts(big, n_limbs):
    """Streaming passes with launches whose unit count does not divide evenly among the
    persistent CTAs, runs of limbs shorter than a block-pass run, repeated primes in one
    launch and all-(q - 1) limbs: equal to the oracle and to the two-pass kernels."""
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = big
    g = inputs.rng(2100 + n_limbs)
    idx = [(7 * i) % len(P.primes) for i in range(n_limbs)]
    primes = [P.primes[i] for i in idx]
    a = np.stack([inputs.uniform_residues(g, [p], P.N)[0] for p in primes])
    a[0] = primes[0] - 1
    got = {}
    for mode in (0, binding.FHE_NTT_STREAM):
        ctx.set_ntt(mode)
        t = dev(a)
        ctx.ntt(t, idx)
        f = host(ctx, t)
        ctx.intt(t, idx)
        got[mode] = (f, host(ctx, t))
    ctx.set_ntt(0)
    assert np.array_equal(got[0][0], got[binding.FHE_NTT_STREAM][0])
    assert np.array_equal(got[binding.FHE_NTT_STREAM][0], oracle.ntt(a, primes))
    assert np.array_equal(got[binding.FHE_NTT_STREAM][1], a)


def test_persistent_transform_rejects_other_flags(big):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = big
    for other in (binding.FHE_NTT_OTF, binding.FHE_NTT_SINGLE_PASS, binding.FHE_NTT_STREAM):
        with pytest.raises(binding.FheError) as e:
            ctx.set_ntt(binding.FHE_NTT_PERSIST | other)
        assert e.value.code == binding.FHE_EINVAL


@pytest.mark.parametrize("n_limbs", [1, 7, 33, 130, 400])
def test_persistent_transform_unit_counts(big, n_limbs):
    """The persistent two-pass transform with fewer tiles than resident CTAs (1 limb: 16 tiles),
    counts that do not divide among them and more limbs than one wave holds (400 limbs, 6400
    tiles per pass), repeated primes and all-(q - 1) limbs: equal to the oracle and to the
    two-pass kernels, forward and inverse, with no expired grid barrier."""
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = big
    g = inputs.rng(2300 + n_limbs)
    idx = [(5 * i) % len(P.primes) for i in range(n_limbs)]
    primes = [P.primes[i] for i in idx]
    a = np.stack([inputs.uniform_residues(g, [p], P.N)[0] for p in primes])
    a[-1] = primes[-1] - 1
    got = {}
    for mode in (0, binding.FHE_NTT_PERSIST):
        ctx.set_ntt(mode)
        t = dev(a)
        ctx.ntt(t, idx)
        f = host(ctx, t)
        ctx.intt(t, idx)
        got[mode] = (f, host(ctx, t))
    ctx.set_ntt(0)
    assert np.array_equal(got[binding.FHE_NTT_PERSIST][0], got[0][0])
    assert np.array_equal(got[binding.FHE_NTT_PERSIST][1], a)
    if n_limbs <= 33:
        assert np.array_equal(got[0][0], oracle.ntt(a, primes))
