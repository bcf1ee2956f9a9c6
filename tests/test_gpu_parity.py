"""GPU parity: every C-ABI entry point against the CPU oracle, residue by
residue (bit-exact: the whole path computes exact residues).

Sizes: N = 2^12 with L = 4, K = 2, dnum = 2 (several tiles and every level),
and the full key-switching shape N = 2^16, L = 24, K = 8, dnum = 3.  Edge
cases: level 1 (one-limb digit), partial last digit, the identity rotation
(index 0 and N/2), negative rotation indices, all-zero and all-(q-1) inputs.
"""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu

CFG1 = "hmult_relin_rescale_N4096_L4"
CFG2 = "hrotate_N65536_L24_plain"


def mk(fhe_lib, name, fused=True, bconv=0):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params(name)
    ctx = binding.Context.from_params(P)
    ctx.set_fused(fused)
    ctx.set_bconv(bconv)
    return P, oracle.OracleParams.from_params(P), ctx


@pytest.fixture(scope="module")
def c1(fhe_lib):
    return mk(fhe_lib, CFG1)


@pytest.fixture(scope="module")
def c2(fhe_lib):
    return mk(fhe_lib, CFG2)


def dev(a):
    from paper_2512_18345_gb300 import binding
    return binding.to_device(a)


def host(t):
    import torch
    from paper_2512_18345_gb300 import binding
    torch.cuda.synchronize()
    return binding.to_numpy(t)


def rand_key(P, g):
    return np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)]) for _ in range(P.dnum)])


# ------------------------------------------------------------------ transforms

@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_ntt_intt_parity(cfg, request):
    P, OP, ctx = request.getfixturevalue(cfg)
    g = inputs.rng(1)
    idx = list(range(len(P.primes)))
    a = inputs.uniform_residues(g, P.primes, P.N)
    a[0] = 0
    a[1] = P.primes[1] - 1
    t = dev(a)
    ctx.ntt(t, idx)
    got = host(t)
    assert np.array_equal(got, oracle.ntt(a, P.primes))
    ctx.intt(t, idx)
    assert np.array_equal(host(t), a)
    b = inputs.uniform_residues(g, P.primes, P.N)
    t = dev(b)
    ctx.intt(t, idx)
    assert np.array_equal(host(t), oracle.intt(b, P.primes))


def test_ntt_noncontiguous_primes_and_empty(c2):
    P, OP, ctx = c2
    g = inputs.rng(2)
    idx = [30, 3, 4, 5, 17, 24]
    pr = [P.primes[i] for i in idx]
    a = inputs.uniform_residues(g, pr, P.N)
    t = dev(a)
    ctx.ntt(t, idx)
    assert np.array_equal(host(t), oracle.ntt(a, pr))
    ctx.ntt(t, [])  # empty list: no work, no error


# ------------------------------------------------------------------ base conversion

@pytest.mark.parametrize("n_in,n_out", [(1, 5), (4, 12), (8, 24), (3, 29)])
def test_bconv_parity(c2, n_in, n_out):
    P, OP, ctx = c2
    g = inputs.rng(10 + n_in)
    in_idx = list(range(n_in))
    out_idx = list(range(n_in, n_in + n_out))
    pin = [P.primes[i] for i in in_idx]
    pout = [P.primes[i] for i in out_idx]
    x = inputs.uniform_residues(g, pin, P.N)
    got = host(ctx.bconv(dev(x), in_idx, out_idx))
    assert np.array_equal(got, oracle.bconv(x, pin, pout))


@pytest.mark.parametrize("fill", ["max", "zero"])
def test_bconv_extremes(c2, fill):
    P, OP, ctx = c2
    in_idx, out_idx = list(range(24, 32)), list(range(24))
    pin = [P.primes[i] for i in in_idx]
    pout = [P.primes[i] for i in out_idx]
    x = np.array([[q - 1] * P.N for q in pin], np.uint32) if fill == "max" else np.zeros((8, P.N), np.uint32)
    got = host(ctx.bconv(dev(x), in_idx, out_idx))
    assert np.array_equal(got, oracle.bconv(x, pin, pout))


def test_bconv_table_cache(c1):
    """fhe_bconv keeps the tables of each (inputs, outputs, kernel) combination in the context:
    repeated and interleaved combinations, both kernels, and more combinations than the context
    keeps (it waits and releases them) all stay bit-exact, queued back to back without a sync."""
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = c1
    g = inputs.rng(15)
    nP = len(P.primes)
    import itertools
    combos = []
    for n_in in (1, 2, 3):
        for ins in itertools.permutations(range(nP), n_in):
            if n_in == 3 and list(ins) != sorted(ins):
                continue
            combos.append((list(ins), [i for i in range(nP) if i not in ins]))
    # 56 index combinations, each with the CUDA-core kernel and every other one with the
    # tensor-core kernel too: 84 table sets, more than the 64 a context keeps; then the first
    # ones again
    runs = [(c, binding.FHE_BCONV_SCALAR) for c in combos] + [(c, binding.FHE_BCONV_TC) for c in combos[::2]]
    runs += runs[:5]
    pending = []
    for (in_idx, out_idx), mode in runs:
        ctx.set_bconv(mode)
        x = inputs.uniform_residues(g, [P.primes[i] for i in in_idx], P.N)
        pending.append((x, in_idx, out_idx, ctx.bconv(dev(x), in_idx, out_idx)))
    ctx.set_bconv(binding.FHE_BCONV_SCALAR)
    for x, in_idx, out_idx, out in pending:
        want = oracle.bconv(x, [P.primes[i] for i in in_idx], [P.primes[i] for i in out_idx])
        assert np.array_equal(host(out), want), (in_idx, out_idx)


# ------------------------------------------------------------------ stages

@pytest.mark.parametrize("cfg,level", [("c1", 4), ("c1", 3), ("c1", 1), ("c2", 24), ("c2", 17), ("c2", 9)])
@pytest.mark.parametrize("fused", [True, False])
def test_modup_parity(cfg, level, fused, request):
    P, OP, ctx = request.getfixturevalue(cfg)
    ctx.set_fused(fused)
    g = inputs.rng(20 + level)
    d = inputs.uniform_residues(g, P.q[:level], P.N)
    ext = host(ctx.modup(dev(d), level))
    ctx.set_fused(True)
    for j in range(OP.beta(level)):
        assert np.array_equal(ext[j], oracle.modup(OP, d, level, j)), f"digit {j}"


@pytest.mark.parametrize("cfg,level", [("c1", 4), ("c1", 1), ("c2", 24), ("c2", 5)])
def test_moddown_parity(cfg, level, request):
    P, OP, ctx = request.getfixturevalue(cfg)
    g = inputs.rng(30 + level)
    u = inputs.uniform_residues(g, OP.ext_primes(level), P.N)
    got = host(ctx.moddown(dev(u), level))
    assert np.array_equal(got, oracle.moddown(OP, u, level))


# ------------------------------------------------------------------ key switching and CKKS ops

@pytest.mark.parametrize("cfg,level", [("c1", 4), ("c1", 3), ("c1", 2), ("c1", 1), ("c2", 24), ("c2", 13), ("c2", 1)])
@pytest.mark.parametrize("fused", [True, False])
def test_keyswitch_parity(cfg, level, fused, request):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = request.getfixturevalue(cfg)
    ctx.set_fused(fused)
    g = inputs.rng(40 + level)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    d = inputs.uniform_residues(g, P.q[:level], P.N)
    got = host(ctx.keyswitch(dev(d), level, binding.FHE_RELIN_KEY))
    ctx.set_fused(True)
    assert np.array_equal(got, oracle.keyswitch(OP, d, level, key))


@pytest.mark.parametrize("cfg,level,rot", [("c1", 4, 1), ("c1", 3, -5), ("c1", 4, 1999), ("c2", 24, 12345),
                                           ("c2", 11, 7), ("c2", 24, -1)])
@pytest.mark.parametrize("fused", [True, False])
def test_rotate_parity(cfg, level, rot, fused, request):
    P, OP, ctx = request.getfixturevalue(cfg)
    ctx.set_fused(fused)
    g = inputs.rng(50 + level)
    key = rand_key(P, g)
    ctx.set_rot_key(rot, dev(key))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    got = host(ctx.rotate(dev(ct), level, rot))
    ctx.set_fused(True)
    assert np.array_equal(got, oracle.rotate(OP, ct, level, rot, key))


def test_rotate_identity(c1):
    P, OP, ctx = c1
    g = inputs.rng(55)
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    for rot in (0, P.N // 2, -P.N // 2):
        assert np.array_equal(host(ctx.rotate(dev(ct), P.L, rot)), ct)


@pytest.mark.parametrize("cfg,level", [("c1", 4), ("c1", 2), ("c2", 24)])
@pytest.mark.parametrize("fused", [True, False])
def test_hmult_rescale_parity(cfg, level, fused, request):
    P, OP, ctx = request.getfixturevalue(cfg)
    ctx.set_fused(fused)
    g = inputs.rng(60 + level)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    a = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    b = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    m = ctx.hmult(dev(a), dev(b), level)
    want = oracle.hmult(OP, a, b, level, key)
    assert np.array_equal(host(m), want)
    r = ctx.rescale(m, level)
    assert np.array_equal(host(r), oracle.rescale(OP, want, level))
    ctx.set_fused(True)


@pytest.mark.parametrize("cfg,level", [("c1", 4), ("c2", 24)])
def test_rotate_hoisted_parity(cfg, level, request):
    P, OP, ctx = request.getfixturevalue(cfg)
    g = inputs.rng(70)
    rots = [0, 1, 2, 5, 15]
    keys = [None] + [rand_key(P, g) for _ in rots[1:]]
    for r, k in zip(rots[1:], keys[1:]):
        ctx.set_rot_key(r, dev(k))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    outs = ctx.rotate_hoisted(dev(ct), level, rots)
    want = oracle.rotate_hoisted(OP, ct, level, rots, keys)
    for i in range(len(rots)):
        assert np.array_equal(host(outs[i]), want[i]), f"rotation {rots[i]}"


def test_pmult_add_parity(c2):
    P, OP, ctx = c2
    g = inputs.rng(80)
    level = 24
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    ct2 = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    pt = inputs.uniform_residues(g, P.q[:level], P.N)
    got = host(ctx.pmult(dev(ct), dev(pt), level))
    assert np.array_equal(got, np.stack([oracle.mul(ct[c], pt, P.q) for c in range(2)]))
    got = host(ctx.add(dev(ct), dev(ct2), level))
    assert np.array_equal(got, np.stack([oracle.add(ct[c], ct2[c], P.q) for c in range(2)]))


def test_batch_plan_equals_single_ops(c1):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = c1
    g = inputs.rng(90)
    rk = rand_key(P, g)
    ctx.set_relin_key(dev(rk))
    items, want = [], []
    for i, it in enumerate(inputs.batch_items(g, 12, 1, P.L)):
        lv, rot = it["level"], it["rot"] % (P.N // 2)
        a = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
        if it["op"] == "rotate" and rot:
            k = rand_key(P, g)
            ctx.set_rot_key(rot, dev(k))
            items.append(dict(op=binding.FHE_OP_ROTATE, level=lv, rot=rot, **{"in": dev(a)}, out=binding.empty((2, lv, P.N))))
            want.append(oracle.rotate(OP, a, lv, rot, k))
        else:
            b = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
            items.append(dict(op=binding.FHE_OP_RELIN, level=lv, **{"in": dev(a)}, in2=dev(b), out=binding.empty((2, lv, P.N))))
            want.append(oracle.hmult(OP, a, b, lv, rk))
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    assert plan.kernel_count > 0
    for _ in range(2):
        plan.launch()
        for it, w in zip(items, want):
            assert np.array_equal(host(it["out"]), w)
    plan.close()


@pytest.mark.parametrize("budget,max_group,lanes,pipe", [(0, 0, 1, 1), (1, 2, 2, 1), (0, 3, 2, 0), (0, 1, 3, 0),
                                                        (0, 0, 2, 0)])
def test_batch_plan_full_size_groups(c2, budget, max_group, lanes, pipe):
    """Mixed rotations / relinearisations / key switches at uneven levels,
    N = 2^16, split into groups of various sizes, on several lanes, with and
    without complementary pipelining: every item bit-exact."""
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = c2
    ctx.set_batch(budget, max_group, lanes)
    ctx.set_pipelining(bool(pipe))
    g = inputs.rng(95 + max_group)
    rk = rand_key(P, g)
    ctx.set_relin_key(dev(rk))
    specs = [("rotate", 24, 777), ("relin", 17, 0), ("rotate", 5, 12345), ("ks", 9, 0), ("rotate", 24, 3),
             ("relin", 1, 0)]
    items, want = [], []
    for op, lv, rot in specs:
        a = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
        out = binding.empty((2, lv, P.N))
        if op == "rotate":
            k = rand_key(P, g)
            ctx.set_rot_key(rot, dev(k))
            items.append(dict(op=binding.FHE_OP_ROTATE, level=lv, rot=rot, **{"in": dev(a)}, out=out))
            want.append(oracle.rotate(OP, a, lv, rot, k))
        elif op == "relin":
            b = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
            items.append(dict(op=binding.FHE_OP_RELIN, level=lv, **{"in": dev(a)}, in2=dev(b), out=out))
            want.append(oracle.hmult(OP, a, b, lv, rk))
        else:
            items.append(dict(op=binding.FHE_OP_KS, level=lv, rot=binding.FHE_RELIN_KEY, **{"in": dev(a[0])}, out=out))
            want.append(oracle.keyswitch(OP, a[0], lv, rk))
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    if max_group:
        assert max(plan.groups) <= max_group
    plan.launch()
    for i, (it, w) in enumerate(zip(items, want)):
        assert np.array_equal(host(it["out"]), w), f"item {i} {specs[i]}"
    plan.close()
    ctx.set_batch(0, 0, 0)
    ctx.set_pipelining(True)


# ------------------------------------------------------------------ CKKS semantics through the GPU path

def test_gpu_rotate_decodes(c1):
    P, OP, ctx = c1
    g = inputs.rng(100)
    sk = oracle.SecretKey(OP, inputs.ternary(g, P.N))
    z = inputs.complex_slots(g, P.N // 2)
    ct = oracle.encrypt(OP, sk, oracle.encode(z, 2.0 ** 25, P.N), P.L, g)
    rot = 77
    key = oracle.rotation_key(OP, sk, rot, g)
    ctx.set_rot_key(rot, dev(key))
    out = host(ctx.rotate(dev(ct), P.L, rot))
    dec = oracle.decode(oracle.decrypt(OP, sk, out, P.L), 2.0 ** 25, P.N)
    # the slot-error model of key switching (oracle/noise.py): prediction within its bound
    from oracle import noise
    err, pred, ratio = noise.check_rotation(OP, sk, ct, P.L, rot, key, dec, np.roll(z, -rot), 2.0 ** 25)
    assert ratio <= 1.0, (err, pred, ratio)


# ------------------------------------------------------------------ host-side validation with a live context

def test_error_statuses(c1):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = c1
    d = binding.empty((2, P.L, P.N))
    with pytest.raises(binding.FheError) as e:
        ctx.keyswitch(d[0], P.L + 1)
    assert e.value.code == binding.FHE_ELEVEL
    with pytest.raises(binding.FheError) as e:
        ctx.rotate(d, P.L, 3, out=d)
    assert e.value.code in (binding.FHE_EALIAS, binding.FHE_ENOKEY)
    with pytest.raises(binding.FheError) as e:
        ctx.rotate(d, P.L, 1234, out=binding.empty((2, P.L, P.N)))
    assert e.value.code == binding.FHE_ENOKEY
    with pytest.raises(binding.FheError) as e:
        ctx.rescale(d, 1)
    assert e.value.code == binding.FHE_ELEVEL
