"""Double-hoisted bootstrapping linear transforms (CoeffToSlot / SlotToCoeff
radix levels) on the GPU: bit-exact against the oracle's double-hoisted
evaluation, level by level and as rescaled chains, at the small ring and at
the paper's bootstrapping shape (N = 2^16, L = 48, alpha = K = 12, dnum = 4)."""
import numpy as np
import pytest

import oracle
from oracle import bootstrap_lt as blt
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


def uniform_level(P, plan, level, g):
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    xp = tuple(P.q[:level]) + tuple(P.p)
    diags = np.stack([inputs.uniform_residues(g, xp, P.N) for _ in range(plan.n_diag)])
    return ct, diags


@pytest.mark.parametrize("kind,which", [("cts", 0), ("cts", 1), ("cts", 2), ("stc", 0)])
@pytest.mark.parametrize("fused", [1, 0])
def test_level_parity_small_ring(fhe_lib, kind, which, fused):
    from paper_2512_18345_gb300 import binding
    name = "cts_stc_N4096_L8"
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    W = inputs.WORKLOADS[name]
    plan = inputs.transform_plans(P.N, W["levels"], kind)[which]
    level = W["cts_level"] - which
    g = inputs.rng(1000 + 10 * which + fused + (5 if kind == "stc" else 0))
    ctx = binding.Context.from_params(P)
    ctx.set_fused(fused)
    keys = {}
    for r in plan.rotations():
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    ct, diags = uniform_level(P, plan, level, g)
    got = host(ctx, ctx.linear_transform_dh(dev(ct), level, plan.baby, plan.giant, dev(diags), plan.idx))
    want = blt.lt_double_hoisted(OP, ct, level, plan.baby, plan.giant, diags, plan.idx, keys)
    assert np.array_equal(got, want)
    ctx.close()


def test_identity_only_transform_is_a_plaintext_product(fhe_lib):
    """baby = giant = [0] with one diagonal: ModDown(pt (.) P ct) = pt (.) ct exactly (the lifted
    ciphertext has zero special limbs)."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("cts_stc_N4096_L8")
    g = inputs.rng(1100)
    ctx = binding.Context.from_params(P)
    level = 6
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    pt = inputs.uniform_residues(g, tuple(P.q[:level]) + tuple(P.p), P.N)[None]
    got = host(ctx, ctx.linear_transform_dh(dev(ct), level, [0], [0], dev(pt), [[0]]))
    want = np.stack([oracle.mul(ct[c], pt[0][:level], P.q) for c in range(2)])
    assert np.array_equal(got, want)
    ctx.close()


def test_chain_small_ring_bit_exact_and_decodes(fhe_lib):
    """CoeffToSlot then SlotToCoeff (3 + 3 levels, each followed by a rescale) on real
    encryptions: every level's output equals the oracle's, and the result decodes to the
    message (round-trip error amplified by at most sqrt(n))."""
    from paper_2512_18345_gb300 import binding
    name = "cts_stc_N4096_L8"
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    W = inputs.WORKLOADS[name]
    g = inputs.rng(1200)
    sk = oracle.SecretKey(OP, inputs.ternary(g, P.N))
    n = P.N // 2
    scale = 2.0 ** W["scale_bits"]
    z = inputs.complex_slots(g, n)
    level = W["cts_level"]
    ct = oracle.encrypt(OP, sk, oracle.encode(z, scale, P.N), level, g)
    ctx = binding.Context.from_params(P)
    ctx.set_bconv(binding.FHE_BCONV_TC)
    log_slots = n.bit_length() - 1
    keys = {}
    d_ct, o_ct = dev(ct), ct
    for kind in ("cts", "stc"):
        plans = inputs.transform_plans(P.N, W["levels"], kind)
        lv = inputs.radix_levels(log_slots, W["levels"])
        if kind == "cts":
            lv = lv[::-1]
        for plan, (lo, hi) in zip(plans, lv):
            for r in plan.rotations():
                if r not in keys:
                    keys[r] = oracle.rotation_key(OP, sk, r, g)
                    ctx.set_rot_key(r, dev(keys[r]))
            D = blt.level_diagonals(P.N, lo, hi, inverse=(kind == "cts"))
            pts = blt.level_plaintexts(OP, D, plan, level, float(P.q[level - 1]))
            d_out = ctx.linear_transform_dh(d_ct, level, plan.baby, plan.giant, dev(pts), plan.idx)
            d_ct = ctx.rescale(d_out, level)
            o_ct = oracle.rescale(OP, blt.lt_double_hoisted(OP, o_ct, level, plan.baby, plan.giant, pts, plan.idx,
                                                            keys), level)
            level -= 1
            assert np.array_equal(host(ctx, d_ct), o_ct), (kind, lo, hi)
    back = oracle.decode(oracle.decrypt(OP, sk, host(ctx, d_ct), level), scale, P.N)
    assert np.abs(back - z).max() < 2.0 ** -5 * np.sqrt(n)
    ctx.close()


@pytest.mark.parametrize("kind,which,level_key,tc", [("cts", 0, "cts_level", False), ("stc", 1, "stc_level", False),
                                                     ("cts", 1, "cts_level", True)])
def test_level_parity_bootstrapping_shape(fhe_lib, kind, which, level_key, tc):
    """N = 2^16, L = 48, K = 12, dnum = 4: the first CoeffToSlot level at l = 48 (32 diagonals,
    15 rotating baby steps and one rotating giant step), the middle SlotToCoeff level at
    l = 33 (63 diagonals, 15 + 3) with the CUDA-core BConv, and the second CoeffToSlot level
    with the tensor-core BConv (its K = 64 shape for the 12-limb digits)."""
    from paper_2512_18345_gb300 import binding
    name = "cts_stc_N65536_L48_a12"
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    W = inputs.WORKLOADS[name]
    plan = inputs.transform_plans(P.N, W["levels"], kind)[which]
    level = W[level_key] - (which if kind == "cts" else 0)
    g = inputs.rng(1300 + which + (50 if tc else 0))
    ctx = binding.Context.from_params(P)
    ctx.set_bconv(binding.FHE_BCONV_TC if tc else binding.FHE_BCONV_SCALAR)
    keys = {}
    for r in plan.rotations():
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    ct, diags = uniform_level(P, plan, level, g)
    got = host(ctx, ctx.linear_transform_dh(dev(ct), level, plan.baby, plan.giant, dev(diags), plan.idx))
    want = blt.lt_double_hoisted(OP, ct, level, plan.baby, plan.giant, diags, plan.idx, keys)
    assert np.array_equal(got, want)
    ctx.close()


def test_diagonal_pass_sparse_pairs(fhe_lib):
    """The diagonal pass's per-group bookkeeping: 32 baby steps (the top bit of the baby-step
    masks), five giant steps (a second group holding one), a giant step without any diagonal,
    baby steps that meet no diagonal in the first group but do in the second, one baby step
    that meets none at all, and diagonals shared by several pairs."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("cts_stc_N4096_L8")
    OP = oracle.OracleParams.from_params(P)
    g = inputs.rng(1470)
    level = 5
    baby = list(range(32))
    giant = [0, 32, 64, 96, 128]
    n_diag = 40
    live = g.random((len(giant), len(baby))) < 0.4
    live[1, :] = False          # giant step 1: no diagonal
    live[:4, [5, 17]] = False   # first group: baby steps 5 and 17 unused ...
    live[4, [5, 17, 31]] = True  # ... the second group uses them and the top mask bit
    live[2, 31] = True
    live[:, 9] = False          # baby step 9: no diagonal anywhere
    idx = np.where(live, g.integers(0, n_diag, size=live.shape), -1).tolist()
    ctx = binding.Context.from_params(P)
    keys = {}
    for r in sorted(set(baby[1:]) | set(giant[1:])):
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    xp = tuple(P.q[:level]) + tuple(P.p)
    diags = np.stack([inputs.uniform_residues(g, xp, P.N) for _ in range(n_diag)])
    got = host(ctx, ctx.linear_transform_dh(dev(ct), level, baby, giant, dev(diags), idx))
    assert np.array_equal(got, blt.lt_double_hoisted(OP, ct, level, baby, giant, diags, idx, keys))
    ctx.close()


def test_rejections(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("cts_stc_N4096_L8")
    g = inputs.rng(1400)
    ctx = binding.Context.from_params(P)
    level = 4
    ct = dev(np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)]))
    pt = dev(inputs.uniform_residues(g, tuple(P.q[:level]) + tuple(P.p), P.N)[None])

    def code(fn):
        with pytest.raises(binding.FheError) as e:
            fn()
        return e.value.code

    assert code(lambda: ctx.linear_transform_dh(ct, level, [0, 1], [0], pt, [[0, 0]])) == binding.FHE_ENOKEY
    assert code(lambda: ctx.linear_transform_dh(ct, level, [0], [3], pt, [[0]])) == binding.FHE_ENOKEY
    assert code(lambda: ctx.linear_transform_dh(ct, level, [0], [0], pt, [[1]])) == binding.FHE_EINVAL
    assert code(lambda: ctx.linear_transform_dh(ct, level, [0], [0], pt, [[-2]])) == binding.FHE_EINVAL
    assert code(lambda: ctx.linear_transform_dh(ct, 0, [0], [0], pt, [[0]])) == binding.FHE_ELEVEL
    assert code(lambda: ctx.linear_transform_dh(ct, level, [0] * 33, [0], pt, [[0] * 33])) == binding.FHE_EINVAL
    assert code(lambda: ctx.linear_transform_dh(ct, level, [0], [0], pt, [[0]], out=ct)) == binding.FHE_EALIAS
    ctx.close()


@pytest.mark.parametrize("level", [1, 2, 3])
def test_low_levels(fhe_lib, level):
    """One digit or a partial last digit (alpha = 2 on this ring): the extended basis is a few
    q-limbs plus the special limbs."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("cts_stc_N4096_L8")
    OP = oracle.OracleParams.from_params(P)
    plan = inputs.bsgs_plan(P.N // 2, 3, 4)
    g = inputs.rng(1450 + level)
    ctx = binding.Context.from_params(P)
    keys = {}
    for r in plan.rotations():
        keys[r] = rand_key(P, g)
        ctx.set_rot_key(r, dev(keys[r]))
    ct, diags = uniform_level(P, plan, level, g)
    got = host(ctx, ctx.linear_transform_dh(dev(ct), level, plan.baby, plan.giant, dev(diags), plan.idx))
    assert np.array_equal(got, blt.lt_double_hoisted(OP, ct, level, plan.baby, plan.giant, diags, plan.idx, keys))
    ctx.close()
