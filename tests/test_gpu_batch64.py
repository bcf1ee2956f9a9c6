"""The fourth workload: 64 ciphertexts at N = 2^16, levels uniform in 4..24, a
mix of relinearisations and rotations, in one graph-captured batched plan.
Every item must be bit-identical to the same operation run alone (whose parity
with the oracle is pinned elsewhere), and a sample of items is checked against
the oracle directly."""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_batch64_mixed_levels(fhe_lib):
    import torch
    from paper_2512_18345_gb300 import binding
    name = "batch64_N65536_L4to24"
    w = inputs.WORKLOADS[name]
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    g = inputs.rng(w["seed"])
    spec = inputs.batch_items(g, w["items"], w["level_lo"], w["level_hi"])
    keys = {}

    def key():
        return np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)])
                         for _ in range(P.dnum)])
    rk = key()
    ctx.set_relin_key(binding.to_device(rk))
    items, host_in = [], []
    for it in spec:
        lv = it["level"]
        a = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
        out = binding.empty((2, lv, P.N))
        if it["op"] == "rotate":
            r = it["rot"]
            if r not in keys:
                keys[r] = key()
                ctx.set_rot_key(r, binding.to_device(keys[r]))
            items.append(dict(op=binding.FHE_OP_ROTATE, level=lv, rot=r, **{"in": binding.to_device(a)}, out=out))
            host_in.append((a, None))
        else:
            b = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
            items.append(dict(op=binding.FHE_OP_RELIN, level=lv, **{"in": binding.to_device(a)},
                              in2=binding.to_device(b), out=out))
            host_in.append((a, b))
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    assert sum(plan.groups) == 64 and plan.kernel_count > 0
    plan.launch()
    plan.launch()  # a replay must give the same result
    ctx.sync()
    got = [binding.to_numpy(it["out"]) for it in items]
    # every item equals the same operation run alone
    for it, gt in zip(items, got):
        if it["op"] == binding.FHE_OP_ROTATE:
            single = ctx.rotate(it["in"], it["level"], it["rot"])
        else:
            single = ctx.hmult(it["in"], it["in2"], it["level"])
        torch.cuda.synchronize()
        assert np.array_equal(binding.to_numpy(single), gt)
    # a sample against the oracle
    for idx in (0, 17, 40, 63):
        a, b = host_in[idx]
        lv = spec[idx]["level"]
        want = oracle.rotate(OP, a, lv, spec[idx]["rot"], keys[spec[idx]["rot"]]) if b is None \
            else oracle.hmult(OP, a, b, lv, rk)
        assert np.array_equal(got[idx], want), idx
    plan.close()
    ctx.close()


def test_headline_configuration_full_size(fhe_lib):
    """The benchmark's step as it is timed: 8 rotations at N = 2^16, L = 24 with
    distinct keys, tensor-core BConv, the autotuned schedule, one CUDA graph,
    replayed twice; every output equals the oracle's."""
    from paper_2512_18345_gb300 import binding
    name = "hrotate_N65536_L24_tc"
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    ctx.set_bconv(binding.FHE_BCONV_TC)
    g = inputs.rng(inputs.WORKLOADS[name]["seed"] + 77)
    items, want, used = [], [], set()
    while len(items) < 8:
        r = inputs.rotation_index(g)
        k = pow(5, r % (P.N // 2), 2 * P.N)
        if k in used:
            continue
        used.add(k)
        key = np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)])
                        for _ in range(P.dnum)])
        ctx.set_rot_key(r, binding.to_device(key))
        ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
        items.append(dict(op=binding.FHE_OP_ROTATE, level=P.L, rot=r, **{"in": binding.to_device(ct)},
                          out=binding.empty((2, P.L, P.N))))
        want.append(oracle.rotate(OP, ct, P.L, r, key))
    tune = ctx.autotune(P.L, len(items))
    assert tune["bconv_mode"] == binding.FHE_BCONV_TC
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    plan.launch()
    plan.launch()
    ctx.sync()
    for it, w in zip(items, want):
        assert np.array_equal(binding.to_numpy(it["out"]), w)
    plan.close()
    ctx.close()
