"""Schedule autotuner for batched plans: it measures candidate schedules on the
device, applies the fastest, and plans built under the chosen schedule stay
bit-exact against the oracle (a schedule changes timing, never results)."""
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


def test_autotune_small_ring_then_bit_exact(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    r = ctx.autotune(P.L, 6, binding.FHE_TUNE_BCONV)
    assert 1 <= r["lanes"] <= 4 and r["candidates"] >= 2 and r["us_per_ks"] > 0
    assert r["bconv_mode"] in (binding.FHE_BCONV_SCALAR, binding.FHE_BCONV_TC)
    assert ctx.info()["bconv_mode"] == r["bconv_mode"]
    # the filler key of the tuning run is gone again
    with pytest.raises(binding.FheError) as err:
        ctx.keyswitch(dev(np.zeros((P.L, P.N), np.uint32)), P.L)
    assert err.value.code == binding.FHE_ENOKEY
    g = inputs.rng(700)
    items, want = [], []
    for lv, rot in [(4, 3), (3, 100), (4, 77), (2, 5), (4, 1000), (3, 9)]:
        k = rand_key(P, g)
        ctx.set_rot_key(rot, dev(k))
        a = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
        items.append(dict(op=binding.FHE_OP_ROTATE, level=lv, rot=rot, **{"in": dev(a)},
                          out=binding.empty((2, lv, P.N))))
        want.append(oracle.rotate(OP, a, lv, rot, k))
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    plan.launch()
    for it, w in zip(items, want):
        assert np.array_equal(host(ctx, it["out"]), w)
    plan.close()
    ctx.close()


def test_autotune_full_size_keeps_the_relin_key(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hrotate_N65536_L24_tc")
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    g = inputs.rng(710)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    ctx.set_bconv(binding.FHE_BCONV_TC)
    r = ctx.autotune(P.L, 4)
    assert r["bconv_mode"] == binding.FHE_BCONV_TC  # without FHE_TUNE_BCONV the kernel stays
    assert r["default_us_per_ks"] > 0 and r["us_per_ks"] <= r["default_us_per_ks"]
    d = inputs.uniform_residues(g, P.q, P.N)
    got = host(ctx, ctx.keyswitch(dev(d), P.L))
    assert np.array_equal(got, oracle.keyswitch(OP, d, P.L, key))
    ctx.close()


@pytest.mark.parametrize("level,n_items,flags,code", [(0, 4, 0, "FHE_ELEVEL"), (5, 4, 0, "FHE_ELEVEL"),
                                                      (4, 0, 0, "FHE_EINVAL"), (4, 65, 0, "FHE_EINVAL"),
                                                      (4, 4, 8, "FHE_EINVAL")])
def test_autotune_rejects_bad_arguments(fhe_lib, level, n_items, flags, code):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    ctx = binding.Context.from_params(P)
    with pytest.raises(binding.FheError) as err:
        ctx.autotune(level, n_items, flags)
    assert err.value.code == getattr(binding, code)
    ctx.close()


def test_autotune_cache_records_then_serves(fhe_lib, tmp_path):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    path = tmp_path / "tune.txt"
    ctx = binding.Context.from_params(P)
    r1 = ctx.autotune(P.L, 4, cache=str(path))
    assert r1["candidates"] >= 2
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and "items=4" in lines[0] and f"N={P.N}" in lines[0]
    ctx.close()
    ctx2 = binding.Context.from_params(P)
    r2 = ctx2.autotune(P.L, 4, cache=str(path))
    assert r2["candidates"] == 0  # served from the file, nothing measured
    for k in ("lanes", "l2_budget_bytes", "bconv_mode", "ip_ctas_per_sm"):
        assert r2[k] == r1[k]
    with open(path, "a") as f:  # a malformed line and another key leave the lookup alone
        f.write("not an entry\n")
        f.write(lines[0].replace("items=4", "items=5") + "\n")
    assert ctx2.autotune(P.L, 4, cache=str(path))["candidates"] == 0
    r4 = ctx2.autotune(P.L, 3, cache=str(path))  # a new batch size is measured and recorded
    assert r4["candidates"] >= 2 and len(path.read_text().splitlines()) == 4
    ctx2.close()
