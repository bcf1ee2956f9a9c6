"""The paper's own key-switching shapes (Table "ks-param"): (l, alpha, beta) =
(24, 12, 2) and (48, 12, 4) with K = alpha = 12 at N = 2^16, 31-bit primes, with
the CUDA-core conversion and with the tensor-core conversion (its K = 64 shape
for digits of 9..12 limbs); every residue equals the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = ["paper_ks_N65536_L24_a12", "paper_ks_N65536_L48_a12"]


def rand_key(P, g):
    return np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)]) for _ in range(P.dnum)])


@pytest.mark.parametrize("name", SHAPES)
@pytest.mark.parametrize("tc", [False, True])
def test_paper_shape_keyswitch_rotate_and_batch(fhe_lib, name, tc):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    ctx.set_bconv(binding.FHE_BCONV_TC if tc else binding.FHE_BCONV_SCALAR)
    g = inputs.rng(inputs.WORKLOADS[name]["seed"] + (7 if tc else 0))
    key = rand_key(P, g)
    ctx.set_relin_key(binding.to_device(key))
    d = inputs.uniform_residues(g, P.q, P.N)
    got = ctx.keyswitch(binding.to_device(d), P.L)
    ctx.sync()
    assert np.array_equal(binding.to_numpy(got), oracle.keyswitch(OP, d, P.L, key))
    rot = inputs.rotation_index(g)
    rk = rand_key(P, g)
    ctx.set_rot_key(rot, binding.to_device(rk))
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    got = ctx.rotate(binding.to_device(ct), P.L, rot)
    ctx.sync()
    assert np.array_equal(binding.to_numpy(got), oracle.rotate(OP, ct, P.L, rot, rk))
    # a batch at uneven levels (partial last digits) equals the single operations
    items = []
    for lv in (P.L, P.L - 5, 13):
        a = np.stack([inputs.uniform_residues(g, P.q[:lv], P.N) for _ in range(2)])
        items.append(dict(op=binding.FHE_OP_ROTATE, level=lv, rot=rot, **{"in": binding.to_device(a)},
                          out=binding.empty((2, lv, P.N))))
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    plan.launch()
    for it in items:
        single = ctx.rotate(it["in"], it["level"], rot)
        ctx.sync()
        assert np.array_equal(binding.to_numpy(it["out"]), binding.to_numpy(single))
    plan.close()
    ctx.close()


def test_tensor_core_limits(fhe_lib):
    """The tensor-core conversion takes digits and special-prime counts of at most 12 limbs."""
    from paper_2512_18345_gb300 import binding
    P = inputs.make_params(1 << 12, 13, 13, 1, bits=30)  # alpha = K = 13
    ctx = binding.Context.from_params(P)
    with pytest.raises(binding.FheError) as err:
        ctx.set_bconv(binding.FHE_BCONV_TC)
    assert err.value.code == binding.FHE_EUNSUPPORTED
    ctx.close()
