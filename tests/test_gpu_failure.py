"""Failure detection without a GPU fault, and writes that stay inside their
buffers.

* A bounded device-side wait that expires (the self-test waits on a barrier
  nothing arrives on) is reported by the next fhe_ctx_sync as FHE_ETIMEOUT,
  the status is cleared, and the context keeps computing bit-exact results.
* Every output buffer sits between canary words; rotations, HMult, rescale,
  batched plans and the base conversion leave the canaries untouched.
* An allocation failure injected on the host (the context's memory limit) is
  reported as FHE_ENOMEM before anything is launched, and the context keeps
  working once the limit is lifted."""
import numpy as np
import pytest

import oracle
from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu

CANARY = 0x5A5A5A5A
PAD = 1024  # words on each side (keeps the output 16-byte aligned)


def dev(a):
    from paper_2512_18345_gb300 import binding
    return binding.to_device(a)


def rand_key(P, g):
    return np.stack([np.stack([inputs.uniform_residues(g, P.primes, P.N) for _ in range(2)]) for _ in range(P.dnum)])


def padded(shape):
    """An output tensor of `shape` inside a canary-filled allocation."""
    import torch
    n = int(np.prod(shape))
    full = torch.full((n + 2 * PAD,), CANARY, dtype=torch.int32, device="cuda")
    return full, full[PAD:PAD + n].view(*shape)


def canaries_intact(full) -> bool:
    import torch
    torch.cuda.synchronize()
    h = full.cpu().numpy().view(np.uint32)
    return bool((h[:PAD] == CANARY).all() and (h[-PAD:] == CANARY).all())


@pytest.fixture(scope="module")
def small(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    ctx = binding.Context.from_params(P)
    yield P, oracle.OracleParams.from_params(P), ctx
    ctx.close()


def test_bounded_wait_expiry_reports_timeout_then_recovers(small):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = small
    ctx.selftest_wait_timeout()
    with pytest.raises(binding.FheError) as err:
        ctx.sync()
    assert err.value.code == binding.FHE_ETIMEOUT
    ctx.sync()  # the status was cleared
    g = inputs.rng(800)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    d = inputs.uniform_residues(g, P.q, P.N)
    out = ctx.keyswitch(dev(d), P.L)
    ctx.sync()
    assert np.array_equal(binding.to_numpy(out), oracle.keyswitch(OP, d, P.L, key))


@pytest.mark.parametrize("bconv", ["scalar", "tc"])
def test_outputs_stay_within_their_buffers(small, bconv):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = small
    ctx.set_bconv(binding.FHE_BCONV_TC if bconv == "tc" else binding.FHE_BCONV_SCALAR)
    g = inputs.rng(810)
    rk = rand_key(P, g)
    ctx.set_relin_key(dev(rk))
    rot = 7
    kr = rand_key(P, g)
    ctx.set_rot_key(rot, dev(kr))
    a = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    b = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    L, N = P.L, P.N
    f1, o1 = padded((2, L, N))
    ctx.rotate(dev(a), L, rot, out=o1)
    f2, o2 = padded((2, L, N))
    ctx.hmult(dev(a), dev(b), L, out=o2)
    f3, o3 = padded((2, L - 1, N))
    ctx.rescale(dev(a), L, out=o3)
    f4, o4 = padded((2, L, N))
    plan = ctx.batch_plan([dict(op=binding.FHE_OP_ROTATE, level=L, rot=rot, **{"in": dev(a)}, out=o4)],
                          binding.FHE_PLAN_GRAPH)
    plan.launch()
    f5, o5 = padded((3, N))
    ctx.bconv(dev(inputs.uniform_residues(g, P.q[:2], N)), [0, 1], [2, 3, 4], out=o5)
    for f in (f1, f2, f3, f4, f5):
        assert canaries_intact(f)
    ctx.sync()
    assert np.array_equal(binding.to_numpy(o1), oracle.rotate(OP, a, L, rot, kr))
    assert np.array_equal(binding.to_numpy(o4), binding.to_numpy(o1))
    plan.close()
    ctx.set_bconv(binding.FHE_BCONV_SCALAR)


def test_memory_limit_injects_enomem_and_recovers(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    g = inputs.rng(2100)
    key = rand_key(P, g)

    def code(fn):
        with pytest.raises(binding.FheError) as e:
            fn()
        return e.value.code

    ctx.set_memory_limit(1)  # nothing may grow: the key copy is refused
    assert code(lambda: ctx.set_relin_key(dev(key))) == binding.FHE_ENOMEM
    ctx.set_memory_limit(0)
    ctx.set_relin_key(dev(key))
    # no room beyond what is held (the key and the context's first workspace slot): a single
    # key switch runs in that slot, a batch of three items needs two more and is refused
    held = ctx.info()["key_bytes"] + ctx.info()["workspace_bytes"]
    ctx.set_memory_limit(held + 1)
    ds = [inputs.uniform_residues(g, P.q, P.N) for _ in range(3)]
    got = ctx.keyswitch(dev(ds[0]), P.L)
    ctx.sync()
    assert np.array_equal(binding.to_numpy(got), oracle.keyswitch(OP, ds[0], P.L, key))
    items = [dict(op=binding.FHE_OP_KS, level=P.L, rot=binding.FHE_RELIN_KEY, **{"in": dev(d)},
                  out=binding.empty((2, P.L, P.N))) for d in ds]
    assert code(lambda: ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)) == binding.FHE_ENOMEM
    ctx.sync()  # nothing was launched: no device-side failure either
    ctx.set_memory_limit(0)
    plan = ctx.batch_plan(items, binding.FHE_PLAN_GRAPH)
    plan.launch()
    ctx.sync()
    for it, d in zip(items, ds):
        assert np.array_equal(binding.to_numpy(it["out"]), oracle.keyswitch(OP, d, P.L, key))
    plan.close()
    # the linear transforms' scratch counts too
    ctx.set_memory_limit(ctx.info()["key_bytes"] + ctx.info()["workspace_bytes"] + 1)
    ct = dev(np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)]))
    pt = dev(inputs.uniform_residues(g, tuple(P.q) + tuple(P.p), P.N)[None])
    assert code(lambda: ctx.linear_transform_dh(ct, P.L, [0], [0], pt, [[0]])) == binding.FHE_ENOMEM
    ctx.set_memory_limit(0)
    ctx.linear_transform_dh(ct, P.L, [0], [0], pt, [[0]])
    ctx.sync()
    ctx.close()
