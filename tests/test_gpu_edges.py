"""Edge cases of the boundary and the method: every level of a ring (partial
digits included) on both BConv kernels, keys of maximal residues, extreme and
negative rotation indices,
rescale down to one limb, and the host-side rejection of misaligned, aliased
or empty requests (no kernel runs for those)."""
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
def small(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    ctx = binding.Context.from_params(P)
    yield P, oracle.OracleParams.from_params(P), ctx
    ctx.close()


@pytest.mark.parametrize("bconv", ["scalar", "tc"])
def test_keyswitch_every_level(small, bconv):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = small
    ctx.set_bconv(binding.FHE_BCONV_TC if bconv == "tc" else binding.FHE_BCONV_SCALAR)
    g = inputs.rng(900)
    key = rand_key(P, g)
    ctx.set_relin_key(dev(key))
    for level in range(1, P.L + 1):  # alpha = 2: levels 1 and 3 end in a partial digit
        d = inputs.uniform_residues(g, P.q[:level], P.N)
        assert np.array_equal(host(ctx, ctx.keyswitch(dev(d), level)), oracle.keyswitch(OP, d, level, key)), level
    ctx.set_bconv(binding.FHE_BCONV_SCALAR)


@pytest.mark.parametrize("name", ["hmult_relin_rescale_N4096_L4", "hrotate_N65536_L24_tc", "paper_ks_N65536_L48_a12"])
@pytest.mark.parametrize("fill", ["max", "uniform"])
def test_maximal_keys(fhe_lib, name, fill):
    """Every key residue q - 1, so each inner-product product is as large as the ModUp value
    it meets allows (up to four digits' products before a reduction at L = 48); with
    fill = "max" the rotated ciphertext is q - 1 everywhere as well (the pass-through term
    P sigma(c0) then at its largest).  Key switch, rotation and hoisted rotations, against
    the oracle."""
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    ctx = binding.Context.from_params(P)
    g = inputs.rng(930 + len(name) + (1 if fill == "max" else 0))
    key = np.stack([np.stack([np.array([[p - 1] * P.N for p in P.primes], np.uint32)] * 2)] * P.dnum)
    level = P.L

    def poly():
        if fill == "max":
            return np.array([[q - 1] * P.N for q in P.q[:level]], np.uint32)
        return inputs.uniform_residues(g, P.q[:level], P.N)

    ctx.set_relin_key(dev(key))
    d = poly()
    assert np.array_equal(host(ctx, ctx.keyswitch(dev(d), level)), oracle.keyswitch(OP, d, level, key))
    rot = 3
    ctx.set_rot_key(rot, dev(key))
    ct = np.stack([poly(), poly()])
    assert np.array_equal(host(ctx, ctx.rotate(dev(ct), level, rot)), oracle.rotate(OP, ct, level, rot, key))
    ctx.set_rot_key(5, dev(key))
    outs = ctx.rotate_hoisted(dev(ct), level, [rot, 5])
    for o, w in zip(outs, oracle.rotate_hoisted(OP, ct, level, [rot, 5], [key, key])):
        assert np.array_equal(host(ctx, o), w)
    ctx.close()


@pytest.mark.parametrize("rot", [1, -1, -5, 2047, 2049, 4095])
def test_rotation_indices(small, rot):
    P, OP, ctx = small
    g = inputs.rng(910 + rot % 97)
    key = rand_key(P, g)
    ctx.set_rot_key(rot, dev(key))
    ct = np.stack([inputs.uniform_residues(g, P.q, P.N) for _ in range(2)])
    assert np.array_equal(host(ctx, ctx.rotate(dev(ct), P.L, rot)), oracle.rotate(OP, ct, P.L, rot, key))


@pytest.mark.parametrize("level", [2, 3, 4])
def test_rescale_to_every_level(small, level):
    P, OP, ctx = small
    g = inputs.rng(920 + level)
    ct = np.stack([inputs.uniform_residues(g, P.q[:level], P.N) for _ in range(2)])
    assert np.array_equal(host(ctx, ctx.rescale(dev(ct), level)), oracle.rescale(OP, ct, level))


def test_misaligned_aliased_and_empty_requests_are_rejected(small):
    from paper_2512_18345_gb300 import binding
    P, OP, ctx = small
    L, N = P.L, P.N
    g = inputs.rng(930)
    ctx.set_relin_key(dev(rand_key(P, g)))
    ctx.set_rot_key(3, dev(rand_key(P, g)))
    good = binding.empty((2, L, N))
    raw = binding.empty((2 * L * N + 4,))
    bad = raw[1:1 + 2 * L * N].view(2, L, N)  # 4 bytes past a 16-byte boundary

    def code(fn):
        with pytest.raises(binding.FheError) as err:
            fn()
        return err.value.code

    assert code(lambda: ctx.keyswitch(bad[0], L)) == binding.FHE_EINVAL
    assert code(lambda: ctx.rotate(bad, L, 3)) == binding.FHE_EINVAL
    assert code(lambda: ctx.rotate(good, L, 3, out=bad)) == binding.FHE_EINVAL
    assert code(lambda: ctx.hmult(good, bad, L)) == binding.FHE_EINVAL
    assert code(lambda: ctx.rescale(bad, L)) == binding.FHE_EINVAL
    assert code(lambda: ctx.bconv(bad[0, :2], [0, 1], [2])) == binding.FHE_EINVAL
    item = dict(op=binding.FHE_OP_ROTATE, level=L, rot=3)
    assert code(lambda: ctx.batch_plan([dict(item, **{"in": bad}, out=binding.empty((2, L, N)))])) == binding.FHE_EINVAL
    assert code(lambda: ctx.batch_plan([dict(item, **{"in": good}, out=bad)])) == binding.FHE_EINVAL
    relin = dict(op=binding.FHE_OP_RELIN, level=L, **{"in": good}, in2=bad, out=binding.empty((2, L, N)))
    assert code(lambda: ctx.batch_plan([relin])) == binding.FHE_EINVAL
    assert code(lambda: ctx.batch_plan([dict(item, **{"in": good}, out=good)])) == binding.FHE_EALIAS
    assert code(lambda: ctx.batch_plan([])) == binding.FHE_EINVAL
    ctx.sync()  # nothing was launched; the context is intact
