"""Pins of the oracle's bootstrapping linear transforms (CoeffToSlot /
SlotToCoeff as radix levels of butterfly stages, evaluated with double
hoisting): the stage products against the DFT matrix written from its
definition, the diagonal form against dense matrix products, the
baby-step / giant-step split against the level's offsets, and the homomorphic
evaluation against the FP64 matrix-vector product after decryption."""
import numpy as np
import pytest

import oracle
from oracle import bootstrap_lt as blt
from paper_2512_18345_gb300 import inputs


def dense(D, n):
    """Dense matrix of a diagonal form: M[r][(r + k) mod n] = D_k[r]."""
    M = np.zeros((n, n), dtype=np.complex128)
    r = np.arange(n)
    for k, d in D.items():
        M[r, (r + k) % n] += d
    return M


@pytest.mark.parametrize("N", [16, 64, 256])
def test_slot_to_coeff_stages_equal_the_dft_definition(N):
    n = N // 2
    g = inputs.rng(900 + N)
    v = inputs.complex_slots(g, n)
    out = v.copy()
    for s in range(1, n.bit_length()):
        out = blt.apply_diagonals(blt.stage_diagonals(N, s), out)
    want = blt.dft_matrix(N) @ v[blt.bitrev_perm(n)]
    assert np.abs(out - want).max() < 1e-9 * n


@pytest.mark.parametrize("N", [16, 64, 256])
def test_coeff_to_slot_stages_invert_the_dft(N):
    n = N // 2
    g = inputs.rng(910 + N)
    z = inputs.complex_slots(g, n)
    out = z.copy()
    for s in range(n.bit_length() - 1, 0, -1):
        out = blt.apply_diagonals(blt.stage_diagonals(N, s, inverse=True), out)
    # bitrev(U^-1 z): U applied to its bit-reversal gives z back
    assert np.abs(blt.dft_matrix(N) @ out[blt.bitrev_perm(n)] - z).max() < 1e-9 * n


def test_slot_to_coeff_matches_decoding_of_a_real_polynomial():
    # the decode map of the oracle (pinned against its own O(N^2) definition) is U applied to
    # a_k = m_k + i m_{k+n}; the stages applied to bitrev(a) give the same slots
    N, n = 64, 32
    g = inputs.rng(920)
    m = g.integers(-1000, 1000, size=N)
    a = m[:n] + 1j * m[n:]
    out = a[blt.bitrev_perm(n)].astype(np.complex128)
    for s in range(1, n.bit_length()):
        out = blt.apply_diagonals(blt.stage_diagonals(N, s), out)
    assert np.abs(out - oracle.decode(m, 1.0, N)).max() < 1e-7


@pytest.mark.parametrize("N,levels", [(64, 2), (256, 3), (512, 3)])
@pytest.mark.parametrize("inverse", [False, True])
def test_level_diagonals_equal_dense_products(N, levels, inverse):
    n = N // 2
    for lo, hi in inputs.radix_levels(n.bit_length() - 1, levels):
        D = blt.level_diagonals(N, lo, hi, inverse)
        stages = range(lo, hi + 1) if not inverse else range(hi, lo - 1, -1)
        want = np.eye(n, dtype=np.complex128)
        for s in stages:
            want = dense(blt.stage_diagonals(N, s, inverse), n) @ want
        assert np.abs(dense(D, n) - want).max() < 1e-12
        # every nonzero diagonal is one of the plan's offsets (the structure the workload predicts)
        plan = inputs.bsgs_plan(n, lo, hi)
        assert set(D) <= set(plan.offsets)


@pytest.mark.parametrize("n,lo,hi", [(2048, 1, 4), (2048, 5, 8), (2048, 9, 11), (32768, 11, 15), (32768, 6, 10),
                                     (32768, 1, 5), (8, 1, 1), (8, 1, 3)])
def test_bsgs_plan_covers_each_offset_once(n, lo, hi):
    plan = inputs.bsgs_plan(n, lo, hi)
    D = (1 << (hi - lo + 1)) - 1
    want = {(d * plan.step) % n for d in range(-D, D + 1)}
    assert set(plan.offsets) == want and len(plan.offsets) == len(want)
    hit = {}
    for g, row in enumerate(plan.idx):
        assert any(j >= 0 for j in row)
        for b, j in enumerate(row):
            if j >= 0:
                assert (plan.giant[g] + plan.baby[b]) % n == plan.offsets[j]
                hit[j] = hit.get(j, 0) + 1
    assert sorted(hit) == list(range(plan.n_diag)) and set(hit.values()) == {1}
    assert plan.baby[0] == 0 and 0 in plan.giant


def test_plaintext_rotation_identity():
    # rot_G(pt (.) rot_b(z)) = diag_k (.) rot_k(z) for pt = roll(diag_k, G): the slot algebra
    # level_plaintexts relies on, checked in the clear
    n = 64
    g = inputs.rng(930)
    z, d = inputs.complex_slots(g, n), inputs.complex_slots(g, n)
    G, b = 40, 5
    pt = np.roll(d, G)
    lhs = np.roll(pt * np.roll(z, -b), -G)
    assert np.allclose(lhs, d * np.roll(z, -(G + b)))


def _setup(name, seed):
    P = inputs.workload_params(name)
    OP = oracle.OracleParams.from_params(P)
    W = inputs.WORKLOADS[name]
    g = inputs.rng(seed)
    sk = oracle.SecretKey(OP, inputs.ternary(g, P.N))
    return P, OP, W, g, sk


def _chain(P, OP, W, g, sk, kind, level, scale, noise):
    plans = inputs.transform_plans(P.N, W["levels"], kind)
    keys = {}
    for pl in plans:
        for r in pl.rotations():
            if r not in keys:
                keys[r] = oracle.rotation_key(OP, sk, r, g, noise=noise)
    levels = inputs.radix_levels((P.N // 2).bit_length() - 1, W["levels"])
    if kind == "cts":
        levels = levels[::-1]
    pts = []
    for i, (pl, (lo, hi)) in enumerate(zip(plans, levels)):
        D = blt.level_diagonals(P.N, lo, hi, inverse=(kind == "cts"))
        pts.append(blt.level_plaintexts(OP, D, pl, level - i, float(P.q[level - i - 1])))
    return plans, pts, keys, levels


@pytest.mark.parametrize("noise,bound", [(False, 2.0 ** -12), (True, 2.0 ** -7)])
def test_homomorphic_coeff_to_slot_then_slot_to_coeff_decodes(noise, bound):
    """CoeffToSlot (3 double-hoisted levels + rescales) decrypts to bitrev(U^-1 z); SlotToCoeff
    after it decrypts to U bitrev(.) of what CoeffToSlot decrypted to, and the round trip
    returns z.  Each level's plaintexts are encoded at the scale of the prime its rescale
    drops, so the ciphertext scale stays Delta = 2^28.  Without key and encryption noise
    only the rescale roundings remain (about 2^-13 here); with sigma = 3.2 the key-switching
    noise of this small ring is near 2^-9 after SlotToCoeff."""
    name = "cts_stc_N4096_L8"
    P, OP, W, g, sk = _setup(name, 940)
    n = P.N // 2
    scale = 2.0 ** W["scale_bits"]
    z = inputs.complex_slots(g, n)
    level = W["cts_level"]
    ct = oracle.encrypt(OP, sk, oracle.encode(z, scale, P.N), level, g, noise=noise)
    plans, pts, keys, levels = _chain(P, OP, W, g, sk, "cts", level, scale, noise)
    ct1 = blt.radix_transform(OP, ct, level, plans, pts, keys)
    l1 = level - len(plans)
    got = oracle.decode(oracle.decrypt(OP, sk, ct1, l1), scale, P.N)
    want = z.copy()
    for lo, hi in levels:
        want = blt.apply_diagonals(blt.level_diagonals(P.N, lo, hi, inverse=True), want)
    assert np.abs(blt.dft_matrix(P.N) @ want[blt.bitrev_perm(n)] - z).max() < 1e-9 * n
    err = np.abs(got - want).max()
    assert err < bound, err
    plans2, pts2, keys2, levels2 = _chain(P, OP, W, g, sk, "stc", l1, scale, noise)
    ct2 = blt.radix_transform(OP, ct1, l1, plans2, pts2, keys2)
    back = oracle.decode(oracle.decrypt(OP, sk, ct2, l1 - len(plans2)), scale, P.N)
    want2 = got.copy()
    for lo, hi in levels2:
        want2 = blt.apply_diagonals(blt.level_diagonals(P.N, lo, hi, inverse=False), want2)
    err2 = np.abs(back - want2).max()
    assert err2 < 4 * bound, err2
    # the round trip: CoeffToSlot's error comes back amplified by up to sqrt(n) (U / sqrt(n) is unitary)
    err3 = np.abs(back - z).max()
    assert err3 < 4 * bound * np.sqrt(n), err3
    print("noise", noise, "cts", err, "stc", err2, "round trip", err3)


def test_double_hoisting_matches_plain_evaluation_after_decryption():
    """One level without key or encryption noise: the double-hoisted result (before rescale)
    decrypts to the FP64 matrix-vector product within 2^-16 (its only rounding is the final
    ModDown), while a plain evaluation -- every rotation an ordinary key switch with its own
    ModUp and ModDown, every product in Q_l -- carries a ModDown rounding per rotation times the
    plaintext scale; both agree within that.  A dropped term or a wrong rotation would give
    errors of the size of the slots."""
    name = "cts_stc_N4096_L8"
    P, OP, W, g, sk = _setup(name, 950)
    n = P.N // 2
    scale = 2.0 ** W["scale_bits"]
    level = W["stc_level"]
    z = inputs.complex_slots(g, n)
    ct = oracle.encrypt(OP, sk, oracle.encode(z, scale, P.N), level, g, noise=False)
    lo, hi = inputs.radix_levels(n.bit_length() - 1, W["levels"])[0]
    plan = inputs.bsgs_plan(n, lo, hi)
    D = blt.level_diagonals(P.N, lo, hi, inverse=False)
    dscale = float(P.q[level - 1])
    pts = blt.level_plaintexts(OP, D, plan, level, dscale)
    keys = {r: oracle.rotation_key(OP, sk, r, g, noise=False) for r in plan.rotations()}
    dh = blt.lt_double_hoisted(OP, ct, level, plan.baby, plan.giant, pts, plan.idx, keys)
    acc = None
    for gi, row in enumerate(plan.idx):
        for b, j in enumerate(row):
            if j < 0:
                continue
            rb = ct if plan.baby[b] == 0 else oracle.rotate(OP, ct, level, plan.baby[b], keys[plan.baby[b]])
            t = np.stack([oracle.mul(rb[c], pts[j][:level], P.q) for c in range(2)])
            if plan.giant[gi]:
                t = oracle.rotate(OP, t, level, plan.giant[gi], keys[plan.giant[gi]])
            acc = t if acc is None else np.stack([oracle.add(acc[c], t[c], P.q) for c in range(2)])
    a = oracle.decode(oracle.decrypt(OP, sk, dh, level), scale * dscale, P.N)
    b = oracle.decode(oracle.decrypt(OP, sk, acc, level), scale * dscale, P.N)
    want = blt.apply_diagonals(D, z)
    assert np.abs(a - want).max() < 2.0 ** -16
    assert np.abs(b - want).max() < 2.0 ** -7
    assert np.abs(a - want).max() * 64 < np.abs(b - want).max()  # hoisting ModDown removes its roundings
