"""The allocation-free base conversion (fhe_bconv_noalloc) against the
allocating one (fhe_bconv), called through the C ABI.

fhe_bconv_noalloc exists for callers that cannot allocate device memory once
they run: a process whose framework pool already holds all free device memory,
or a real-time loop that must not take cudaMalloc's device-wide
synchronization.  Its scratch is one fixed device array shared by every call,
so the tests make two different calls in a row: the second must not see the
first one's leftovers.  The file name sorts last so that a run stopping at the
first failure has run every other test first.
"""
import numpy as np
import pytest

from paper_2512_18345_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_bconv_noalloc_matches_bconv_twice(fhe_lib):
    import torch
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hrotate_N65536_L24_plain")
    ctx = binding.Context.from_params(P)
    g = inputs.rng(4242)
    calls = [(list(range(24, 32)), list(range(24))),        # 8 special primes -> 24 ciphertext primes
             (list(range(3, 8)), list(range(8, 32)) + [0])]  # 5 inputs -> 25 outputs, other primes
    for in_idx, out_idx in calls:
        x = inputs.uniform_residues(g, [P.primes[i] for i in in_idx], P.N)
        xd = binding.to_device(x)
        want = ctx.bconv(xd, in_idx, out_idx)
        got = binding.empty((len(out_idx), P.N))
        got.fill_(-1)
        ctx.bconv_noalloc(xd, in_idx, out_idx, got)
        torch.cuda.synchronize()
        assert np.array_equal(binding.to_numpy(got), binding.to_numpy(want))
    ctx.close()


def test_bconv_noalloc_queued_behind_other_work(fhe_lib):
    """Both calls are enqueued while the stream is still busy, so neither has run when the
    second one returns: each call's tables travel with its own launch."""
    import torch
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hrotate_N65536_L24_plain")
    ctx = binding.Context.from_params(P)
    g = inputs.rng(4343)
    calls = [(list(range(16, 24)), list(range(16)) + list(range(24, 32))),
             (list(range(0, 3)), list(range(3, 30)))]
    xs = [binding.to_device(inputs.uniform_residues(g, [P.primes[i] for i in c[0]], P.N)) for c in calls]
    wants = [ctx.bconv(x, c[0], c[1]) for x, c in zip(xs, calls)]
    torch.cuda.synchronize()
    outs = [binding.empty((len(c[1]), P.N)) for c in calls]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        torch.cuda._sleep(20_000_000)  # about 10 ms of one busy thread
        for x, c, o in zip(xs, calls, outs):
            ctx.bconv_noalloc(x, c[0], c[1], o, stream=s)
    s.synchronize()
    for o, w in zip(outs, wants):
        assert np.array_equal(binding.to_numpy(o), binding.to_numpy(w))
    ctx.close()


def test_bconv_noalloc_rejects_sizes_beyond_its_scratch(fhe_lib):
    from paper_2512_18345_gb300 import binding
    P = inputs.workload_params("hrotate_N65536_L24_plain")
    ctx = binding.Context.from_params(P)
    x = binding.empty((9, P.N))
    out = binding.empty((4, P.N))
    with pytest.raises(binding.FheError) as e:
        ctx.bconv_noalloc(x, list(range(9)), list(range(9, 13)), out)
    assert e.value.code == binding.FHE_EINVAL and "scratch" in str(e.value)
    ctx.close()
