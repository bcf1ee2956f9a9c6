"""The allocation-free base conversion (fhe_bconv_noalloc) against the
allocating one (fhe_bconv), called through the C ABI.

fhe_bconv_noalloc exists for callers that cannot allocate device memory
(stream capture in progress, latency-critical loops, a framework pool holding
all memory).  Its scratch is one fixed device array shared by every call, so
the test makes two different calls in a row: the second must not see the
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
