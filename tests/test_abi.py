"""The C-ABI library loads and exports every entry point include/fhe.h
declares; host-side argument validation works without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2512_18345_gb300 import binding, inputs

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fhe.h")


def declared():
    return sorted(set(re.findall(r"^FHE_API\s+[\w\s\*]*?\b(fhe_\w+)\(", open(HEADER).read(), flags=re.M)))


def test_header_declarations_match_binding(fhe_lib):
    names = declared()
    assert len(names) >= 20
    assert sorted(binding.EXPORTS) == names


def test_every_declared_symbol_is_exported(fhe_lib):
    for name in declared():
        assert hasattr(fhe_lib, name), name
        assert ctypes.cast(getattr(fhe_lib, name), ctypes.c_void_p).value


def test_library_is_sm103a_only():
    from paper_2512_18345_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)


def _create(N, q, p, dnum):
    h = ctypes.c_void_p()
    qa = (ctypes.c_uint32 * len(q))(*q)
    pa = (ctypes.c_uint32 * len(p))(*p)
    rc = binding.lib().fhe_ctx_create(ctypes.byref(h), N, qa, len(q), pa, len(p), dnum, 0)
    return rc, h


def test_bad_parameters_rejected_before_device_use(fhe_lib):
    P = inputs.workload_params("hmult_relin_rescale_N4096_L4")
    q, p = list(P.q), list(P.p)
    rc, h = _create(P.N, q[:-1] + [q[0]], p, 2)            # repeated prime
    assert rc == binding.FHE_EPRIME and not h.value
    rc, _ = _create(P.N, q[:-1] + [q[-1] + 2 * P.N * 0 + 2], p, 2)  # not prime / not 1 mod 2N
    assert rc == binding.FHE_EPRIME
    rc, _ = _create(P.N, q[:-1] + [(1 << 31) + 1], p, 2)     # >= 2^31
    assert rc == binding.FHE_EPRIME
    rc, _ = _create(2048, q, p, 2)                            # unsupported ring degree
    assert rc == binding.FHE_EUNSUPPORTED
    rc, _ = _create(P.N, q, p, 0)                             # dnum out of range
    assert rc == binding.FHE_EINVAL
    assert binding.lib().fhe_last_error()


def test_null_handles_rejected(fhe_lib):
    L = binding.lib()
    assert L.fhe_ctx_destroy(None) == binding.FHE_EINVAL
    assert L.fhe_keyswitch(None, None, 1, 0, None, None) == binding.FHE_EINVAL
    assert L.fhe_batch_launch(None, None) == binding.FHE_EINVAL
    assert L.fhe_plan_kernel_count(None) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        binding.lib()
