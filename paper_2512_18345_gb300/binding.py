"""Thin ctypes binding of the C ABI in include/fhe.h (argument marshalling only).

Device buffers are torch tensors (dtype int32 or uint32, contiguous, on the
context's device) holding the uint32 residues; the binding passes their
data_ptr() and the current torch stream's handle.  Every computation runs in
libfhe_gb300.so; there is no Python or CPU fallback: if the library is not
built, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence

import numpy as np

from . import build as _build

FHE_OK = 0
FHE_EINVAL, FHE_ELEVEL, FHE_ENOKEY, FHE_EPRIME, FHE_ENOMEM = -1, -2, -3, -4, -5
FHE_ECUDA, FHE_EALIAS, FHE_ETIMEOUT, FHE_EUNSUPPORTED = -6, -7, -8, -9
FHE_RELIN_KEY = -(2 ** 31)
FHE_BCONV_SCALAR, FHE_BCONV_TC = 0, 1
FHE_OP_KS, FHE_OP_ROTATE, FHE_OP_RELIN = 0, 1, 2
FHE_PLAN_GRAPH = 1
FHE_TUNE_BCONV = 1
FHE_TUNE_NTT = 2
FHE_TUNE_SHAPE = 4
FHE_NTT_OTF, FHE_NTT_SINGLE_PASS, FHE_NTT_STREAM, FHE_NTT_PERSIST = 1, 2, 4, 8

# every entry point declared in include/fhe.h
EXPORTS = (
    "fhe_ctx_create", "fhe_ctx_destroy", "fhe_ctx_info", "fhe_ctx_set_bconv", "fhe_ctx_set_fused", "fhe_ctx_sync",
    "fhe_set_relin_key", "fhe_set_rot_key", "fhe_keyswitch", "fhe_rotate", "fhe_hmult", "fhe_rescale",
    "fhe_rotate_hoisted", "fhe_linear_transform", "fhe_linear_transform_dh", "fhe_pmult", "fhe_add", "fhe_ntt", "fhe_intt", "fhe_modup", "fhe_moddown",
    "fhe_bconv", "fhe_batch_plan", "fhe_batch_launch", "fhe_plan_destroy", "fhe_plan_kernel_count",
    "fhe_plan_groups", "fhe_ctx_set_batch",
    "fhe_trace_enable", "fhe_trace_read", "fhe_probe_bandwidth", "fhe_probe_int", "fhe_autotune", "fhe_autotune_cached", "fhe_ctx_set_pipelining", "fhe_ctx_set_ntt", "fhe_ctx_set_kernel_shape", "fhe_ctx_get_kernel_shape", "fhe_ctx_set_memory_limit", "fhe_selftest_wait_timeout", "fhe_bconv_noalloc", "fhe_last_error",
)


class FheError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class FheInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_int), ("K", ctypes.c_int), ("dnum", ctypes.c_int),
                ("alpha", ctypes.c_int), ("device", ctypes.c_int), ("limb_bytes", ctypes.c_size_t),
                ("key_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
                ("table_bytes", ctypes.c_size_t), ("n_rot_keys", ctypes.c_int), ("bconv_mode", ctypes.c_int),
                ("psi", ctypes.c_uint32 * 64)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double)]


class IntPeaks(ctypes.Structure):
    _fields_ = [("clock_mhz", ctypes.c_double), ("butterflies_per_s", ctypes.c_double),
                ("mac64_per_s", ctypes.c_double), ("imad_per_s", ctypes.c_double),
                ("imad_hi_per_s", ctypes.c_double), ("add_min_per_s", ctypes.c_double), ("sms", ctypes.c_int)]


class KernelShape(ctypes.Structure):
    _fields_ = [("fuse_ip_moddown", ctypes.c_int), ("bconv_tc_ctas", ctypes.c_int),
                ("ntt_stream_stages", ctypes.c_int), ("ntt_stream_ctas", ctypes.c_int),
                ("bconv_tc_pipeline", ctypes.c_int), ("ip_staged_gather", ctypes.c_int),
                ("ip_staged_ctas", ctypes.c_int), ("ip_staged_depth", ctypes.c_int)]


class TuneResult(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int), ("l2_budget_bytes", ctypes.c_size_t), ("max_group", ctypes.c_int),
                ("bconv_mode", ctypes.c_int), ("n_groups", ctypes.c_int), ("us_per_ks", ctypes.c_double),
                ("default_us_per_ks", ctypes.c_double), ("candidates", ctypes.c_int),
                ("ip_ctas_per_sm", ctypes.c_int), ("comp_pipe", ctypes.c_int), ("ntt_mode", ctypes.c_int),
                ("shape", KernelShape)]


class KsItem(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("level", ctypes.c_int), ("rot", ctypes.c_int32),
                ("in_", ctypes.c_void_p), ("in2", ctypes.c_void_p), ("out", ctypes.c_void_p)]


_lib = None
vp = ctypes.c_void_p
ip = ctypes.POINTER(ctypes.c_int)


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libfhe_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(paper_2512_18345_gb300.build.build_library() or __graft_entry__.build())")
    L = ctypes.CDLL(path)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    sig = {
        "fhe_ctx_create": [ctypes.POINTER(vp), ctypes.c_uint32, u32p, ctypes.c_int, u32p, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int],
        "fhe_ctx_destroy": [vp],
        "fhe_ctx_info": [vp, ctypes.POINTER(FheInfo)],
        "fhe_ctx_set_bconv": [vp, ctypes.c_int],
        "fhe_ctx_set_fused": [vp, ctypes.c_int],
        "fhe_ctx_sync": [vp],
        "fhe_set_relin_key": [vp, vp, vp],
        "fhe_set_rot_key": [vp, ctypes.c_int32, vp, vp],
        "fhe_keyswitch": [vp, vp, ctypes.c_int, ctypes.c_int32, vp, vp],
        "fhe_rotate": [vp, vp, ctypes.c_int, ctypes.c_int32, vp, vp],
        "fhe_hmult": [vp, vp, vp, ctypes.c_int, vp, vp],
        "fhe_rescale": [vp, vp, ctypes.c_int, vp, vp],
        "fhe_rotate_hoisted": [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                               ctypes.POINTER(vp), vp],
        "fhe_linear_transform": [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp],
        "fhe_linear_transform_dh": [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int32), ctypes.c_int, vp, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int32), vp, vp],
        "fhe_pmult": [vp, vp, vp, ctypes.c_int, vp, vp],
        "fhe_add": [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp],
        "fhe_ntt": [vp, vp, ip, ctypes.c_int, vp],
        "fhe_intt": [vp, vp, ip, ctypes.c_int, vp],
        "fhe_modup": [vp, vp, ctypes.c_int, vp, vp],
        "fhe_moddown": [vp, vp, ctypes.c_int, vp, vp],
        "fhe_bconv": [vp, vp, ip, ctypes.c_int, vp, ip, ctypes.c_int, vp],
        "fhe_batch_plan": [vp, ctypes.POINTER(KsItem), ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
        "fhe_batch_launch": [vp, vp],
        "fhe_plan_destroy": [vp],
        "fhe_plan_kernel_count": [vp],
        "fhe_plan_groups": [vp, ip, ctypes.c_int],
        "fhe_ctx_set_batch": [vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int],
        "fhe_selftest_wait_timeout": [vp, vp],
        "fhe_ctx_set_pipelining": [vp, ctypes.c_int],
        "fhe_ctx_set_ntt": [vp, ctypes.c_int],
        "fhe_ctx_set_kernel_shape": [vp, ctypes.POINTER(KernelShape)],
        "fhe_ctx_get_kernel_shape": [vp, ctypes.POINTER(KernelShape)],
        "fhe_ctx_set_memory_limit": [vp, ctypes.c_size_t],
        "fhe_autotune": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(TuneResult), vp],
        "fhe_autotune_cached": [vp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(TuneResult), vp],
        "fhe_trace_enable": [vp, ctypes.c_int],
        "fhe_probe_bandwidth": [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "fhe_probe_int": [ctypes.c_int, ctypes.POINTER(IntPeaks)],
        "fhe_trace_read": [vp, ctypes.POINTER(KernelStat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "fhe_bconv_noalloc": [vp, vp, ip, ctypes.c_int, vp, ip, ctypes.c_int, vp],
        "fhe_last_error": [],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "fhe_last_error" else ctypes.c_int
    _lib = L
    return L


def check(rc: int) -> None:
    if rc != FHE_OK:
        raise FheError(rc, lib().fhe_last_error().decode())


def _ptr(t) -> vp:
    """Device pointer of a torch tensor (int32 / uint32, contiguous)."""
    if t is None:
        return vp(0)
    assert t.is_contiguous(), "buffers must be contiguous"
    return vp(t.data_ptr())


def _stream(stream) -> vp:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return vp(s.cuda_stream)


def _idx(xs: Sequence[int]):
    return (ctypes.c_int * len(xs))(*xs)


def to_device(a: np.ndarray, device: int = 0):
    """uint32 numpy array -> contiguous int32 torch tensor on cuda:device (bit copy)."""
    import torch
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(f"cuda:{device}")


def to_numpy(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def empty(shape, device: int = 0):
    import torch
    return torch.empty(tuple(shape), dtype=torch.int32, device=f"cuda:{device}")


def probe_bandwidth(device: int = 0, nbytes: int = 64 << 20, reps: int = 50) -> dict:
    """L2 (block smaller than L2) or DRAM bandwidth of 128-bit accesses, GB/s."""
    r, w, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(lib().fhe_probe_bandwidth(device, nbytes, reps, ctypes.byref(r), ctypes.byref(w), ctypes.byref(c)))
    return {"read": r.value, "write": w.value, "copy": c.value, "bytes": nbytes}


def probe_int(device: int = 0) -> dict:
    """Integer-pipe rates (units per second over the GPU) of register-only chains: the NTT's
    forward butterfly, the 64-bit multiply-accumulate, IMAD, IMAD.HI and add+min."""
    r = IntPeaks()
    check(lib().fhe_probe_int(device, ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in IntPeaks._fields_}


class Plan:
    def __init__(self, ctx: "Context", handle: vp, keep: list):
        self.ctx, self.h, self._keep = ctx, handle, keep

    def launch(self, stream=None) -> None:
        check(lib().fhe_batch_launch(self.h, _stream(stream)))

    @property
    def kernel_count(self) -> int:
        return lib().fhe_plan_kernel_count(self.h)

    @property
    def groups(self) -> List[int]:
        arr = (ctypes.c_int * 256)()
        n = lib().fhe_plan_groups(self.h, arr, 256)
        if n < 0:
            check(n)
        return list(arr[: min(n, 256)])

    def close(self) -> None:
        if self.h:
            check(lib().fhe_plan_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """An fhe_ctx: parameters, device tables, keys and workspace on one GPU."""

    def __init__(self, N: int, q: Sequence[int], p: Sequence[int], dnum: int, device: int = 0):
        self.N, self.q, self.p, self.dnum, self.device = N, list(q), list(p), dnum, device
        qa = (ctypes.c_uint32 * len(q))(*q)
        pa = (ctypes.c_uint32 * len(p))(*p)
        h = vp()
        check(lib().fhe_ctx_create(ctypes.byref(h), N, qa, len(q), pa, len(p), dnum, device))
        self.h = h

    @classmethod
    def from_params(cls, P, device: int = 0) -> "Context":
        return cls(P.N, P.q, P.p, P.dnum, device)

    def close(self) -> None:
        if getattr(self, "h", None):
            check(lib().fhe_ctx_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def L(self):
        return len(self.q)

    @property
    def K(self):
        return len(self.p)

    def info(self) -> dict:
        i = FheInfo()
        check(lib().fhe_ctx_info(self.h, ctypes.byref(i)))
        d = {f: getattr(i, f) for f, _ in FheInfo._fields_ if f != "psi"}
        d["psi"] = list(i.psi)[: i.L + i.K]
        return d

    def sync(self) -> None:
        """Synchronize the device; raises FheError(FHE_ETIMEOUT) if a device-side wait expired."""
        check(lib().fhe_ctx_sync(self.h))

    def set_bconv(self, mode: int) -> None:
        check(lib().fhe_ctx_set_bconv(self.h, mode))

    def set_batch(self, l2_budget_bytes: int = 0, max_group: int = 0, lanes: int = 0) -> None:
        check(lib().fhe_ctx_set_batch(self.h, l2_budget_bytes, max_group, lanes))

    def selftest_wait_timeout(self, stream=None) -> None:
        """Enqueue a bounded wait that expires; the next sync reports FHE_ETIMEOUT."""
        check(lib().fhe_selftest_wait_timeout(self.h, _stream(stream)))

    def autotune(self, level: int, n_items: int, flags: int = 0, stream=None, cache: Optional[str] = None) -> dict:
        """Measure the batched-plan schedules on the device and keep the fastest
        (with `cache`: reuse or record the choice in that file)."""
        r = TuneResult()
        if cache:
            check(lib().fhe_autotune_cached(self.h, os.fsencode(cache), level, n_items, flags, ctypes.byref(r),
                                            _stream(stream)))
        else:
            check(lib().fhe_autotune(self.h, level, n_items, flags, ctypes.byref(r), _stream(stream)))
        out = {f: getattr(r, f) for f, _ in TuneResult._fields_ if f != "shape"}
        out["shape"] = {f: getattr(r.shape, f) for f, _ in KernelShape._fields_}
        return out

    def set_memory_limit(self, nbytes: int) -> None:
        """Cap the device memory the context may still grow into (0: no cap)."""
        check(lib().fhe_ctx_set_memory_limit(self.h, int(nbytes)))

    def set_ntt(self, flags: int) -> None:
        """NTT kernel variants: 0, FHE_NTT_OTF | FHE_NTT_SINGLE_PASS | FHE_NTT_STREAM flags, or FHE_NTT_PERSIST."""
        check(lib().fhe_ctx_set_ntt(self.h, int(flags)))

    def kernel_shape(self) -> dict:
        r = KernelShape()
        check(lib().fhe_ctx_get_kernel_shape(self.h, ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in KernelShape._fields_}

    def set_kernel_shape(self, **kw) -> None:
        """Change some fields of the kernel shape (fuse_ip_moddown, bconv_tc_ctas,
        ntt_stream_stages, ntt_stream_ctas, bconv_tc_pipeline, ip_staged_gather, ip_staged_ctas,
        ip_staged_depth); the others keep their values."""
        cur = self.kernel_shape()
        unknown = set(kw) - set(cur)
        if unknown:
            raise ValueError(f"unknown kernel-shape fields {sorted(unknown)}")
        cur.update(kw)
        r = KernelShape(**{k: int(v) for k, v in cur.items()})
        check(lib().fhe_ctx_set_kernel_shape(self.h, ctypes.byref(r)))

    def set_pipelining(self, on: bool) -> None:
        check(lib().fhe_ctx_set_pipelining(self.h, 1 if on else 0))

    def set_fused(self, fused: bool) -> None:
        check(lib().fhe_ctx_set_fused(self.h, int(bool(fused))))

    def trace(self, on: bool) -> None:
        check(lib().fhe_trace_enable(self.h, int(bool(on))))

    def trace_read(self) -> dict:
        """{kernel name: (launches, total ms)} since the last read (synchronizes)."""
        arr = (KernelStat * 64)()
        n = ctypes.c_int()
        check(lib().fhe_trace_read(self.h, arr, 64, ctypes.byref(n)))
        return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(min(n.value, 64))}

    def set_relin_key(self, key, stream=None) -> None:
        check(lib().fhe_set_relin_key(self.h, _ptr(key), _stream(stream)))

    def set_rot_key(self, rot: int, key, stream=None) -> None:
        check(lib().fhe_set_rot_key(self.h, rot, _ptr(key), _stream(stream)))

    def _out(self, out, shape):
        return out if out is not None else empty(shape, self.device)

    def keyswitch(self, d, level: int, key_id: int = FHE_RELIN_KEY, out=None, stream=None):
        out = self._out(out, (2, level, self.N))
        check(lib().fhe_keyswitch(self.h, _ptr(d), level, key_id, _ptr(out), _stream(stream)))
        return out

    def rotate(self, ct, level: int, rot: int, out=None, stream=None):
        out = self._out(out, (2, level, self.N))
        check(lib().fhe_rotate(self.h, _ptr(ct), level, rot, _ptr(out), _stream(stream)))
        return out

    def hmult(self, a, b, level: int, out=None, stream=None):
        out = self._out(out, (2, level, self.N))
        check(lib().fhe_hmult(self.h, _ptr(a), _ptr(b), level, _ptr(out), _stream(stream)))
        return out

    def rescale(self, ct, level: int, out=None, stream=None):
        out = self._out(out, (2, level - 1, self.N))
        check(lib().fhe_rescale(self.h, _ptr(ct), level, _ptr(out), _stream(stream)))
        return out

    def rotate_hoisted(self, ct, level: int, rots: Sequence[int], outs=None, stream=None):
        outs = outs if outs is not None else [empty((2, level, self.N), self.device) for _ in rots]
        n = len(rots)
        r = (ctypes.c_int32 * n)(*rots)
        o = (vp * n)(*[o.data_ptr() for o in outs])
        check(lib().fhe_rotate_hoisted(self.h, _ptr(ct), level, r, n, o, _stream(stream)))
        return outs

    def linear_transform(self, ct, level: int, diags, baby: int, giant: int, out=None, stream=None):
        out = self._out(out, (2, level, self.N))
        check(lib().fhe_linear_transform(self.h, _ptr(ct), level, _ptr(diags), baby, giant, _ptr(out), _stream(stream)))
        return out

    def linear_transform_dh(self, ct, level: int, baby, giant, diags, idx, out=None, stream=None):
        """Double-hoisted transform; diags [n_diag][level+K][N] (device), idx [n_giant][n_baby] host ints."""
        out = self._out(out, (2, level, self.N))
        baby, giant = list(baby), list(giant)
        flat = [int(x) for row in idx for x in row]
        b = (ctypes.c_int32 * len(baby))(*baby)
        g = (ctypes.c_int32 * len(giant))(*giant)
        ix = (ctypes.c_int32 * len(flat))(*flat)
        n_diag = int(diags.shape[0])
        check(lib().fhe_linear_transform_dh(self.h, _ptr(ct), level, b, len(baby), g, len(giant), _ptr(diags), n_diag,
                                            ix, _ptr(out), _stream(stream)))
        return out

    def pmult(self, ct, pt, level: int, out=None, stream=None):
        out = self._out(out, (2, level, self.N))
        check(lib().fhe_pmult(self.h, _ptr(ct), _ptr(pt), level, _ptr(out), _stream(stream)))
        return out

    def add(self, a, b, level: int, npoly: int = 2, out=None, stream=None):
        out = self._out(out, (npoly, level, self.N))
        check(lib().fhe_add(self.h, _ptr(a), _ptr(b), npoly, level, _ptr(out), _stream(stream)))
        return out

    def ntt(self, a, prime_idx: Sequence[int], stream=None):
        check(lib().fhe_ntt(self.h, _ptr(a), _idx(prime_idx), len(prime_idx), _stream(stream)))
        return a

    def intt(self, a, prime_idx: Sequence[int], stream=None):
        check(lib().fhe_intt(self.h, _ptr(a), _idx(prime_idx), len(prime_idx), _stream(stream)))
        return a

    def beta(self, level: int) -> int:
        alpha = -(-self.L // self.dnum)
        return -(-level // alpha)

    def modup(self, d, level: int, ext=None, stream=None):
        ext = self._out(ext, (self.beta(level), level + self.K, self.N))
        check(lib().fhe_modup(self.h, _ptr(d), level, _ptr(ext), _stream(stream)))
        return ext

    def moddown(self, u, level: int, out=None, stream=None):
        out = self._out(out, (level, self.N))
        check(lib().fhe_moddown(self.h, _ptr(u), level, _ptr(out), _stream(stream)))
        return out

    def bconv(self, x, in_idx: Sequence[int], out_idx: Sequence[int], out=None, stream=None):
        out = self._out(out, (len(out_idx), self.N))
        check(lib().fhe_bconv(self.h, _ptr(x), _idx(in_idx), len(in_idx), _ptr(out), _idx(out_idx), len(out_idx),
                              _stream(stream)))
        return out

    def bconv_noalloc(self, x, in_idx: Sequence[int], out_idx: Sequence[int], out, stream=None):
        """fhe_bconv without any device allocation (fixed shared scratch; out must be given)."""
        check(lib().fhe_bconv_noalloc(self.h, _ptr(x), _idx(in_idx), len(in_idx), _ptr(out), _idx(out_idx),
                                      len(out_idx), _stream(stream)))
        return out

    def batch_plan(self, items: Iterable[dict], flags: int = FHE_PLAN_GRAPH) -> Plan:
        items = list(items)
        arr = (KsItem * max(1, len(items)))()
        keep = []
        for i, it in enumerate(items):
            arr[i].op, arr[i].level, arr[i].rot = it["op"], it["level"], it.get("rot", 0)
            arr[i].in_ = it["in"].data_ptr()
            arr[i].in2 = it["in2"].data_ptr() if it.get("in2") is not None else 0
            arr[i].out = it["out"].data_ptr()
            keep += [it["in"], it.get("in2"), it["out"]]
        h = vp()
        check(lib().fhe_batch_plan(self.h, arr, len(items), flags, ctypes.byref(h)))
        return Plan(self, h, keep)
