"""Python side of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Wraps the plain C oracle (`fhe_oracle.c`) with ctypes and adds the host-side
CKKS pieces the CUDA library does not implement (encoding, encryption,
decryption, key generation) plus the big-integer CRT used by the pins.

Conventions (restated from the CKKS literature the paper cites for the
mathematics it leaves out, Section II-A):
  * a polynomial at level l is [l][N] uint32, limb i modulo q_i, NTT form
    (bit-reversed evaluation order, see `fhe_oracle.c`);
  * a ciphertext is (c0, c1) with c0 + c1 * s = m + small (mod Q_l);
  * a switching key from s' to s is, for each digit j < dnum,
      b_j = -a_j s + e_j + g_j s',  g_j = [P]_{q_i} on digit j's q-limbs and 0
    on every other limb (q or p),  stored [dnum][2][L+K][N] as (b_j, a_j);
  * slot j of a message is its value at zeta^(5^j), zeta = exp(i pi / N).

Pin status of every oracle function (the tests under `tests/` hold the pins):
  ntt / intt           pinned: O(N^2) definition, convolution theorem, inverse
  bconv                pinned: big-integer CRT (x + e Q*, one e per column)
  modup                pinned: CRT check of every converted limb
  moddown              pinned: big-integer floor(U / P) - e, e in [0, K)
  keyswitch            pinned: closed-form error bound with a noise-free key
  automorph_ntt        pinned: coefficient-domain definition + slot rotation
  rotate / hoisted     pinned: decode equals the rotated message
  hmult / rescale      pinned: big-integer floor(C / q_last); decode = z1 z2
  encode / decode      pinned: O(N^2) slot evaluation, ring homomorphism
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fhe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

u32p = ctypes.POINTER(ctypes.c_uint32)


def build_oracle(force: bool = False) -> str:
    """Compile fhe_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_int), ("K", ctypes.c_int),
                ("dnum", ctypes.c_int), ("primes", u32p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build_oracle())
            L = _lib
            L.orc_powmod.restype = ctypes.c_uint32
            L.orc_powmod.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
            L.orc_invmod.restype = ctypes.c_uint32
            L.orc_invmod.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_psi.restype = ctypes.c_uint32
            L.orc_psi.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_galois_elt.restype = ctypes.c_uint32
            L.orc_galois_elt.argtypes = [ctypes.c_int32, ctypes.c_uint32]
            for f in ("orc_ntt", "orc_intt"):
                getattr(L, f).argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint32]
            for f in ("orc_ntt_limbs", "orc_intt_limbs"):
                getattr(L, f).argtypes = [u32p, ctypes.c_int, u32p, ctypes.c_uint32]
            L.orc_bconv.argtypes = [u32p, ctypes.c_int, u32p, u32p, ctypes.c_int, u32p, ctypes.c_uint32]
            L.orc_automorph_coef.argtypes = [u32p, u32p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            L.orc_automorph_ntt.argtypes = [u32p, u32p, ctypes.c_uint32, ctypes.c_uint32]
            P = ctypes.POINTER(_Params)
            L.orc_modup.argtypes = [P, u32p, ctypes.c_int, ctypes.c_int, u32p]
            L.orc_inner_product.argtypes = [P, u32p, ctypes.c_int, u32p, u32p]
            L.orc_moddown.argtypes = [P, u32p, ctypes.c_int, u32p]
            L.orc_keyswitch.argtypes = [P, u32p, ctypes.c_int, u32p, u32p]
            L.orc_rotate.argtypes = [P, u32p, ctypes.c_int, ctypes.c_int32, u32p, u32p]
            L.orc_rotate_hoisted.argtypes = [P, u32p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                             ctypes.POINTER(u32p), u32p]
            L.orc_hmult.argtypes = [P, u32p, u32p, ctypes.c_int, u32p, u32p]
            L.orc_rescale.argtypes = [P, u32p, ctypes.c_int, u32p]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            for f in ("orc_modup", "orc_keyswitch", "orc_rotate", "orc_rotate_hoisted", "orc_hmult", "orc_rescale"):
                getattr(L, f).restype = ctypes.c_int
        return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(u32p)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


class OracleParams:
    """Parameter set handed to the C oracle (keeps the prime array alive)."""

    def __init__(self, N: int, q: Sequence[int], p: Sequence[int], dnum: int):
        self.N, self.q, self.p, self.dnum = int(N), tuple(int(x) for x in q), tuple(int(x) for x in p), int(dnum)
        self.primes_arr = _u32(list(self.q) + list(self.p))
        self.c = _Params(self.N, len(self.q), len(self.p), self.dnum, _p(self.primes_arr))

    @classmethod
    def from_params(cls, P) -> "OracleParams":
        return cls(P.N, P.q, P.p, P.dnum)

    @property
    def L(self):
        return len(self.q)

    @property
    def K(self):
        return len(self.p)

    @property
    def alpha(self):
        return -(-self.L // self.dnum)

    def beta(self, level):
        return -(-level // self.alpha)

    @property
    def primes(self):
        return self.q + self.p

    def ext_primes(self, level):
        return self.q[:level] + self.p

    @property
    def P_prod(self) -> int:
        r = 1
        for x in self.p:
            r *= x
        return r

    def ref(self):
        return ctypes.byref(self.c)


# ------------------------------------------------------------------ scalar helpers

def psi(q: int, N: int) -> int:
    return int(lib().orc_psi(q, N))


def galois_elt(rot: int, N: int) -> int:
    return int(lib().orc_galois_elt(rot, N))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(n)


# ------------------------------------------------------------------ transforms

def ntt(a: np.ndarray, primes: Sequence[int]) -> np.ndarray:
    """Limb-wise forward NTT of an [n][N] array (returns a new array)."""
    a = _u32(a).copy()
    n, N = a.shape
    lib().orc_ntt_limbs(_p(a), n, _p(_u32(primes[:n])), N)
    return a


def intt(a: np.ndarray, primes: Sequence[int]) -> np.ndarray:
    a = _u32(a).copy()
    n, N = a.shape
    lib().orc_intt_limbs(_p(a), n, _p(_u32(primes[:n])), N)
    return a


def bconv(x: np.ndarray, q_in: Sequence[int], p_out: Sequence[int]) -> np.ndarray:
    """Fast base conversion of a coefficient-form [len(q_in)][N] array."""
    x = _u32(x)
    n_in, N = x.shape
    out = np.empty((len(p_out), N), dtype=np.uint32)
    lib().orc_bconv(_p(x), n_in, _p(_u32(q_in)), _p(out), len(p_out), _p(_u32(p_out)), N)
    return out


def automorph_coef(a: np.ndarray, k: int, primes: Sequence[int]) -> np.ndarray:
    a = _u32(a)
    out = np.empty_like(a)
    for i in range(a.shape[0]):
        lib().orc_automorph_coef(_p(a[i]), _p(out[i]), a.shape[1], k, primes[i])
    return out


def automorph_ntt(a: np.ndarray, k: int) -> np.ndarray:
    a = _u32(a)
    out = np.empty_like(a)
    for i in range(a.shape[0]):
        lib().orc_automorph_ntt(_p(a[i]), _p(out[i]), a.shape[1], k)
    return out


# ------------------------------------------------------------------ key switching ops

def modup(P: OracleParams, d: np.ndarray, level: int, j: int) -> np.ndarray:
    d = _u32(d)
    ext = np.zeros((level + P.K, P.N), dtype=np.uint32)
    rc = lib().orc_modup(P.ref(), _p(d), level, j, _p(ext))
    assert rc == 0
    return ext


def inner_product(P: OracleParams, ext: np.ndarray, level: int, key: np.ndarray) -> np.ndarray:
    u = np.empty((2, level + P.K, P.N), dtype=np.uint32)
    lib().orc_inner_product(P.ref(), _p(_u32(ext)), level, _p(_u32(key)), _p(u))
    return u


def moddown(P: OracleParams, u: np.ndarray, level: int) -> np.ndarray:
    out = np.empty((level, P.N), dtype=np.uint32)
    lib().orc_moddown(P.ref(), _p(_u32(u)), level, _p(out))
    return out


def keyswitch(P: OracleParams, d: np.ndarray, level: int, key: np.ndarray) -> np.ndarray:
    out = np.empty((2, level, P.N), dtype=np.uint32)
    rc = lib().orc_keyswitch(P.ref(), _p(_u32(d)), level, _p(_u32(key)), _p(out))
    assert rc == 0
    return out


def rotate(P: OracleParams, ct: np.ndarray, level: int, rot: int, key: np.ndarray) -> np.ndarray:
    out = np.empty((2, level, P.N), dtype=np.uint32)
    rc = lib().orc_rotate(P.ref(), _p(_u32(ct)), level, rot, _p(_u32(key)), _p(out))
    assert rc == 0
    return out


def rotate_hoisted(P: OracleParams, ct: np.ndarray, level: int, rots: Sequence[int],
                   keys: Sequence[np.ndarray]) -> np.ndarray:
    n = len(rots)
    outs = np.empty((n, 2, level, P.N), dtype=np.uint32)
    keys_c = [_u32(k) if k is not None else np.zeros(1, np.uint32) for k in keys]
    kp = (u32p * n)(*[_p(k) for k in keys_c])
    r = (ctypes.c_int32 * n)(*rots)
    rc = lib().orc_rotate_hoisted(P.ref(), _p(_u32(ct)), level, r, n, kp, _p(outs))
    assert rc == 0
    return outs


def hmult(P: OracleParams, a: np.ndarray, b: np.ndarray, level: int, key: np.ndarray) -> np.ndarray:
    out = np.empty((2, level, P.N), dtype=np.uint32)
    rc = lib().orc_hmult(P.ref(), _p(_u32(a)), _p(_u32(b)), level, _p(_u32(key)), _p(out))
    assert rc == 0
    return out


def rescale(P: OracleParams, ct: np.ndarray, level: int) -> np.ndarray:
    out = np.empty((2, level - 1, P.N), dtype=np.uint32)
    rc = lib().orc_rescale(P.ref(), _p(_u32(ct)), level, _p(out))
    assert rc == 0
    return out


def add(a: np.ndarray, b: np.ndarray, primes: Sequence[int]) -> np.ndarray:
    q = np.asarray(primes[: a.shape[-2]], dtype=np.uint64)[:, None]
    return ((a.astype(np.uint64) + b.astype(np.uint64)) % q).astype(np.uint32)


def mul(a: np.ndarray, b: np.ndarray, primes: Sequence[int]) -> np.ndarray:
    q = np.asarray(primes[: a.shape[-2]], dtype=np.uint64)[:, None]
    return ((a.astype(np.uint64) * b.astype(np.uint64)) % q).astype(np.uint32)


def neg(a: np.ndarray, primes: Sequence[int]) -> np.ndarray:
    q = np.asarray(primes[: a.shape[-2]], dtype=np.uint64)[:, None]
    return ((q - a.astype(np.uint64)) % q).astype(np.uint32)


def bsgs_linear_transform(P: OracleParams, ct: np.ndarray, level: int, diags: np.ndarray, baby: int, giant: int,
                          rot_keys: dict) -> np.ndarray:
    """Baby-step / giant-step plaintext matrix-vector product (before rescale):
        sum_g rot_{baby*g}( sum_b diag[g*baby + b] (.) rot_b(ct) ),
    with the baby rotations hoisted (one shared ModUp).  diags is
    [giant*baby][level][N] NTT-form plaintexts.  rot_keys maps rotation index
    -> key.  Output [2][level][N]."""
    rots = list(range(baby))
    keys = [rot_keys.get(r) if r else None for r in rots]
    babies = rotate_hoisted(P, ct, level, rots, keys)
    primes = P.primes
    acc = None
    for g in range(giant):
        inner = None
        for b in range(baby):
            d = diags[g * baby + b]
            term = np.stack([mul(babies[b][c], d, primes) for c in range(2)])
            inner = term if inner is None else np.stack([add(inner[c], term[c], primes) for c in range(2)])
        if g:
            inner = rotate(P, inner, level, baby * g, rot_keys[baby * g])
        acc = inner if acc is None else np.stack([add(acc[c], inner[c], primes) for c in range(2)])
    return acc


# ------------------------------------------------------------------ integers, CRT

def to_rns(coeffs: Sequence[int] | np.ndarray, primes: Sequence[int]) -> np.ndarray:
    """Integer (possibly negative or big) coefficients -> [len(primes)][N] residues."""
    c = np.asarray(coeffs, dtype=object)
    out = np.empty((len(primes), len(c)), dtype=np.uint32)
    small = all(isinstance(x, (int, np.integer)) and abs(int(x)) < (1 << 62) for x in c[:8])
    for i, q in enumerate(primes):
        if small:
            out[i] = np.mod(np.asarray(coeffs, dtype=np.int64), q).astype(np.uint32)
        else:
            out[i] = np.array([int(x) % q for x in c], dtype=np.uint32)
    return out


def crt(residues: np.ndarray, primes: Sequence[int], centered: bool = True) -> List[int]:
    """Big-integer CRT of [n][N] residues; centered lift to (-Q/2, Q/2] if asked."""
    n, N = residues.shape
    Q = 1
    for q in primes[:n]:
        Q *= int(q)
    acc = np.zeros(N, dtype=object)
    for i in range(n):
        q = int(primes[i])
        Mi = Q // q
        ci = Mi * pow(Mi % q, -1, q)
        acc = acc + residues[i].astype(object) * ci
    acc = acc % Q
    if centered:
        half = Q // 2
        acc = np.where(acc > half, acc - Q, acc)
    return [int(x) for x in acc]


# ------------------------------------------------------------------ CKKS encode / decode

def _slot_exponents(N: int) -> np.ndarray:
    e = np.empty(N // 2, dtype=np.int64)
    x = 1
    for j in range(N // 2):
        e[j] = x
        x = x * 5 % (2 * N)
    return e


def encode_real(z: np.ndarray, N: int) -> np.ndarray:
    """tau^-1(z) as real coefficients (before scaling/rounding):
    m_n = (2/N) Re( sum_j z_j zeta^(-5^j n) ), n < N, via one length-2N FFT."""
    A = np.zeros(2 * N, dtype=np.complex128)
    A[_slot_exponents(N)] = z
    F = np.fft.fft(A)  # F[n] = sum_e A[e] exp(-2 pi i e n / 2N) = sum_j z_j zeta^(-5^j n)
    return (2.0 / N) * F[:N].real


def round_half_away(x: np.ndarray) -> np.ndarray:
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def encode(z: np.ndarray, scale: float, N: int) -> np.ndarray:
    """Integer coefficients round(scale * tau^-1(z)), round half away from zero (int64)."""
    return round_half_away(scale * encode_real(z, N)).astype(np.int64)


def decode(m: Sequence[float] | np.ndarray, scale: float, N: int) -> np.ndarray:
    """tau(m) / scale: slot j = sum_n m_n zeta^(5^j n) / scale."""
    M = np.zeros(2 * N, dtype=np.complex128)
    M[:N] = np.asarray([float(x) for x in m], dtype=np.float64)
    G = np.fft.ifft(M) * (2 * N)  # G[e] = sum_n M[n] exp(2 pi i e n / 2N)
    return G[_slot_exponents(N)] / scale


# ------------------------------------------------------------------ keys, encryption

class SecretKey:
    """Ternary secret s; `ntt` holds NTT(s) over all L + K primes."""

    def __init__(self, P: OracleParams, coeffs: np.ndarray):
        self.P = P
        self.coeffs = np.asarray(coeffs, dtype=np.int64)
        self.ntt = ntt(to_rns(self.coeffs, P.primes), P.primes)

    @property
    def hamming_weight(self) -> int:
        return int(np.count_nonzero(self.coeffs))


def automorph_int(coeffs: np.ndarray, k: int) -> np.ndarray:
    """sigma_k on an integer polynomial: X^n -> X^(nk mod 2N), X^N = -1."""
    N = len(coeffs)
    out = np.zeros(N, dtype=np.int64)
    e = (np.arange(N, dtype=np.int64) * k) % (2 * N)
    pos = e < N
    out[e[pos]] = coeffs[pos]
    out[e[~pos] - N] = -coeffs[~pos]
    return out


def negacyclic_mul_int(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Plain O(N^2) product in Z[X]/(X^N + 1) (python ints; small N only)."""
    N = len(a)
    out = [0] * N
    for i in range(N):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += ai * int(b[j])
            else:
                out[k - N] -= ai * int(b[j])
    return out


def switching_key(P: OracleParams, sk: SecretKey, s_from_ntt: np.ndarray, g: np.random.Generator,
                  noise: bool = True) -> np.ndarray:
    """Key switching s' -> s.  s_from_ntt is NTT(s') over all L+K primes.
    For each digit j (draw order: a_j, then e_j):  a_j uniform, e_j Gaussian,
    b_j = -a_j s + e_j + g_j s'.  Returns [dnum][2][L+K][N] = (b_j, a_j)."""
    from paper_2512_18345_gb300 import inputs
    primes = P.primes
    n = len(primes)
    key = np.empty((P.dnum, 2, n, P.N), dtype=np.uint32)
    Pp = P.P_prod
    for j in range(P.dnum):
        a = inputs.uniform_residues(g, primes, P.N)
        e = inputs.gaussian(g, P.N)
        if not noise:
            e = np.zeros_like(e)
        e_ntt = ntt(to_rns(e, primes), primes)
        b = add(neg(mul(a, sk.ntt, primes), primes), e_ntt, primes)
        lo, hi = j * P.alpha, min((j + 1) * P.alpha, P.L)
        for i in range(lo, hi):
            q = primes[i]
            gs = (np.asarray(s_from_ntt[i], dtype=np.uint64) * (Pp % q)) % q
            b[i] = ((b[i].astype(np.uint64) + gs) % q).astype(np.uint32)
        key[j, 0], key[j, 1] = b, a
    return key


def relin_key(P: OracleParams, sk: SecretKey, g, noise: bool = True) -> np.ndarray:
    return switching_key(P, sk, mul(sk.ntt, sk.ntt, P.primes), g, noise)


def rotation_key(P: OracleParams, sk: SecretKey, rot: int, g, noise: bool = True) -> np.ndarray:
    k = galois_elt(rot, P.N)
    s_rot = automorph_int(sk.coeffs, k)
    return switching_key(P, sk, ntt(to_rns(s_rot, P.primes), P.primes), g, noise)


def encrypt(P: OracleParams, sk: SecretKey, m_coeffs, level: int, g, noise: bool = True) -> np.ndarray:
    """Secret-key encryption at `level`: c1 = a uniform, c0 = -a s + e + m (NTT form).
    Draw order: a, then e."""
    from paper_2512_18345_gb300 import inputs
    q = P.q[:level]
    a = inputs.uniform_residues(g, q, P.N)
    e = inputs.gaussian(g, P.N)
    if not noise:
        e = np.zeros_like(e)
    m_ntt = ntt(to_rns(m_coeffs, q), q)
    e_ntt = ntt(to_rns(e, q), q)
    c0 = add(add(neg(mul(a, sk.ntt[:level], q), q), e_ntt, q), m_ntt, q)
    return np.stack([c0, a])


def decrypt(P: OracleParams, sk: SecretKey, ct: np.ndarray, level: int) -> List[int]:
    """c0 + c1 s mod Q_level, centered big-integer coefficients."""
    q = P.q[:level]
    m_ntt = add(ct[0], mul(ct[1], sk.ntt[:level], q), q)
    return crt(intt(m_ntt, q), q)


def phase_ntt(P: OracleParams, sk: SecretKey, ct: np.ndarray, level: int) -> np.ndarray:
    q = P.q[:level]
    return add(ct[0], mul(ct[1], sk.ntt[:level], q), q)
