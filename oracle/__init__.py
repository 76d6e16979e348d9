"""CPU oracle for the CKKS hybrid key-switching path (FIDESlib, arXiv 2507.04775).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the library.  The arithmetic
lives in ``fides_oracle.c`` (u128 ``%`` products, textbook transforms); this
module loads it with ctypes and adds the client side the paper leaves to
OpenFHE (Sec. III-A): CKKS encoding/decoding in FP64, CRT reconstruction with
Python integers, and a small key/ciphertext helper.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fides_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfides_oracle.so")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_intp = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over limbs)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.or_ctx_create.restype = ctypes.c_void_p
        L.or_ctx_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p]
        L.or_ctx_free.argtypes = [ctypes.c_void_p]
        L.or_ctx_psi.restype = ctypes.c_uint64
        L.or_ctx_psi.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_ctx_alpha.restype = ctypes.c_int
        L.or_ctx_alpha.argtypes = [ctypes.c_void_p]
        L.or_beta.restype = ctypes.c_int
        L.or_beta.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_set_threads.restype = ctypes.c_int
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_mul_mod.restype = ctypes.c_uint64
        L.or_mul_mod.argtypes = [ctypes.c_uint64] * 3
        L.or_pow_mod.restype = ctypes.c_uint64
        L.or_pow_mod.argtypes = [ctypes.c_uint64] * 3
        L.or_is_prime.restype = ctypes.c_int
        L.or_is_prime.argtypes = [ctypes.c_uint64]
        L.or_smallest_generator.restype = ctypes.c_uint64
        L.or_smallest_generator.argtypes = [ctypes.c_uint64]
        L.or_find_primes.restype = ctypes.c_int
        L.or_find_primes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_int, _u64p]
        for name in ("or_ntt_naive", "or_intt_naive"):
            getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_int, _u64p, _u64p]
        for name in ("or_ntt", "or_intt"):
            getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_int, _u64p]
        for name in ("or_ntt_limbs", "or_intt_limbs"):
            getattr(L, name).argtypes = [ctypes.c_void_p, _u64p, _intp, ctypes.c_int]
        L.or_bconv.argtypes = [ctypes.c_void_p, _u64p, _intp, ctypes.c_int, _u64p, _intp, ctypes.c_int]
        L.or_bconv_centred.argtypes = L.or_bconv.argtypes
        L.or_ctx_set_rounding.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_ctx_set_rounding.restype = None
        L.or_modup.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, _u64p]
        L.or_moddown.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, _u64p]
        L.or_keyswitch.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, _u64p, _u64p, _u64p]
        L.or_hmult.argtypes = [ctypes.c_void_p, _u64p, _u64p, ctypes.c_int, _u64p, _u64p]
        L.or_galois_elt.restype = ctypes.c_uint64
        L.or_galois_elt.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.or_automorph_coeff.argtypes = [ctypes.c_void_p, _u64p, _u64p, ctypes.c_int, _intp, ctypes.c_uint64]
        L.or_automorph_eval.argtypes = [ctypes.c_void_p, _u64p, _u64p, ctypes.c_int, ctypes.c_uint64]
        L.or_rotate.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, ctypes.c_int64, _u64p, _u64p]
        L.or_rescale.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, _u64p]
        L.or_rescale_round.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, _u64p]
        L.or_automorph_ct.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, ctypes.c_uint64, _u64p, _u64p]
        L.or_conjugate.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, _u64p, _u64p]
        L.or_rotate_hoisted.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, _u64p,
                                        _u64p]
        L.or_linear_transform.restype = ctypes.c_int
        L.or_linear_transform.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, ctypes.c_int, _intp, _u64p,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_void_p, _u64p, _u64p]
        L.or_modraise.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, _u64p]
        L.or_mul_monomial.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, ctypes.c_uint64, _u64p]
        for name in ("or_hadd", "or_hsub", "or_ptadd", "or_ptmult", "or_scalar_add", "or_scalar_mult"):
            getattr(L, name).argtypes = [ctypes.c_void_p, _u64p, _u64p, ctypes.c_int, _u64p]
        L.or_from_signed.argtypes = [ctypes.c_void_p, _i64p, _intp, ctypes.c_int, _u64p]
        L.or_keygen.argtypes = [ctypes.c_void_p, _u64p, _u64p, _u64p, _i64p, _u64p]
        L.or_encrypt.argtypes = [ctypes.c_void_p, ctypes.c_int, _i64p, _i64p, _u64p, _u64p, _u64p]
        L.or_decrypt.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int, _u64p, _u64p]
        L.or_pointwise_mul.argtypes = [ctypes.c_void_p, _u64p, _u64p, _intp, ctypes.c_int, _u64p]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.uint64:
        return a.ctypes.data_as(_u64p)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_i64p)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_intp)
    raise TypeError(a.dtype)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


# -- number theory ----------------------------------------------------------

def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (timing only); returns the count in effect."""
    return int(lib().or_set_threads(int(n)))


def is_prime(n: int) -> bool:
    return bool(lib().or_is_prime(n))


def mul_mod(a: int, b: int, q: int) -> int:
    return int(lib().or_mul_mod(a, b, q))


def smallest_generator(q: int) -> int:
    return int(lib().or_smallest_generator(q))


def find_primes(logN: int, bits: int, count: int, exclude=()) -> list[int]:
    ex = _u64(list(exclude) or [0])
    out = np.zeros(max(count, 1), dtype=np.uint64)
    n = lib().or_find_primes(logN, bits, count, _p(ex), len(exclude), _p(out))
    if n != count:
        raise ValueError("not enough primes")
    return [int(x) for x in out[:count]]


# -- context ----------------------------------------------------------------

class Context:
    """Oracle context: ``nq`` q-primes then ``nk`` special primes at ring
    degree N = 2^logN with ``dnum`` key-switching digits.  ``nearest`` selects
    the rounding of ModDown and Rescale (see ``set_rounding``)."""

    def __init__(self, logN: int, q_primes, p_primes, dnum: int, nearest: bool = False):
        self.logN = logN
        self.N = 1 << logN
        self.q = [int(x) for x in q_primes]
        self.p = [int(x) for x in p_primes]
        self.primes = self.q + self.p
        self.nq, self.nk, self.dnum = len(self.q), len(self.p), dnum
        arr = _u64(self.primes)
        h = lib().or_ctx_create(logN, self.nq, self.nk, dnum, _p(arr))
        if not h:
            raise ValueError("invalid oracle parameters")
        self._h = ctypes.c_void_p(h)
        self.alpha = lib().or_ctx_alpha(self._h)
        self.set_rounding(nearest)

    def set_rounding(self, nearest: bool):
        """Floor (False, the default) or round-to-nearest (True) for every
        ModDown (centred conversion of the special limbs) and Rescale (centred
        SwitchModulo)."""
        self.nearest = bool(nearest)
        lib().or_ctx_set_rounding(self._h, 1 if nearest else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_ctx_free(h)
            self._h = None

    # structure
    def psi(self, i: int) -> int:
        return int(lib().or_ctx_psi(self._h, i))

    def beta(self, nl: int) -> int:
        return int(lib().or_beta(self._h, nl))

    def ext_primes(self, nl: int) -> list[int]:
        return self.q[:nl] + self.p

    # transforms on one limb
    def ntt_naive(self, a, i: int) -> np.ndarray:
        a = _u64(a); out = np.empty_like(a)
        lib().or_ntt_naive(self._h, i, _p(a), _p(out)); return out

    def intt_naive(self, a, i: int) -> np.ndarray:
        a = _u64(a); out = np.empty_like(a)
        lib().or_intt_naive(self._h, i, _p(a), _p(out)); return out

    def ntt(self, a, i: int) -> np.ndarray:
        a = _u64(a).copy(); lib().or_ntt(self._h, i, _p(a)); return a

    def intt(self, a, i: int) -> np.ndarray:
        a = _u64(a).copy(); lib().or_intt(self._h, i, _p(a)); return a

    def ntt_limbs(self, a, pidx) -> np.ndarray:
        a = _u64(a).copy(); pi = _i32(pidx)
        lib().or_ntt_limbs(self._h, _p(a), _p(pi), len(pi)); return a

    def intt_limbs(self, a, pidx) -> np.ndarray:
        a = _u64(a).copy(); pi = _i32(pidx)
        lib().or_intt_limbs(self._h, _p(a), _p(pi), len(pi)); return a

    # key-switching steps
    def bconv(self, src, src_idx, dst_idx, centred: bool = False) -> np.ndarray:
        """Eq. 1 from canonical residues, or (centred) from the centred ones."""
        src = _u64(src); si = _i32(src_idx); di = _i32(dst_idx)
        out = np.empty((len(di), self.N), dtype=np.uint64)
        fn = lib().or_bconv_centred if centred else lib().or_bconv
        fn(self._h, _p(src), _p(si), len(si), _p(out), _p(di), len(di)); return out

    def modup(self, d) -> np.ndarray:
        d = _u64(d); nl = d.shape[0]
        out = np.empty((self.beta(nl), nl + self.nk, self.N), dtype=np.uint64)
        lib().or_modup(self._h, _p(d), nl, _p(out)); return out

    def moddown(self, x) -> np.ndarray:
        x = _u64(x); nl = x.shape[0] - self.nk
        out = np.empty((nl, self.N), dtype=np.uint64)
        lib().or_moddown(self._h, _p(x), nl, _p(out)); return out

    def keyswitch(self, d, evk):
        d = _u64(d); evk = _u64(evk); nl = d.shape[0]
        o0 = np.empty((nl, self.N), dtype=np.uint64); o1 = np.empty_like(o0)
        lib().or_keyswitch(self._h, _p(d), nl, _p(evk), _p(o0), _p(o1)); return o0, o1

    def hmult(self, a, b, rlk) -> np.ndarray:
        a = _u64(a); b = _u64(b); rlk = _u64(rlk); nl = a.shape[1]
        out = np.empty_like(a)
        lib().or_hmult(self._h, _p(a), _p(b), nl, _p(rlk), _p(out)); return out

    def galois_elt(self, steps: int) -> int:
        return int(lib().or_galois_elt(self._h, steps))

    def automorph_eval(self, a, g: int) -> np.ndarray:
        a = _u64(a); nl = a.shape[0]; out = np.empty_like(a)
        lib().or_automorph_eval(self._h, _p(a), _p(out), nl, g); return out

    def automorph_coeff(self, a, g: int, pidx=None) -> np.ndarray:
        a = _u64(a); nl = a.shape[0]; out = np.empty_like(a)
        pi = _i32(range(nl) if pidx is None else pidx)
        lib().or_automorph_coeff(self._h, _p(a), _p(out), nl, _p(pi), g); return out

    def rotate(self, a, steps: int, rk) -> np.ndarray:
        a = _u64(a); rk = _u64(rk); nl = a.shape[1]; out = np.empty_like(a)
        lib().or_rotate(self._h, _p(a), nl, steps, _p(rk), _p(out)); return out

    def conjugate(self, a, ck) -> np.ndarray:
        a = _u64(a); ck = _u64(ck); nl = a.shape[1]; out = np.empty_like(a)
        lib().or_conjugate(self._h, _p(a), nl, _p(ck), _p(out)); return out

    def rotate_hoisted(self, a, steps, rks) -> np.ndarray:
        """[n_rot][2][nl][N]: rotation by each steps[k] with key rks[k], one shared ModUp."""
        a = _u64(a); nl = a.shape[1]
        st = np.ascontiguousarray(steps, dtype=np.int64)
        keys = _u64(np.stack([_u64(k) for k in rks]))
        out = np.empty((len(st), 2, nl, self.N), dtype=np.uint64)
        lib().or_rotate_hoisted(self._h, _p(a), nl, len(st), st.ctypes.data, _p(keys), _p(out)); return out

    def linear_transform(self, a, diag_idx, pts, n1: int, keys: dict) -> np.ndarray:
        """BSGS diagonal-method linear transform: pts[k] is the plaintext of
        rot_{-n1 floor(i/n1)}(d_i) for i = diag_idx[k]; keys: {steps: key}."""
        a = _u64(a); nl = a.shape[1]
        di = _i32(diag_idx)
        p = _u64(np.stack([_u64(x) for x in pts]))
        ks = np.ascontiguousarray(list(keys), dtype=np.int64)
        kk = _u64(np.stack([_u64(keys[k]) for k in keys])) if keys else np.zeros(1, dtype=np.uint64)
        out = np.empty_like(a)
        rc = lib().or_linear_transform(self._h, _p(a), nl, len(di), _p(di), _p(p), n1, len(ks), ks.ctypes.data,
                                       _p(kk), _p(out))
        if rc != 0:
            raise KeyError("a rotation key of the transform is missing")
        return out

    def modraise(self, a, nl: int) -> np.ndarray:
        """[2][1][N] modulo q_0 -> [2][nl][N], centred lift."""
        a = _u64(a); out = np.empty((2, nl, self.N), dtype=np.uint64)
        lib().or_modraise(self._h, _p(a), nl, _p(out)); return out

    def mul_monomial(self, a, k: int) -> np.ndarray:
        a = _u64(a); nl = a.shape[1]; out = np.empty_like(a)
        lib().or_mul_monomial(self._h, _p(a), nl, k, _p(out)); return out

    def hsquare(self, a, rlk) -> np.ndarray:
        return self.hmult(a, a, rlk)

    def _ct_op(self, name, a, b):
        a = _u64(a); b = _u64(b); nl = a.shape[1]; out = np.empty_like(a)
        getattr(lib(), name)(self._h, _p(a), _p(b), nl, _p(out)); return out

    def hadd(self, a, b) -> np.ndarray:
        return self._ct_op("or_hadd", a, b)

    def hsub(self, a, b) -> np.ndarray:
        return self._ct_op("or_hsub", a, b)

    def ptadd(self, a, pt) -> np.ndarray:
        return self._ct_op("or_ptadd", a, pt)

    def ptmult(self, a, pt) -> np.ndarray:
        return self._ct_op("or_ptmult", a, pt)

    def scalar_add(self, a, k) -> np.ndarray:
        """k: the constant's residues, one per limb of a."""
        return self._ct_op("or_scalar_add", a, k)

    def scalar_mult(self, a, k) -> np.ndarray:
        return self._ct_op("or_scalar_mult", a, k)

    def rescale(self, a, nearest: bool | None = None) -> np.ndarray:
        """Rescale by the last prime: floor(x / q_l), or round(x / q_l) with
        nearest (default: the context's rounding)."""
        if nearest is None:
            nearest = self.nearest
        a = _u64(a); nl = a.shape[1]
        out = np.empty((2, nl - 1, self.N), dtype=np.uint64)
        fn = lib().or_rescale_round if nearest else lib().or_rescale
        fn(self._h, _p(a), nl, _p(out)); return out

    # client side
    def from_signed(self, v, pidx) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.int64); pi = _i32(pidx)
        out = np.empty((len(pi), self.N), dtype=np.uint64)
        lib().or_from_signed(self._h, _p(v), _p(pi), len(pi), _p(out)); return out

    def pointwise_mul(self, a, b, pidx) -> np.ndarray:
        a = _u64(a); b = _u64(b); pi = _i32(pidx); out = np.empty_like(a)
        lib().or_pointwise_mul(self._h, _p(a), _p(b), _p(pi), len(pi), _p(out)); return out

    def to_eval_full(self, v) -> np.ndarray:
        """signed coefficients -> evaluation form under every prime"""
        idx = list(range(len(self.primes)))
        return self.ntt_limbs(self.from_signed(v, idx), idx)

    def keygen(self, s_eval, sp_eval, a, e) -> np.ndarray:
        s_eval = _u64(s_eval); sp_eval = _u64(sp_eval); a = _u64(a)
        e = np.ascontiguousarray(e, dtype=np.int64)
        out = np.empty((self.dnum, 2, len(self.primes), self.N), dtype=np.uint64)
        lib().or_keygen(self._h, _p(s_eval), _p(sp_eval), _p(a), _p(e), _p(out)); return out

    def encrypt(self, m, e, a, s_eval) -> np.ndarray:
        m = np.ascontiguousarray(m, dtype=np.int64); e = np.ascontiguousarray(e, dtype=np.int64)
        a = _u64(a); s_eval = _u64(s_eval); nl = a.shape[0]
        out = np.empty((2, nl, self.N), dtype=np.uint64)
        lib().or_encrypt(self._h, nl, _p(m), _p(e), _p(a), _p(s_eval), _p(out)); return out

    def decrypt_residues(self, ct, s_eval) -> np.ndarray:
        ct = _u64(ct); s_eval = _u64(s_eval); nl = ct.shape[1]
        out = np.empty((nl, self.N), dtype=np.uint64)
        lib().or_decrypt(self._h, _p(ct), nl, _p(s_eval), _p(out)); return out


# -- CRT with Python integers (RNS, Sec. II) ---------------------------------

def crt(residues: np.ndarray, primes) -> list[int]:
    """x in [0, prod primes) from its residues (limb-major [n][N])."""
    primes = [int(p) for p in primes]
    Q = 1
    for p in primes:
        Q *= p
    coef = []
    for p in primes:
        Qi = Q // p
        coef.append(Qi * pow(Qi % p, -1, p))
    N = residues.shape[1]
    cols = [residues[i].tolist() for i in range(len(primes))]
    out = [0] * N
    for i, c in enumerate(coef):
        col = cols[i]
        for n in range(N):
            out[n] += col[n] * c
    return [x % Q for x in out]


def centered(xs, Q: int) -> list[int]:
    half = Q // 2
    return [x - Q if x > half else x for x in xs]


# -- CKKS encoding (canonical embedding, FP64) -------------------------------

def _slot_exponents(N: int, n: int) -> np.ndarray:
    """5^j mod 2N for j < n (slot j <-> root zeta^(5^j), zeta = exp(i pi / N))."""
    e = np.empty(n, dtype=np.int64)
    x = 1
    for j in range(n):
        e[j] = x
        x = (x * 5) % (2 * N)
    return e


def encode_direct(z: np.ndarray, N: int, scale: float) -> np.ndarray:
    """Coefficients of m with m(zeta^(5^j)) = scale z_j and m(conj) = conj,
    i.e. m_i = (2/N) Re sum_j w_j zeta^(-5^j i), by direct O(N n) sums;
    rounded half away from zero to int64 (full packing, n = N/2 slots)."""
    n = z.size
    if n != N // 2:
        raise ValueError("encode_direct expects N/2 slots")
    ex = _slot_exponents(N, n)
    w = z * scale
    ang = -np.pi * np.outer(ex, np.arange(N)) / N
    m = (2.0 / N) * np.real(w @ np.exp(1j * ang))
    return (np.sign(m) * np.floor(np.abs(m) + 0.5)).astype(np.int64)


def encode(z: np.ndarray, N: int, scale: float) -> np.ndarray:
    """Same as ``encode_direct`` through one length-N FFT:
    m_i = (1/N) Re( e^(-i pi i / N) FFT(u)_i ) with u_k = value at odd 2k+1."""
    n = z.size
    if n != N // 2:
        raise ValueError("encode expects N/2 slots")
    ex = _slot_exponents(N, n)
    u = np.zeros(N, dtype=np.complex128)
    w = z * scale
    u[(ex - 1) // 2] = w
    u[((2 * N - ex) - 1) // 2] = np.conj(w)
    m = np.real(np.exp(-1j * np.pi * np.arange(N) / N) * np.fft.fft(u)) / N
    m = np.sign(m) * np.floor(np.abs(m) + 0.5)
    return m.astype(np.int64)


def decode(coeffs, N: int, scale: float) -> np.ndarray:
    """Slots z_j = m(zeta^(5^j)) / scale from (centred, integer) coefficients."""
    m = np.array([float(x) for x in coeffs], dtype=np.float64) / scale
    vals = np.fft.ifft(m * np.exp(1j * np.pi * np.arange(N) / N)) * N   # value at 2k+1
    ex = _slot_exponents(N, N // 2)
    return vals[(ex - 1) // 2]


def decode_direct(coeffs, N: int, scale: float) -> np.ndarray:
    m = np.array([float(x) for x in coeffs], dtype=np.float64) / scale
    ex = _slot_exponents(N, N // 2)
    ang = np.pi * np.outer(ex, np.arange(N)) / N
    return np.exp(1j * ang) @ m
