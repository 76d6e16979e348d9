"""Python binding of the C ABI in ``include/fides.h`` (argument marshalling only).

Every step of the computation runs in the CUDA library ``_build/libfides.so``;
this module converts torch tensors to device pointers, passes the current torch
stream, and turns negative return codes into exceptions.  There is no CPU
fallback: if the library is missing, every call raises.

Buffers are torch tensors on the context's device, contiguous, of dtype
``torch.int64`` or ``torch.uint64`` (the bits are the u64 residues).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfides.so")

FIDES_OK = 0
ERRORS = {-1: "FIDES_ERR_ARG", -2: "FIDES_ERR_UNSUPPORTED", -3: "FIDES_ERR_NOMEM", -4: "FIDES_ERR_CUDA",
          -5: "FIDES_ERR_TIMEOUT", -6: "FIDES_ERR_PRIME", -7: "FIDES_ERR_KEY", -8: "FIDES_ERR_BUSY",
          -9: "FIDES_ERR_CANCELLED"}
ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_KEY, ERR_BUSY, ERR_CANCELLED = -1, -3, -4, -5, -7, -8, -9

EXPORTS = ["fides_last_error", "fides_version", "fides_find_primes", "fides_ctx_create", "fides_ctx_destroy",
           "fides_ctx_beta", "fides_ctx_psi", "fides_galois_elt", "fides_ntt", "fides_intt", "fides_modup",
           "fides_moddown", "fides_keyswitch", "fides_hmult", "fides_rotate", "fides_rescale",
           "fides_trace_enable", "fides_trace_reset", "fides_trace_read", "fides_kernel_launches",
           "fides_rescale_noalloc", "fides_measure_modmul_peak", "fides_batch_create", "fides_batch_run",
           "fides_batch_capture", "fides_batch_info", "fides_batch_destroy", "fides_ctx_autotune",
           "fides_ctx_ntt_tile", "fides_server_create", "fides_server_destroy", "fides_server_set_relin_key",
           "fides_server_add_rotation_key", "fides_server_submit", "fides_server_poll", "fides_server_release",
           "fides_server_cancel", "fides_server_pause", "fides_server_inject", "fides_server_stats_read",
           "fides_now_ns", "fides_hsquare", "fides_conjugate", "fides_rotate_hoisted", "fides_hadd", "fides_hsub",
           "fides_ptadd", "fides_ptmult", "fides_scalar_add", "fides_scalar_mult", "fides_linear_transform",
           "fides_linear_transform_work_words", "fides_modraise", "fides_mul_i", "fides_program_create",
           "fides_program_info", "fides_program_run", "fides_program_destroy", "fides_ctx_tune_table",
           "fides_ctx_status", "fides_ctx_tensor_bconv", "fides_ctx_selftest_wait", "fides_hmult_rescale",
           "fides_rescale_round", "fides_key_register", "fides_key_destroy", "fides_key_galois",
           "fides_batch_configure", "fides_batch_autotune", "fides_batch_tuning", "fides_ctx_set_rounding",
           "fides_ctx_rounding", "fides_ctx_add_stream", "fides_ctx_selftest_conversion"]

OP_HMULT, OP_ROTATE, OP_RESCALE = 1, 2, 3
ROUND_FLOOR, ROUND_NEAREST = 0, 1
FAULT_LAUNCH_ERROR, FAULT_STALL = 1, 2
STATUS_WAIT_TIMEOUT = 1      # fides_ctx_status bit: a bounded device wait ran out


class FidesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "FIDES_ERR"), code, msg))
        self.code = code


class fides_trace_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


class fides_ct(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n_limbs", ctypes.c_int), ("scale", ctypes.c_double)]


class fides_op(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("stage", ctypes.c_int), ("a", fides_ct), ("b", fides_ct),
                ("out", fides_ct), ("key", ctypes.c_void_p), ("steps", ctypes.c_int64)]


class fides_server_config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("n_lanes", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("max_pending", ctypes.c_int), ("timeout_us", ctypes.c_int64), ("simulate", ctypes.c_int),
                ("sim_ns_per_limb", ctypes.c_int64), ("logN", ctypes.c_int), ("L", ctypes.c_int),
                ("K", ctypes.c_int), ("dnum", ctypes.c_int)]


class fides_request(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("a", fides_ct), ("b", fides_ct), ("steps", ctypes.c_int64),
                ("tag", ctypes.c_uint64)]


class fides_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("type", ctypes.c_int), ("status", ctypes.c_int),
                ("out", fides_ct), ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_launch_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64), ("group_ops", ctypes.c_int),
                ("lane", ctypes.c_int)]


class fides_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "rejected", "cancelled", "completed", "failed", "timed_out", "groups", "grouped_ops",
        "max_group", "pending", "in_flight", "held", "arena_bytes", "arena_used", "arena_peak",
        "admission_stalls", "kernel_launches")] + [("device_ms", ctypes.c_double), ("max_lanes_busy", ctypes.c_int)]


class fides_instr(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("dst", ctypes.c_int), ("a", ctypes.c_int), ("b", ctypes.c_int),
                ("arg", ctypes.c_int)]


class fides_lt(ctypes.Structure):
    _fields_ = [("n_diag", ctypes.c_int), ("diag_idx", ctypes.POINTER(ctypes.c_int)),
                ("dev_pts", ctypes.POINTER(ctypes.c_void_p)), ("n1", ctypes.c_int), ("pt_scale", ctypes.c_double)]


class fides_program_desc(ctypes.Structure):
    _fields_ = [("n_instr", ctypes.c_int), ("instr", ctypes.POINTER(fides_instr)), ("n_regs", ctypes.c_int),
                ("in_reg", ctypes.c_int), ("out_reg", ctypes.c_int), ("in_limbs", ctypes.c_int),
                ("out_scale", ctypes.c_double), ("n_lt", ctypes.c_int), ("lt", ctypes.POINTER(fides_lt)),
                ("n_const", ctypes.c_int), ("consts", ctypes.POINTER(ctypes.c_void_p)),
                ("const_scale", ctypes.POINTER(ctypes.c_double)), ("relin_key", ctypes.c_void_p),
                ("conj_key", ctypes.c_void_p), ("n_rot_keys", ctypes.c_int),
                ("rot_keys", ctypes.POINTER(ctypes.c_void_p)),
                ("n_lin", ctypes.c_int), ("lin_start", ctypes.POINTER(ctypes.c_int)),
                ("lin_reg", ctypes.POINTER(ctypes.c_int)), ("lin_const", ctypes.POINTER(ctypes.c_int))]


_lib = None
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p
_i = ctypes.c_int


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfides.so is missing (%s); build it with __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.fides_last_error.restype = ctypes.c_char_p
        L.fides_version.restype = ctypes.c_char_p
        L.fides_find_primes.argtypes = [_i, _i, _i, _u64p, _i, _u64p]
        L.fides_ctx_create.argtypes = [_i, _i, _i, _u64p, _i, ctypes.POINTER(_vp)]
        L.fides_ctx_destroy.argtypes = [_vp]
        L.fides_ctx_destroy.restype = None
        L.fides_ctx_beta.argtypes = [_vp, _i]
        L.fides_ctx_psi.argtypes = [_vp, _i]
        L.fides_ctx_psi.restype = ctypes.c_uint64
        L.fides_galois_elt.argtypes = [_vp, ctypes.c_int64]
        L.fides_galois_elt.restype = ctypes.c_uint64
        for name in ("fides_ntt", "fides_intt"):
            getattr(L, name).argtypes = [_vp, _vp, _i, _i, _i, _vp]
        L.fides_modup.argtypes = [_vp, _vp, _i, _vp, _vp]
        L.fides_moddown.argtypes = [_vp, _vp, _i, _vp, _vp]
        L.fides_keyswitch.argtypes = [_vp, _vp, _i, _vp, _vp, _vp, _vp]
        L.fides_key_register.argtypes = [_vp, _vp, ctypes.c_uint64, ctypes.POINTER(_vp)]
        L.fides_key_destroy.argtypes = [_vp]
        L.fides_key_destroy.restype = None
        L.fides_key_galois.argtypes = [_vp]
        L.fides_key_galois.restype = ctypes.c_uint64
        ctp = ctypes.POINTER(fides_ct)
        L.fides_hmult.argtypes = [_vp, ctp, ctp, _vp, ctp, _vp]
        L.fides_hmult_rescale.argtypes = [_vp, ctp, ctp, _vp, ctp, _vp]
        L.fides_rotate.argtypes = [_vp, ctp, ctypes.c_int64, _vp, ctp, _vp]
        L.fides_rescale.argtypes = [_vp, ctp, ctp, _vp]
        L.fides_rescale_round.argtypes = [_vp, ctp, ctp, _vp]
        L.fides_rescale_noalloc.argtypes = [_vp, ctp, ctp, _vp]
        L.fides_trace_enable.argtypes = [_i]
        L.fides_trace_reset.restype = None
        L.fides_trace_read.argtypes = [ctypes.POINTER(fides_trace_stat), _i, ctypes.POINTER(_i)]
        L.fides_kernel_launches.restype = ctypes.c_uint64
        L.fides_ctx_autotune.argtypes = [_vp, _i, _vp]
        L.fides_ctx_status.argtypes = [_vp, ctypes.POINTER(_i)]
        L.fides_ctx_tensor_bconv.argtypes = [_vp]
        L.fides_ctx_set_rounding.argtypes = [_vp, _i]
        L.fides_ctx_add_stream.argtypes = [_vp, _vp]
        L.fides_ctx_selftest_conversion.argtypes = [_vp, _i, _vp]
        L.fides_ctx_rounding.argtypes = [_vp]
        L.fides_ctx_selftest_wait.argtypes = [_vp, _i, _vp]
        L.fides_ctx_ntt_tile.argtypes = [_vp, _i, _i]
        L.fides_batch_create.argtypes = [_vp, ctypes.POINTER(fides_op), _i, ctypes.POINTER(_vp)]
        L.fides_batch_run.argtypes = [_vp, _vp]
        L.fides_batch_capture.argtypes = [_vp, _vp]
        L.fides_batch_info.argtypes = [_vp, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t)]
        L.fides_batch_destroy.argtypes = [_vp]
        L.fides_batch_destroy.restype = None
        L.fides_batch_configure.argtypes = [_vp, _i, _i, _i]
        L.fides_batch_autotune.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_double)]
        L.fides_batch_tuning.argtypes = [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                                         ctypes.POINTER(_i)]
        L.fides_measure_modmul_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.fides_server_create.argtypes = [_vp, ctypes.POINTER(fides_server_config), ctypes.POINTER(_vp)]
        L.fides_server_destroy.argtypes = [_vp]
        L.fides_server_destroy.restype = None
        L.fides_server_set_relin_key.argtypes = [_vp, _vp]
        L.fides_server_add_rotation_key.argtypes = [_vp, ctypes.c_int64, _vp]
        L.fides_server_submit.argtypes = [_vp, ctypes.POINTER(fides_request), ctypes.POINTER(ctypes.c_uint64)]
        L.fides_server_poll.argtypes = [_vp, ctypes.POINTER(fides_completion), _i, ctypes.c_int64, ctypes.POINTER(_i)]
        L.fides_server_release.argtypes = [_vp, ctypes.c_uint64]
        L.fides_server_cancel.argtypes = [_vp, ctypes.c_uint64]
        L.fides_server_pause.argtypes = [_vp, _i]
        L.fides_server_inject.argtypes = [_vp, _i, ctypes.c_int64]
        L.fides_server_stats_read.argtypes = [_vp, ctypes.POINTER(fides_server_stats)]
        L.fides_now_ns.restype = ctypes.c_int64
        L.fides_hsquare.argtypes = [_vp, ctp, _vp, ctp, _vp]
        L.fides_conjugate.argtypes = [_vp, ctp, _vp, ctp, _vp]
        L.fides_rotate_hoisted.argtypes = [_vp, ctp, _i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_vp), ctp, _vp]
        L.fides_hadd.argtypes = [_vp, ctp, ctp, ctp, _vp]
        L.fides_hsub.argtypes = [_vp, ctp, ctp, ctp, _vp]
        L.fides_ptadd.argtypes = [_vp, ctp, _vp, ctp, _vp]
        L.fides_ptmult.argtypes = [_vp, ctp, _vp, ctypes.c_double, ctp, _vp]
        L.fides_scalar_add.argtypes = [_vp, ctp, _u64p, ctp, _vp]
        L.fides_scalar_mult.argtypes = [_vp, ctp, _u64p, ctypes.c_double, ctp, _vp]
        L.fides_linear_transform_work_words.argtypes = [_vp, _i, _i, ctypes.POINTER(_i), _i,
                                                        ctypes.POINTER(ctypes.c_size_t)]
        L.fides_linear_transform.argtypes = [_vp, ctp, _i, ctypes.POINTER(_i), ctypes.POINTER(_vp), ctypes.c_double,
                                             _i, _i, ctypes.POINTER(_vp), _vp, ctypes.c_size_t, ctp, _vp]
        L.fides_modraise.argtypes = [_vp, ctp, ctp, _vp]
        L.fides_mul_i.argtypes = [_vp, ctp, _i, ctp, _vp]
        L.fides_program_create.argtypes = [_vp, ctypes.POINTER(fides_program_desc), ctypes.POINTER(_vp)]
        L.fides_program_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_i), ctypes.POINTER(_i)]
        L.fides_program_run.argtypes = [_vp, ctp, ctp, _vp, ctypes.c_size_t, _vp]
        L.fides_program_destroy.argtypes = [_vp]
        L.fides_program_destroy.restype = None
        L.fides_ctx_tune_table.argtypes = [_vp, ctypes.c_char_p, _i]
        _lib = L
    return _lib


def _check(rc: int):
    if rc != FIDES_OK:
        raise FidesError(rc, lib().fides_last_error().decode())


def version() -> str:
    return lib().fides_version().decode()


def trace_enable(on: bool = True):
    """Bracket every kernel launch and public operation with CUDA events."""
    _check(lib().fides_trace_enable(1 if on else 0))


def trace_reset():
    lib().fides_trace_reset()


def trace_read() -> dict:
    """{name: (launches, total_ms)} for everything traced since the last reset."""
    n = ctypes.c_int(0)
    _check(lib().fides_trace_read(None, 0, ctypes.byref(n)))
    buf = (fides_trace_stat * max(1, n.value))()
    _check(lib().fides_trace_read(buf, n.value, ctypes.byref(n)))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(n.value)}


def measure_modmul_peak() -> float:
    """Sustained 10^9 Shoup products per second of the current device."""
    g, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().fides_measure_modmul_peak(ctypes.byref(g), ctypes.byref(ms)))
    return g.value


def kernel_launches() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(lib().fides_kernel_launches())


def find_primes(logN: int, bits: int, count: int, exclude=()) -> list[int]:
    ex = np.ascontiguousarray(list(exclude) or [0], dtype=np.uint64)
    out = np.zeros(max(count, 1), dtype=np.uint64)
    _check(lib().fides_find_primes(logN, bits, count, ex.ctypes.data_as(_u64p), len(exclude),
                                   out.ctypes.data_as(_u64p)))
    return [int(x) for x in out[:count]]


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, words: int | None = None, name: str = "buffer"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype not in (torch.int64, torch.uint64):
        raise TypeError("%s must be int64/uint64" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if words is not None and t.numel() < words:
        raise ValueError("%s holds %d words, needs %d" % (name, t.numel(), words))
    return ctypes.c_void_p(t.data_ptr())


def to_device(a: np.ndarray, device="cuda"):
    """uint64 numpy array -> int64 CUDA tensor with the same bits."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


def to_host(t) -> np.ndarray:
    """CUDA tensor -> uint64 numpy array with the same bits."""
    return t.detach().cpu().contiguous().numpy().view(np.uint64)


class Context:
    """A library context (``fides_ctx``) on the current CUDA device."""

    def __init__(self, logN: int, q_primes, p_primes, dnum: int):
        self.logN, self.N = logN, 1 << logN
        self.q = [int(x) for x in q_primes]
        self.p = [int(x) for x in p_primes]
        self.L, self.K, self.dnum = len(self.q), len(self.p), dnum
        self.alpha = -(-self.L // dnum)
        arr = np.ascontiguousarray(self.q + self.p, dtype=np.uint64)
        h = ctypes.c_void_p()
        _check(lib().fides_ctx_create(logN, self.L, dnum, arr.ctypes.data_as(_u64p), self.K, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fides_ctx_destroy(self._h)
            self._h = None

    __del__ = close

    # -- structure ---------------------------------------------------------
    def beta(self, n_limbs: int) -> int:
        return lib().fides_ctx_beta(self._h, n_limbs)

    def status(self) -> int:
        """Device status bits since the last call (STATUS_WAIT_TIMEOUT: a
        bounded wait of a tensor-core conversion ran out); clears them."""
        f = _i(0)
        _check(lib().fides_ctx_status(self._h, ctypes.byref(f)))
        return f.value

    def selftest_wait(self, limit_us: int = 1000, stream=None):
        """Runs a device wait that nothing completes, limited to limit_us; it
        sets STATUS_WAIT_TIMEOUT in the status word (see status())."""
        _check(lib().fides_ctx_selftest_wait(self._h, limit_us, _stream(stream)))

    def selftest_conversion(self, limit_us: int = 5000, stream=None):
        """Runs the top-level ModUp conversion with one CTA whose first tile
        never arrives and every wait limited to limit_us; that CTA gives up,
        sets STATUS_WAIT_TIMEOUT and frees its tensor memory
        (fides_ctx_selftest_conversion)."""
        _check(lib().fides_ctx_selftest_conversion(self._h, limit_us, _stream(stream)))

    def add_stream(self, stream):
        """Give `stream` (a torch.cuda.Stream; default the current stream) its
        own scratch pool, so single-operation calls on it may overlap calls on
        other streams of this context (fides_ctx_add_stream)."""
        _check(lib().fides_ctx_add_stream(self._h, _stream(stream)))

    def set_rounding(self, nearest: bool):
        """Floor (False, the default) or round-to-nearest (True) for every
        ModDown and Rescale of this context (fides_ctx_set_rounding)."""
        _check(lib().fides_ctx_set_rounding(self._h, ROUND_NEAREST if nearest else ROUND_FLOOR))

    @property
    def nearest(self) -> bool:
        return lib().fides_ctx_rounding(self._h) == ROUND_NEAREST

    @property
    def tensor_bconv(self) -> bool:
        """Whether base conversions run on the tensor cores."""
        return bool(lib().fides_ctx_tensor_bconv(self._h))

    def psi(self, i: int) -> int:
        return int(lib().fides_ctx_psi(self._h, i))

    def galois_elt(self, steps: int) -> int:
        return int(lib().fides_galois_elt(self._h, steps))

    def autotune(self, max_limbs: int = 128, stream=None, cache: str | None = None):
        """Time the NTT tile variants per pass and limb count; keep the fastest.
        With `cache`, a table tuned earlier for the same device and parameters
        is loaded from that JSON file instead, and a new one is saved there."""
        key = None
        if cache:
            import json
            import torch
            key = {"device": torch.cuda.get_device_name(), "logN": self.logN, "L": self.L, "K": self.K,
                   "library": version()}
            try:
                entry = json.load(open(cache))
                if entry.get("key") == key:
                    self.set_tune_table(bytes(entry["table"]))
                    return
            except (OSError, ValueError, KeyError, TypeError, FidesError):
                pass
        _check(lib().fides_ctx_autotune(self._h, max_limbs, _stream(stream)))
        if cache:
            import json
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump({"key": key, "table": list(self.tune_table())}, f)
            os.replace(tmp, cache)

    def tune_table(self) -> bytes:
        buf = ctypes.create_string_buffer(4 * 129)
        _check(lib().fides_ctx_tune_table(self._h, buf, 0))
        return buf.raw

    def set_tune_table(self, table: bytes):
        if len(table) != 4 * 129:
            raise ValueError("a tune table has %d entries" % (4 * 129))
        _check(lib().fides_ctx_tune_table(self._h, ctypes.create_string_buffer(bytes(table), 4 * 129), 1))

    def ntt_tile(self, pass_kind: int, n_limbs: int) -> int:
        """Tile width chosen for pass 0..3 (fwd cols, fwd rows, inv rows, inv cols)."""
        return int(lib().fides_ctx_ntt_tile(self._h, pass_kind, n_limbs))

    # -- primitives --------------------------------------------------------
    def ntt(self, t, first_prime: int, n_limbs: int, batch: int = 1, stream=None):
        _check(lib().fides_ntt(self._h, _ptr(t, batch * n_limbs * self.N), first_prime, n_limbs, batch,
                               _stream(stream)))

    def intt(self, t, first_prime: int, n_limbs: int, batch: int = 1, stream=None):
        _check(lib().fides_intt(self._h, _ptr(t, batch * n_limbs * self.N), first_prime, n_limbs, batch,
                                _stream(stream)))

    def modup(self, d, n_limbs: int, ext, stream=None):
        ne = n_limbs + self.K
        _check(lib().fides_modup(self._h, _ptr(d, n_limbs * self.N, "d"), n_limbs,
                                 _ptr(ext, self.beta(n_limbs) * ne * self.N, "ext"), _stream(stream)))

    def moddown(self, x, n_limbs: int, out, stream=None):
        _check(lib().fides_moddown(self._h, _ptr(x, (n_limbs + self.K) * self.N, "x"), n_limbs,
                                   _ptr(out, n_limbs * self.N, "out"), _stream(stream)))

    def keyswitch(self, d, n_limbs: int, evk: "Key", out0, out1, stream=None):
        w = n_limbs * self.N
        _check(lib().fides_keyswitch(self._h, _ptr(d, w, "d"), n_limbs, _key(evk),
                                     _ptr(out0, w, "out0"), _ptr(out1, w, "out1"), _stream(stream)))

    def key_words(self) -> int:
        return self.dnum * 2 * (self.L + self.K) * self.N

    # -- switching keys ------------------------------------------------------
    def register_key(self, t, galois: int) -> "Key":
        """Binds the key buffer t ([dnum][2][L+K][N]) to Galois element `galois`
        (0: relinearisation); fides_key_register."""
        return Key(self, t, galois)

    def relin_key(self, t) -> "Key":
        return Key(self, t, 0)

    def rotation_key(self, t, steps: int) -> "Key":
        return Key(self, t, self.galois_elt(steps))

    def conjugation_key(self, t) -> "Key":
        return Key(self, t, 2 * self.N - 1)

    # -- ciphertext operations ---------------------------------------------
    def _ct(self, t, n_limbs: int, scale: float, name: str):
        return fides_ct(_ptr(t, 2 * n_limbs * self.N, name).value, n_limbs, scale)

    def hmult(self, a, b, n_limbs: int, rlk, out, scale_a: float = 1.0, scale_b: float = 1.0, stream=None) -> float:
        ca, cb = self._ct(a, n_limbs, scale_a, "a"), self._ct(b, n_limbs, scale_b, "b")
        co = self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_hmult(self._h, ctypes.byref(ca), ctypes.byref(cb), _key(rlk), ctypes.byref(co),
                                 _stream(stream)))
        return co.scale

    def hmult_rescale(self, a, b, n_limbs: int, rlk, out, scale_a: float = 1.0, scale_b: float = 1.0,
                      stream=None) -> float:
        """Rescale(HMult(a, b)) in one key switch; out has n_limbs - 1 limbs."""
        ca, cb = self._ct(a, n_limbs, scale_a, "a"), self._ct(b, n_limbs, scale_b, "b")
        co = self._ct(out, n_limbs - 1, 0.0, "out")
        _check(lib().fides_hmult_rescale(self._h, ctypes.byref(ca), ctypes.byref(cb), _key(rlk), ctypes.byref(co),
                                         _stream(stream)))
        return co.scale

    def rotate(self, a, n_limbs: int, steps: int, rk, out, scale: float = 1.0, stream=None) -> float:
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_rotate(self._h, ctypes.byref(ca), steps, _key(rk), ctypes.byref(co), _stream(stream)))
        return co.scale

    def rescale(self, a, n_limbs: int, out, scale: float = 1.0, stream=None, nearest: bool = False) -> float:
        """floor(x / q_l) limb-wise, or round(x / q_l) with nearest (fides_rescale_round)."""
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs - 1, 0.0, "out")
        fn = lib().fides_rescale_round if nearest else lib().fides_rescale
        _check(fn(self._h, ctypes.byref(ca), ctypes.byref(co), _stream(stream)))
        return co.scale

    def hsquare(self, a, n_limbs: int, rlk, out, scale: float = 1.0, stream=None) -> float:
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_hsquare(self._h, ctypes.byref(ca), _key(rlk), ctypes.byref(co), _stream(stream)))
        return co.scale

    def conjugate(self, a, n_limbs: int, ck, out, scale: float = 1.0, stream=None) -> float:
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_conjugate(self._h, ctypes.byref(ca), _key(ck), ctypes.byref(co), _stream(stream)))
        return co.scale

    def rotate_hoisted(self, a, n_limbs: int, steps, rks, outs, scale: float = 1.0, stream=None):
        """Rotations of `a` by every steps[k] (key rks[k], output outs[k]) sharing one ModUp."""
        n = len(steps)
        if len(rks) != n or len(outs) != n:
            raise ValueError("steps, rks and outs must have the same length")
        ca = self._ct(a, n_limbs, scale, "a")
        st = (ctypes.c_int64 * n)(*steps)
        keys = (_vp * n)(*[_key(k) for k in rks])
        cts = (fides_ct * n)(*[self._ct(o, n_limbs, 0.0, "out") for o in outs])
        _check(lib().fides_rotate_hoisted(self._h, ctypes.byref(ca), n, st, keys, cts, _stream(stream)))

    def linear_transform(self, a, n_limbs: int, diag_idx, pts, n1: int, keys, out, scale: float = 1.0,
                         pt_scale: float = 1.0, work=None, stream=None) -> float:
        """BSGS diagonal-method transform (fides_linear_transform); pts[k] is
        the device plaintext of diagonal diag_idx[k], pre-rotated; keys are
        rotation Keys (a list, or a dict whose values are used), found by
        their Galois elements."""
        n = len(diag_idx)
        di = (_i * n)(*diag_idx)
        words = ctypes.c_size_t(0)
        _check(lib().fides_linear_transform_work_words(self._h, n_limbs, n, di, n1, ctypes.byref(words)))
        if work is None:
            import torch
            work = torch.empty(max(1, words.value), dtype=torch.int64, device="cuda")
        pp = (_vp * n)(*[_ptr(p, n_limbs * self.N, "pt").value for p in pts])
        ks = list(keys.values()) if isinstance(keys, dict) else list(keys)
        kp = (_vp * max(1, len(ks)))(*[_key(k) for k in ks])
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_linear_transform(self._h, ctypes.byref(ca), n, di, pp, pt_scale, n1, len(ks), kp,
                                            _ptr(work, words.value, "work"), work.numel(), ctypes.byref(co),
                                            _stream(stream)))
        return co.scale

    def modraise(self, a, out, n_limbs: int, scale: float = 1.0, stream=None) -> float:
        """ModRaise of a one-limb ciphertext to n_limbs limbs."""
        ca, co = self._ct(a, 1, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_modraise(self._h, ctypes.byref(ca), ctypes.byref(co), _stream(stream)))
        return co.scale

    def mul_i(self, a, n_limbs: int, out, sign: int = 1, scale: float = 1.0, stream=None) -> float:
        """Slots times i (sign=+1) or -i (sign=-1), exactly."""
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_mul_i(self._h, ctypes.byref(ca), sign, ctypes.byref(co), _stream(stream)))
        return co.scale

    def _ct2(self, fn, a, b, n_limbs, out, scale, stream):
        ca, cb = self._ct(a, n_limbs, scale, "a"), self._ct(b, n_limbs, scale, "b")
        co = self._ct(out, n_limbs, 0.0, "out")
        _check(fn(self._h, ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(co), _stream(stream)))
        return co.scale

    def hadd(self, a, b, n_limbs: int, out, scale: float = 1.0, stream=None) -> float:
        return self._ct2(lib().fides_hadd, a, b, n_limbs, out, scale, stream)

    def hsub(self, a, b, n_limbs: int, out, scale: float = 1.0, stream=None) -> float:
        return self._ct2(lib().fides_hsub, a, b, n_limbs, out, scale, stream)

    def ptadd(self, a, pt, n_limbs: int, out, scale: float = 1.0, stream=None) -> float:
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_ptadd(self._h, ctypes.byref(ca), _ptr(pt, n_limbs * self.N, "pt"), ctypes.byref(co),
                                 _stream(stream)))
        return co.scale

    def ptmult(self, a, pt, n_limbs: int, out, scale: float = 1.0, pt_scale: float = 1.0, stream=None) -> float:
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_ptmult(self._h, ctypes.byref(ca), _ptr(pt, n_limbs * self.N, "pt"), pt_scale,
                                  ctypes.byref(co), _stream(stream)))
        return co.scale

    def _consts(self, k, n_limbs):
        if isinstance(k, int):
            k = [k % q for q in self.q[:n_limbs]]
        arr = np.ascontiguousarray(k, dtype=np.uint64)
        if arr.size < n_limbs:
            raise ValueError("constant needs %d residues" % n_limbs)
        return arr

    def scalar_add(self, a, k, n_limbs: int, out, scale: float = 1.0, stream=None) -> float:
        """k: a Python int (reduced modulo each q_i) or its residues per limb."""
        arr = self._consts(k, n_limbs)
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_scalar_add(self._h, ctypes.byref(ca), arr.ctypes.data_as(_u64p), ctypes.byref(co),
                                      _stream(stream)))
        return co.scale

    def scalar_mult(self, a, k, n_limbs: int, out, scale: float = 1.0, k_scale: float = 1.0, stream=None) -> float:
        arr = self._consts(k, n_limbs)
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs, 0.0, "out")
        _check(lib().fides_scalar_mult(self._h, ctypes.byref(ca), arr.ctypes.data_as(_u64p), k_scale,
                                       ctypes.byref(co), _stream(stream)))
        return co.scale

    def rescale_noalloc(self, a, n_limbs: int, out, scale: float = 1.0, stream=None) -> float:
        """Rescale whose scratch is a static device array (no allocation);
        see fides_rescale_noalloc in include/fides.h."""
        ca, co = self._ct(a, n_limbs, scale, "a"), self._ct(out, n_limbs - 1, 0.0, "out")
        _check(lib().fides_rescale_noalloc(self._h, ctypes.byref(ca), ctypes.byref(co), _stream(stream)))
        return co.scale


class Key:
    """A switching key registered with the library (``fides_key``): the device
    buffer ``tensor`` ([dnum][2][L+K][N], kept referenced here) bound to the
    Galois element it switches from (0: relinearisation).  Registration
    synchronises the device; the buffer must not change while the Key lives."""

    def __init__(self, ctx: "Context", t, galois: int):
        self.ctx, self.tensor, self.galois = ctx, t, int(galois)
        h = ctypes.c_void_p()
        _check(lib().fides_key_register(ctx._h, _ptr(t, ctx.key_words(), "key"), self.galois, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fides_key_destroy(self._h)
            self._h = None

    __del__ = close


def _key(k) -> int:
    """Handle of a Key (the entry points take registered keys, not buffers)."""
    if not isinstance(k, Key) or k._h is None:
        raise TypeError("expected a registered Key (Context.relin_key / rotation_key / conjugation_key / "
                        "register_key), got %s" % type(k).__name__)
    return k._h.value


class Op:
    """One operation of a batch: ``kind`` is OP_HMULT, OP_ROTATE or OP_RESCALE;
    a, b, out are CUDA tensors of ciphertexts [2][n_limbs][N]."""

    def __init__(self, kind, a, n_limbs, out, b=None, key=None, steps=0, stage=0, scale_a=1.0, scale_b=1.0):
        self.kind, self.a, self.n_limbs, self.out, self.b = kind, a, n_limbs, out, b
        self.key, self.steps, self.stage, self.scale_a, self.scale_b = key, steps, stage, scale_a, scale_b
        self.out_scale = None


class Batch:
    """A fixed batch of operations run with one launch per key-switch step per
    stage (fides_batch_*).  Keeps references to every tensor it was built on."""

    def __init__(self, ctx: "Context", ops):
        self.ctx, self.ops = ctx, list(ops)
        arr = (fides_op * max(1, len(self.ops)))()
        N = ctx.N
        for i, o in enumerate(self.ops):
            out_limbs = o.n_limbs - 1 if o.kind == OP_RESCALE else o.n_limbs
            arr[i].type, arr[i].stage = o.kind, o.stage
            arr[i].a = fides_ct(_ptr(o.a, 2 * o.n_limbs * N, "a").value, o.n_limbs, o.scale_a)
            if o.b is not None:
                arr[i].b = fides_ct(_ptr(o.b, 2 * o.n_limbs * N, "b").value, o.n_limbs, o.scale_b)
            arr[i].out = fides_ct(_ptr(o.out, 2 * out_limbs * N, "out").value, out_limbs, 0.0)
            arr[i].key = _key(o.key) if o.key is not None else None
            arr[i].steps = o.steps
        h = ctypes.c_void_p()
        _check(lib().fides_batch_create(ctx._h, arr, len(self.ops), ctypes.byref(h)))
        self._h = h
        for i, o in enumerate(self.ops):
            o.out_scale = arr[i].out.scale

    def run(self, stream=None):
        _check(lib().fides_batch_run(self._h, _stream(stream)))

    def capture(self, stream):
        """Record one run into a CUDA graph; later runs launch the graph."""
        _check(lib().fides_batch_capture(self._h, _stream(stream)))

    def info(self) -> dict:
        n, sb, tb = ctypes.c_int(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
        _check(lib().fides_batch_info(self._h, ctypes.byref(n), ctypes.byref(sb), ctypes.byref(tb)))
        g, t, po, ng = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().fides_batch_tuning(self._h, ctypes.byref(g), ctypes.byref(t), ctypes.byref(po), ctypes.byref(ng)))
        return {"launches": n.value, "scratch_bytes": sb.value, "table_bytes": tb.value, "group_limbs": g.value,
                "tensor_split": t.value, "prime_order": po.value, "groups": ng.value}

    def configure(self, group_limbs: int, tensor_split: int = 1, prime_order: int = 0):
        """Launch groups of at most group_limbs limbs (0: one per stage), the
        tensor-product placement and the NTT limb order (fides_batch_configure)."""
        _check(lib().fides_batch_configure(self._h, group_limbs, tensor_split, prime_order))

    def autotune(self, stream=None) -> float:
        """Times the candidate groupings and tensor placements on this batch and
        keeps the fastest (fides_batch_autotune); returns its ms per run."""
        ms = ctypes.c_double(0.0)
        _check(lib().fides_batch_autotune(self._h, _stream(stream), ctypes.byref(ms)))
        return ms.value

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fides_batch_destroy(self._h)
            self._h = None

    __del__ = close


def now_ns() -> int:
    """CLOCK_MONOTONIC nanoseconds, the clock of the server's timestamps."""
    return int(lib().fides_now_ns())


class _DeviceWords:
    """A raw device range exposed through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, words: int):
        self.__cuda_array_interface__ = {"shape": (words,), "typestr": "<i8", "data": (ptr, False),
                                         "version": 2, "strides": None}


class Completion:
    """A completion record of the request server."""

    def __init__(self, c: "fides_completion", N: int):
        self.id, self.tag, self.type, self.status = int(c.id), int(c.tag), int(c.type), int(c.status)
        self.ptr, self.n_limbs, self.scale = c.out.data, int(c.out.n_limbs), float(c.out.scale)
        self.t_submit_ns, self.t_admit_ns = int(c.t_submit_ns), int(c.t_admit_ns)
        self.t_launch_ns, self.t_done_ns = int(c.t_launch_ns), int(c.t_done_ns)
        self.group_ops, self.lane, self._N = int(c.group_ops), int(c.lane), N

    @property
    def latency_ns(self) -> int:
        return self.t_done_ns - self.t_submit_ns

    def tensor(self):
        """The output ciphertext [2][n_limbs][N] as a CUDA tensor aliasing the
        server's memory (valid until the request is released)."""
        import torch
        if not self.ptr:
            raise ValueError("request %d has no output (status %d)" % (self.id, self.status))
        return torch.as_tensor(_DeviceWords(self.ptr, 2 * self.n_limbs * self._N), device="cuda")


class Server:
    """The request server (fides_server_*): continuous batching of HMult,
    HRotate and Rescale requests on resident ciphertexts.  ``ctx`` may be None
    only with ``simulate=True`` (then ``shape`` = (logN, L, K, dnum))."""

    def __init__(self, ctx, arena_bytes: int, n_lanes: int = 2, max_batch: int = 32, max_pending: int = 1 << 16,
                 timeout_us: int = 0, simulate: bool = False, sim_ns_per_limb: int = 0, shape=None):
        cfg = fides_server_config()
        cfg.arena_bytes, cfg.n_lanes, cfg.max_batch, cfg.max_pending = arena_bytes, n_lanes, max_batch, max_pending
        cfg.timeout_us, cfg.simulate, cfg.sim_ns_per_limb = timeout_us, 1 if simulate else 0, sim_ns_per_limb
        if shape is not None:
            cfg.logN, cfg.L, cfg.K, cfg.dnum = shape
        self.ctx = ctx
        self.N = ctx.N if ctx is not None else (1 << cfg.logN)
        h = ctypes.c_void_p()
        _check(lib().fides_server_create(ctx._h if ctx is not None else None, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}     # request id -> input tensors, until completion
        self._keys = []     # the Keys the server uses
        self._poll_buf = {}

    @staticmethod
    def _addr(t, words, name):
        if isinstance(t, int):   # a raw device address (simulation)
            return t
        return _ptr(t, words, name).value

    @staticmethod
    def _key_arg(key):
        if isinstance(key, int):  # a token (simulation: handles are never dereferenced)
            return key
        return _key(key)

    def set_relin_key(self, key):
        """key: the relinearisation Key (an int token in simulation)."""
        self._keys.append(key)
        _check(lib().fides_server_set_relin_key(self._h, self._key_arg(key)))

    def add_rotation_key(self, steps: int, key):
        """key: the rotation Key of `steps` (an int token in simulation)."""
        self._keys.append(key)
        _check(lib().fides_server_add_rotation_key(self._h, steps, self._key_arg(key)))

    def submit(self, kind: int, a, n_limbs: int, b=None, steps: int = 0, tag: int = 0, scale_a: float = 1.0,
               scale_b: float = 1.0) -> int:
        r = fides_request()
        r.type, r.steps, r.tag = kind, steps, tag
        w = 2 * n_limbs * self.N
        r.a = fides_ct(self._addr(a, w, "a"), n_limbs, scale_a)
        if b is not None:
            r.b = fides_ct(self._addr(b, w, "b"), n_limbs, scale_b)
        rid = ctypes.c_uint64(0)
        _check(lib().fides_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (a, b)
        return rid.value

    def poll(self, max_n: int = 256, timeout_us: int = 0) -> list:
        buf = self._poll_buf.get(max_n)
        if buf is None:
            buf = self._poll_buf[max_n] = (fides_completion * max_n)()
        n = ctypes.c_int(0)
        _check(lib().fides_server_poll(self._h, buf, max_n, timeout_us, ctypes.byref(n)))
        out = [Completion(buf[i], self.N) for i in range(n.value)]
        for c in out:
            self._keep.pop(c.id, None)
        return out

    def release(self, rid: int):
        _check(lib().fides_server_release(self._h, rid))

    def cancel(self, rid: int):
        _check(lib().fides_server_cancel(self._h, rid))

    def pause(self, on: bool = True):
        _check(lib().fides_server_pause(self._h, 1 if on else 0))

    def inject(self, fault: int, arg: int):
        _check(lib().fides_server_inject(self._h, fault, arg))

    def stats(self) -> dict:
        st = fides_server_stats()
        _check(lib().fides_server_stats_read(self._h, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in fides_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fides_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    __del__ = close
