"""CKKS bootstrapping: the precomputation (planner) and its device program.

The paper runs bootstrapping on the GPU with constants precomputed by OpenFHE
(Sec. III-B, Sec. III-F7).  Here ``plan()`` is that precomputation: from the
ring, the q-primes and the input scale it builds a program for the library's
program executor (``fides_program_*`` in include/fides.h):

  ModRaise(1 limb -> L)                             t = m + q_0 I
  CoeffToSlot: 3 linear transforms of c F^H         slots (x_re + i x_im) / 2K, x = t / q_0,
                                                    in bit-reversed order
  u_re = w + conj(w), u_im = -i (w - conj(w))
  EvalMod(u) = Chebyshev interpolant of cos(2 pi (K u - 1/4) / 2^r), evaluated
               with baby steps T_1..T_m and giant steps T_m, T_2m, ... over a
               recursive Chebyshev division, then r steps c <- 2 c^2 - 1
               (= sin 2 pi x ~ 2 pi m / q_0)
  y = e_re + i e_im
  SlotToCoeff: 3 linear transforms of (q_0 / (2 pi D_in)) F
F is the slot DFT U[j][i] = zeta^(5^j i) without its bit reversal, as radix-2
butterfly stages grouped three ways (the level budget).  Every transform's
plaintexts are encoded at the prime its rescale removes, and inside EvalMod
every ciphertext at l limbs carries the exact scale sigma_l
(sigma_{l-1} = sigma_l^2 / q_{l-1}), operands with limbs to spare being
brought down by one product with a constant.

The planner encodes plaintexts itself (``encode_coeffs``: the special FFT
written as the same butterfly stages) and hands them to the device in
coefficient form; ``DeviceProgram`` reduces them modulo each prime and
transforms them with the library's NTT.  ``DeviceProgram`` also accepts a
program whose plaintexts are already residues in evaluation form.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import fides as F

OP = {"MODRAISE": 1, "LT": 2, "RESCALE": 3, "DROP": 4, "HADD": 5, "HSUB": 6, "HMULT": 7, "CONJ": 8, "MULI": 9,
      "CMULT": 10, "CADD": 11, "COPY": 12, "CMAC": 13, "ROT": 14}


class BootProgram:
    """A program: instructions (op, dst, a, b, arg) over registers, linear
    transforms, constants, the rotation steps it needs and its output scale."""

    def __init__(self):
        self.instr, self.lts, self.consts, self.const_scale, self.rot_steps = [], [], [], [], []
        self.lins = []          # CMAC term lists [(register, constant index)]
        self.n_regs = self.in_reg = self.out_reg = 0
        self.out_scale = 0.0


# ---------------------------------------------------------------------------
# slot DFT as butterfly stages
# ---------------------------------------------------------------------------
def _twiddles(ln: int) -> np.ndarray:
    h = ln // 2
    e = np.ones(h, dtype=np.int64)
    for j in range(1, h):
        e[j] = e[j - 1] * 5 % (4 * ln)
    return np.exp(1j * np.pi * e / (2 * ln))


def _stage_diagonals(n: int, ln: int) -> dict:
    """The butterfly stage on blocks of ln slots as diagonals {offset: vector}."""
    h = ln // 2
    w = np.tile(np.concatenate([_twiddles(ln), _twiddles(ln)]), n // ln)
    upper = (np.arange(n) % ln) < h
    diags = {0: np.where(upper, 1.0, -w).astype(complex)}
    for off, vec in ((h, np.where(upper, w, 0)), (n - h, np.where(upper, 0, 1.0))):
        diags[off % n] = diags.get(off % n, 0) + vec.astype(complex)
    return diags


def _compose(outer: dict, inner: dict, n: int) -> dict:
    """Diagonals of outer @ inner."""
    res = {}
    for a, va in outer.items():
        for b, vb in inner.items():
            key = (a + b) % n
            res[key] = res.get(key, 0) + va * np.roll(vb, -a)
    return res


def _adjoint(m: dict, n: int) -> dict:
    return {(n - d) % n: np.conj(np.roll(v, d)) for d, v in m.items()}


def slot_dft_groups(n: int, budget: int) -> list:
    """F = S_n ... S_2 in `budget` groups of consecutive stages, in the order
    they act (the group of S_2 first)."""
    logn = int(round(math.log2(n)))
    base, extra = divmod(logn, budget)
    out, first = [], 1
    for g in range(budget):
        cnt = base + (1 if g < extra else 0)
        acc = None
        for s in range(first, first + cnt):
            st = _stage_diagonals(n, 1 << s)
            acc = st if acc is None else _compose(st, acc, n)
        out.append(acc)
        first += cnt
    return out


def _special_ifft(z: np.ndarray) -> np.ndarray:
    """F^H z / n by applying the adjoint stages S_n^H first, ..., S_2^H last."""
    n = z.size
    v = z.astype(complex).copy()
    ln = n
    while ln >= 2:
        h = ln // 2
        w = _twiddles(ln)
        blk = v.reshape(-1, ln)
        top, bot = blk[:, :h].copy(), blk[:, h:].copy()
        # S^H: out_top = top + bot, out_bot = conj(w) (top - bot)
        blk[:, :h] = top + bot
        blk[:, h:] = np.conj(w) * (top - bot)
        ln = h
    return v / n


def encode_coeffs(z: np.ndarray, scale: float) -> np.ndarray:
    """Integer coefficients (int64, N = 2 len(z)) of the plaintext whose slots
    are scale * z: t_lo + i t_hi = (1/n) U^H (scale z), U = F P."""
    n = z.size
    w = _special_ifft(scale * np.asarray(z))
    bits = int(round(math.log2(n)))
    perm = np.array([int(format(i, "0%db" % bits)[::-1], 2) for i in range(n)]) if n > 1 else np.zeros(1, int)
    w = w[np.argsort(perm)]               # undo the bit reversal: w_i = (F^H z)_{brv(i)}
    t = np.concatenate([w.real, w.imag])
    return (np.sign(t) * np.floor(np.abs(t) + 0.5)).astype(np.int64)


# ---------------------------------------------------------------------------
# Chebyshev series
# ---------------------------------------------------------------------------
def chebyshev_coeffs(f, degree: int) -> np.ndarray:
    return np.polynomial.chebyshev.chebinterpolate(f, degree)


def chebyshev_split(c, D: int):
    """(q, r) with sum c_k T_k = q(u) T_D(u) + r(u), deg r < D."""
    c = np.asarray(c, dtype=float)
    hi = c[D:]
    q = hi.copy()
    q[1:] *= 2.0
    r = c[:D].copy()
    k = np.arange(1, hi.size)
    r[D - k] -= hi[1:]
    return q, r


# ---------------------------------------------------------------------------
# planner
# ---------------------------------------------------------------------------
class _Plan:
    def __init__(self, N: int, q):
        self.N, self.q = N, [int(x) for x in q]
        self.p = BootProgram()
        self.lv, self.sc = [], []
        self.sigma = {}
        self.lowered = {}
        self.period = N // 2    # slots in use: transforms act on vectors of this period

    def new(self, lv, sc):
        self.lv.append(lv)
        self.sc.append(sc)
        self.p.n_regs += 1
        return self.p.n_regs - 1

    def op(self, name, a, b=-1, arg=0, lv=None, sc=None):
        d = self.new(self.lv[a] if lv is None else lv, self.sc[a] if sc is None else sc)
        self.p.instr.append((OP[name], d, a, b, arg))
        return d

    def constant(self, value: float, limbs: int, scale: float) -> int:
        v = int(math.copysign(math.floor(abs(value) + 0.5), value))
        self.p.consts.append(np.array([v % self.q[i] for i in range(limbs)], dtype=np.uint64))
        self.p.const_scale.append(float(scale))
        return len(self.p.consts) - 1

    def rescale(self, a):
        l = self.lv[a]
        return self.op("RESCALE", a, lv=l - 1, sc=self.sc[a] / self.q[l - 1])

    def to_level(self, a, l):
        """a at l limbs with scale sigma[l] (one constant product and a rescale
        when a has more limbs; made once per register and level)."""
        if self.lv[a] == l:
            return a
        key = (a, l)
        if key not in self.lowered:
            self.lowered[key] = self._lower(a, l)
        return self.lowered[key]

    def _lower(self, a, l):
        if self.lv[a] > l + 1:
            a = self.op("DROP", a, arg=l + 1, lv=l + 1)
        cs = self.q[l] * self.sigma[l] / self.sc[a]
        k = self.constant(cs, l + 1, cs)
        return self.rescale(self.op("CMULT", a, arg=k, sc=self.sc[a] * cs))

    def pair(self, a, b):
        l = min(self.lv[a], self.lv[b])
        return self.to_level(a, l), self.to_level(b, l)

    def add(self, a, b, name="HADD"):
        a, b = self.pair(a, b)
        return self.op(name, a, b)

    def mul(self, a, b):
        a, b = self.pair(a, b)
        return self.rescale(self.op("HMULT", a, b, sc=self.sc[a] * self.sc[b]))

    def add_const(self, a, v):
        return self.op("CADD", a, arg=self.constant(v * self.sc[a], self.lv[a], 1.0))

    def transform(self, a, diags: dict):
        n = self.N // 2
        l = self.lv[a]
        ql = float(self.q[l - 1])
        idx = sorted(diags)
        stride = 0
        for i in idx:
            stride = math.gcd(stride, i)
        stride = stride or n
        n1 = min(self.period, stride * (1 << max(0, math.ceil(0.5 * math.log2(len(idx))))))
        coeffs = [encode_coeffs(np.roll(diags[i], n1 * (i // n1)), ql) for i in idx]
        self.p.lts.append({"diag_idx": idx, "coeffs": coeffs, "n1": n1, "pt_scale": ql, "level": l})
        for i in idx:
            for s in (i % n1, n1 * (i // n1)):
                if s % n and s not in self.p.rot_steps:
                    self.p.rot_steps.append(s)
        return self.rescale(self.op("LT", a, arg=len(self.p.lts) - 1, sc=self.sc[a] * ql))


def plan(N: int, q, in_scale: float, K: int = 25, degree: int = 119, double_angle: int = 2, budget: int = 3,
         baby: int = 16, scale0: float = 2.0 ** 54, slots: int | None = None) -> BootProgram:
    """Bootstrapping program for a ciphertext at one limb (modulo q[0]) with
    scale in_scale, in a context with q-primes q (len(q) = L).

    slots: slots in use, a power of two up to N/2 (default).  A sparse
    message (slot vector periodic with that period) is a polynomial in
    X^(N / 2 slots); after ModRaise, adding the rotations by slots, 2 slots,
    4 slots, ... (each step doubling the sum) projects t = m + q_0 I onto that
    subring, times N / (2 slots).  The transforms are the slots-point DFT
    with each diagonal repeated over the N/2 slots, and the trace's factor
    with the DFT's 1 / slots gives the 1 / (N/2) the constants already use."""
    n = N // 2
    ns = n if slots is None else int(slots)
    if not (2 <= ns <= n and ns & (ns - 1) == 0):
        raise ValueError("slots must be a power of two in [2, N/2]")
    L = len(q)
    P = _Plan(N, q)
    P.period = ns
    x = P.new(1, in_scale)
    P.p.in_reg = x
    t = P.op("MODRAISE", x, arg=L, lv=L, sc=scale0)
    step = ns
    while step < n:
        t = P.op("HADD", t, P.op("ROT", t, arg=step))
        if step not in P.p.rot_steps:
            P.p.rot_steps.append(step)
        step *= 2
    groups = slot_dft_groups(ns, budget)
    f = (scale0 / (n * q[0] * 2 * K)) ** (1.0 / budget)
    tile = n // ns
    for G in groups[::-1]:
        t = P.transform(t, {d: np.tile(f * v, tile) for d, v in _adjoint(G, ns).items()})
    c = P.op("CONJ", t)
    u_re = P.op("HADD", t, c)
    u_im = P.op("MULI", P.op("HSUB", t, c), arg=-1)
    coeffs = chebyshev_coeffs(lambda u: np.cos(2 * np.pi * (K * u - 0.25) / 2 ** double_angle), degree)
    e_re = _evalmod(P, u_re, coeffs, baby, double_angle)
    e_im = _evalmod(P, u_im, coeffs, baby, double_angle)
    e_re, e_im = P.pair(e_re, e_im)
    y = P.op("HADD", e_re, P.op("MULI", e_im, arg=1))
    f2 = (q[0] / (2 * np.pi * in_scale)) ** (1.0 / budget)
    for G in groups:
        y = P.transform(y, {d: np.tile(f2 * v, tile) for d, v in G.items()})
    P.p.out_reg = y
    P.p.out_scale = P.sc[y]
    P.p.rot_steps.sort()
    return P.p


def _evalmod(P: _Plan, u: int, coeffs, m: int, double_angle: int) -> int:
    top = P.lv[u]
    P.sigma = {top: P.sc[u]}
    for l in range(top, 1, -1):
        P.sigma[l - 1] = P.sigma[l] ** 2 / P.q[l - 1]

    def double(a):                       # 2 a^2 - 1
        s = P.mul(a, a)
        return P.add_const(P.op("HADD", s, s), -1.0)

    T = [None, u]
    for i in range(2, m + 1):
        if i % 2 == 0:
            T.append(double(T[i // 2]))
        else:
            pr = P.mul(T[(i + 1) // 2], T[(i - 1) // 2])
            T.append(P.add(P.op("HADD", pr, pr), T[1], name="HSUB"))
    giants = [T[m]]
    while m << len(giants) < len(coeffs):
        giants.append(double(giants[-1]))

    def linear(c):
        """sum_b c_b T_b: one multiply-accumulate reading every T_b at its own
        level, constants chosen so the rescaled sum has scale sigma."""
        used = [b for b in range(1, len(c)) if c[b] != 0.0] or [1]
        l = min(P.lv[T[b]] for b in used) - 1
        terms = []
        for b in used:
            cs = P.q[l] * P.sigma[l] / P.sc[T[b]]
            terms.append((T[b], P.constant((c[b] if b < len(c) else 0.0) * cs, l + 1, cs)))
        P.p.lins.append(terms)
        first_reg, first_k = terms[0]
        acc = P.op("CMAC", first_reg, b=l + 1, arg=len(P.p.lins) - 1, lv=l + 1,
                   sc=P.sc[first_reg] * P.p.const_scale[first_k])
        acc = P.rescale(acc)
        return P.add_const(acc, c[0]) if c[0] != 0.0 else acc

    def evaluate(c, k):
        if len(c) <= m:
            return linear(c)
        qc, rc = chebyshev_split(c, m << (k - 1))
        return P.add(P.mul(evaluate(qc, k - 1), giants[k - 1]), evaluate(rc, k - 1))

    e = evaluate(np.asarray(coeffs), len(giants))
    for _ in range(double_angle):
        e = double(e)
    return e


# ---------------------------------------------------------------------------
# device program
# ---------------------------------------------------------------------------
class DeviceProgram:
    """A program uploaded for ``fides_program_run``.  Plaintexts come either
    in coefficient form (``lt["coeffs"]``, int64 [N] each: reduced modulo every
    prime of the transform's level and transformed on the device) or as
    evaluation-form residues (``lt["pts"]``, [limbs][N])."""

    def __init__(self, ctx, prog, relin_key, conj_key, rot_keys, in_limbs: int = 1):
        """relin_key, conj_key: Keys (or None); rot_keys: rotation Keys (a list,
        or a dict whose values are used), found by their Galois elements."""
        import torch
        self.ctx = ctx
        N = ctx.N
        rot = list(rot_keys.values()) if isinstance(rot_keys, dict) else list(rot_keys)
        self._keep = [relin_key, conj_key] + rot
        self._pts = []
        lt_arr = (F.fides_lt * max(1, len(prog.lts)))()
        self._lt_tabs = []
        for k, t in enumerate(prog.lts):
            lvl = t["level"]
            devs = []
            if "coeffs" in t:
                qs = np.array(ctx.q[:lvl], dtype=np.int64)
                for cf in t["coeffs"]:
                    res = np.mod(np.asarray(cf, dtype=np.int64)[None, :], qs[:, None]).astype(np.uint64)
                    d = F.to_device(res)
                    ctx.ntt(d, 0, lvl)
                    devs.append(d)
            else:
                devs = [F.to_device(np.asarray(p)[:lvl]) for p in t["pts"]]
            self._pts.extend(devs)
            idx = (ctypes.c_int * len(t["diag_idx"]))(*t["diag_idx"])
            ptrs = (ctypes.c_void_p * len(devs))(*[d.data_ptr() for d in devs])
            self._lt_tabs.append((idx, ptrs))
            lt_arr[k].n_diag = len(devs)
            lt_arr[k].diag_idx = ctypes.cast(idx, ctypes.POINTER(ctypes.c_int))
            lt_arr[k].dev_pts = ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p))
            lt_arr[k].n1 = t["n1"]
            lt_arr[k].pt_scale = t["pt_scale"]
        torch.cuda.synchronize()
        ins = (F.fides_instr * len(prog.instr))(*[F.fides_instr(*x) for x in prog.instr])
        L = ctx.L
        const_rows = []
        for cst in prog.consts:
            row = np.zeros(L, dtype=np.uint64)
            row[:len(cst)] = cst
            const_rows.append(row)
        self._const_rows = const_rows
        cptr = (ctypes.c_void_p * max(1, len(const_rows)))(*[r.ctypes.data for r in const_rows])
        cscale = (ctypes.c_double * max(1, len(prog.const_scale)))(*prog.const_scale)
        kp = (ctypes.c_void_p * max(1, len(rot)))(*[F._key(k) for k in rot])
        d = F.fides_program_desc()
        d.n_instr, d.instr = len(prog.instr), ctypes.cast(ins, ctypes.POINTER(F.fides_instr))
        d.n_regs, d.in_reg, d.out_reg, d.in_limbs = prog.n_regs, prog.in_reg, prog.out_reg, in_limbs
        d.out_scale = prog.out_scale
        d.n_lt, d.lt = len(prog.lts), ctypes.cast(lt_arr, ctypes.POINTER(F.fides_lt))
        d.n_const = len(const_rows)
        d.consts = ctypes.cast(cptr, ctypes.POINTER(ctypes.c_void_p))
        d.const_scale = ctypes.cast(cscale, ctypes.POINTER(ctypes.c_double))
        d.relin_key = F._key(relin_key) if relin_key is not None else None
        d.conj_key = F._key(conj_key) if conj_key is not None else None
        d.n_rot_keys = len(rot)
        d.rot_keys = ctypes.cast(kp, ctypes.POINTER(ctypes.c_void_p))
        lins = getattr(prog, "lins", [])
        starts = [0]
        for lin in lins:
            starts.append(starts[-1] + len(lin))
        ls = (ctypes.c_int * len(starts))(*starts)
        lr = (ctypes.c_int * max(1, starts[-1]))(*[r for lin in lins for r, _ in lin])
        lc = (ctypes.c_int * max(1, starts[-1]))(*[k for lin in lins for _, k in lin])
        d.n_lin = len(lins)
        d.lin_start = ctypes.cast(ls, ctypes.POINTER(ctypes.c_int))
        d.lin_reg = ctypes.cast(lr, ctypes.POINTER(ctypes.c_int))
        d.lin_const = ctypes.cast(lc, ctypes.POINTER(ctypes.c_int))
        self._refs = (ins, lt_arr, cptr, cscale, kp, ls, lr, lc)
        h = ctypes.c_void_p()
        F._check(F.lib().fides_program_create(ctx._h, ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        w, nb, ol = ctypes.c_size_t(0), ctypes.c_int(0), ctypes.c_int(0)
        F._check(F.lib().fides_program_info(h, ctypes.byref(w), ctypes.byref(nb), ctypes.byref(ol)))
        self.work_words, self.buffers, self.out_limbs = w.value, nb.value, ol.value
        self.in_limbs = in_limbs
        self.work = torch.empty(max(1, self.work_words), dtype=torch.int64, device="cuda")

    def run(self, a, out, scale: float = 1.0, stream=None) -> float:
        ca = self.ctx._ct(a, self.in_limbs, scale, "a")
        co = self.ctx._ct(out, self.out_limbs, 0.0, "out")
        F._check(F.lib().fides_program_run(self._h, ctypes.byref(ca), ctypes.byref(co),
                                           F._ptr(self.work, self.work_words, "work"), self.work.numel(),
                                           F._stream(stream)))
        return co.scale

    def close(self):
        if getattr(self, "_h", None) and F._lib is not None:
            F._lib.fides_program_destroy(self._h)
            self._h = None

    __del__ = close
