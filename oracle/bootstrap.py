"""CKKS bootstrapping on the oracle: planner and interpreter.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper bootstraps with CoeffToSlot / SlotToCoeff as baby-step giant-step
linear transforms with hoisted rotations and EvalMod as a polynomial
approximation with double-angle steps (Sec. III-F6, Sec. III-F7); its
constants come from OpenFHE's precomputation (Sec. III-B).  Here the
precomputation is ``plan()``: it turns the parameters into a *program* -- a
list of homomorphic instructions over registers, the plaintext diagonals of
the linear transforms and the scalar constants -- and ``run()`` executes a
program with the oracle's operations.  A program is plain data, so the same
program can be executed by the CUDA library and compared residue for residue.

Algorithm (n = N/2 slots, ciphertext at one limb q_0 with scale D_in):
  1. ModRaise to L limbs: decrypts to t = m + q_0 I (I small).
  2. CoeffToSlot: w~ = c F^H z, where the slot DFT U (U[j][i] = zeta^(5^j i))
     factors as U = F P (F = S_n ... S_4 S_2 radix-2 butterfly stages, P the
     bit reversal); with real coefficients, (1/n) U^H applied to the slots of
     t gives t_i + i t_{i+n}, so c F^H yields them in bit-reversed order.  F^H
     is split into three groups of stages, each one linear transform (level
     budget 3) followed by a rescale; c = S_0 / (n q_0 2K) makes the slots
     (x_re + i x_im) / (2K), x = t / q_0.
  3. Real and imaginary parts: u_re = w + conj(w), u_im = -i (w - conj(w)).
  4. EvalMod on each: the Chebyshev interpolant of cos(2 pi (K u - 1/4) / 2^r)
     on [-1, 1], evaluated with baby steps T_1..T_m, giant steps T_m, T_2m, ...
     and recursive Chebyshev division; then r double-angle steps
     (c <- 2 c^2 - 1) give sin(2 pi x) ~ 2 pi m / q_0.
  5. y = e_re + i e_im; SlotToCoeff: z = (q_0 / (2 pi D_in)) F y in three
     groups of stages, each a linear transform and a rescale.
Every plaintext of a transform is encoded at the scale of the prime its
rescale removes, so transforms keep the scale; scalar constants are encoded
the same way, so products by constants keep it too.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from oracle import encode

# instruction codes (shared program format)
MODRAISE, LT, RESCALE, DROP, HADD, HSUB, HMULT, CONJ, MULI, CMULT, CADD, COPY, CMAC, ROT = range(1, 15)


@dataclass
class Program:
    instr: list = field(default_factory=list)       # (op, dst, a, b, arg)
    lts: list = field(default_factory=list)         # dict(diag_idx, pts, n1, pt_scale, level)
    consts: list = field(default_factory=list)      # residues (uint64, one per limb of its level)
    const_scale: list = field(default_factory=list)
    n_regs: int = 0
    in_reg: int = 0
    out_reg: int = 0
    rot_steps: list = field(default_factory=list)
    out_scale: float = 0.0
    lins: list = field(default_factory=list)        # CMAC term lists: [(register, constant index)]


# ---------------------------------------------------------------------------
# slot DFT factorisation
# ---------------------------------------------------------------------------
def dft_stage(n: int, ln: int) -> dict:
    """Butterfly stage on blocks of ln slots as {diagonal offset: vector}:
    out[b+j] = v[b+j] + w_j v[b+j+ln/2], out[b+j+ln/2] = v[b+j] - w_j v[b+j+ln/2],
    w_j = exp(i pi (5^j mod 4 ln) / (2 ln))."""
    h = ln // 2
    r = np.arange(n)
    pos = r % ln
    top = pos < h
    j = np.where(top, pos, pos - h)
    w = np.exp(1j * np.pi * np.array([pow(5, int(x), 4 * ln) for x in range(h)]) / (2 * ln))[j]
    d0 = np.where(top, 1.0 + 0j, -w)
    dp = np.where(top, w, 0j)
    dm = np.where(top, 0j, 1.0 + 0j)
    out = {0: d0}
    out[h % n] = out.get(h % n, 0) + dp
    out[(-h) % n] = out.get((-h) % n, 0) + dm
    return out


def diag_mul(A: dict, B: dict, n: int) -> dict:
    """Product of two matrices given by diagonals: (AB)_d[r] = sum A_d1[r] B_d2[r + d1]."""
    out = {}
    for d1, a in A.items():
        for d2, b in B.items():
            d = (d1 + d2) % n
            out[d] = out.get(d, 0) + a * np.roll(b, -d1)
    return {d: v for d, v in out.items() if np.max(np.abs(v)) > 1e-300}


def diag_adjoint(M: dict, n: int) -> dict:
    """Conjugate transpose: (M^H)_d[r] = conj(M_{-d}[r + d])."""
    return {(-d) % n: np.conj(np.roll(v, d)) for d, v in M.items()}


def dft_groups(n: int, budget: int = 3) -> list:
    """F = S_n ... S_2 as `budget` products of consecutive stages, listed in
    the order they apply to a vector (first: the group holding S_2)."""
    logn = n.bit_length() - 1
    sizes = [logn // budget + (1 if k < logn % budget else 0) for k in range(budget)]
    groups, s = [], 1
    for sz in sizes:
        M = None
        for ln in (2 ** (s + t) for t in range(sz)):
            st = dft_stage(n, ln)
            M = st if M is None else diag_mul(st, M, n)
        groups.append(M)
        s += sz
    return groups


# ---------------------------------------------------------------------------
# Chebyshev series
# ---------------------------------------------------------------------------
def cheb_interp(f, d: int) -> np.ndarray:
    """Coefficients c_0..c_d of the degree-d Chebyshev interpolant of f on [-1, 1]."""
    th = np.pi * (np.arange(d + 1) + 0.5) / (d + 1)
    fx = f(np.cos(th))
    c = np.array([2.0 / (d + 1) * np.sum(fx * np.cos(k * th)) for k in range(d + 1)])
    c[0] /= 2
    return c


def cheb_divide(c, D: int):
    """c = q T_D + r with deg r < D (T_D T_j = (T_{D+j} + T_{|D-j|}) / 2)."""
    c = list(c)
    q = [c[D]] + [2 * c[D + j] for j in range(1, len(c) - D)]
    r = c[:D]
    for j in range(1, len(c) - D):
        r[D - j] -= c[D + j]
    return q, r


# ---------------------------------------------------------------------------
# planner
# ---------------------------------------------------------------------------
class _Builder:
    def __init__(self, client, q, scale0):
        self.cl, self.q, self.N = client, q, client.ctx.N
        self.prog = Program()
        self.level, self.scale = {}, {}
        self.S0 = scale0

    def reg(self, level, scale):
        r = self.prog.n_regs
        self.prog.n_regs += 1
        self.level[r], self.scale[r] = level, scale
        return r

    def emit(self, op, a, b=-1, arg=0, level=None, scale=None):
        dst = self.reg(level, scale)
        self.prog.instr.append((op, dst, a, b, arg))
        return dst

    def const(self, residues, scale):
        self.prog.consts.append(np.asarray(residues, dtype=np.uint64))
        self.prog.const_scale.append(float(scale))
        return len(self.prog.consts) - 1

    def residues(self, v: float, nl: int):
        x = int(np.sign(v) * np.floor(abs(v) + 0.5))
        return [x % qi for qi in self.q[:nl]]

    # -- operations with level/scale bookkeeping --------------------------
    # Inside EvalMod every ciphertext at nl limbs carries exactly the scale
    # sigma[nl], with sigma[nl - 1] = sigma[nl]^2 / q_{nl-1}: products of two
    # operands at one level land on the next level's scale by themselves, and
    # an operand with limbs to spare is brought to a lower level and its scale
    # by one product with a constant and a rescale (adjust).
    def set_base(self, nl, scale):
        self.sigma = {nl: scale}
        for k in range(nl, 1, -1):
            self.sigma[k - 1] = self.sigma[k] ** 2 / self.q[k - 1]

    def rescale(self, a):
        nl = self.level[a]
        return self.emit(RESCALE, a, level=nl - 1, scale=self.scale[a] / self.q[nl - 1])

    def drop(self, a, nl):
        if self.level[a] == nl:
            return a
        return self.emit(DROP, a, arg=nl, level=nl, scale=self.scale[a])

    def adjust(self, a, nl):
        """a at nl limbs with scale sigma[nl] (computed once per register and level)."""
        if self.level[a] == nl:
            return a
        memo = self.__dict__.setdefault("_adjusted", {})
        if (a, nl) not in memo:
            memo[(a, nl)] = self._adjust(a, nl)
        return memo[(a, nl)]

    def _adjust(self, a, nl):
        a = self.drop(a, nl + 1)
        cs = self.q[nl] * self.sigma[nl] / self.scale[a]
        k = self.const(self.residues(cs, nl + 1), cs)
        m = self.emit(CMULT, a, arg=k, level=nl + 1, scale=self.scale[a] * cs)
        return self.rescale(m)

    def align(self, a, b):
        nl = min(self.level[a], self.level[b])
        return self.adjust(a, nl), self.adjust(b, nl)

    def add(self, a, b):
        a, b = self.align(a, b)
        return self.emit(HADD, a, b, level=self.level[a], scale=self.scale[a])

    def sub(self, a, b):
        a, b = self.align(a, b)
        return self.emit(HSUB, a, b, level=self.level[a], scale=self.scale[a])

    def mult(self, a, b):
        a, b = self.align(a, b)
        m = self.emit(HMULT, a, b, level=self.level[a], scale=self.scale[a] * self.scale[b])
        return self.rescale(m)

    def cadd(self, a, v: float):
        nl = self.level[a]
        k = self.const(self.residues(v * self.scale[a], nl), 1.0)
        return self.emit(CADD, a, arg=k, level=nl, scale=self.scale[a])

    def lt(self, a, diags: dict, n1: int):
        nl = self.level[a]
        n = self.N // 2
        ql = float(self.q[nl - 1])
        idx = sorted(diags)
        pts = [self.cl.encode_eval(np.roll(diags[i], n1 * (i // n1)), nl, ql) for i in idx]
        self.prog.lts.append({"diag_idx": idx, "pts": pts, "n1": n1, "pt_scale": ql, "level": nl})
        for i in idx:
            for s in (i % n1, n1 * (i // n1)):
                if s % n and s not in self.prog.rot_steps:
                    self.prog.rot_steps.append(s)
        m = self.emit(LT, a, arg=len(self.prog.lts) - 1, level=nl, scale=self.scale[a] * ql)
        return self.rescale(m)


def _bsgs_n1(idx, n: int) -> int:
    """Baby-step size for a diagonal set: the offsets are multiples of a power
    of two `stride`; n1 = stride * 2^ceil(log2(sqrt(count)))."""
    stride = n
    for i in idx:
        if i:
            stride = math.gcd(stride, i)
    cnt = len(idx)
    return min(n, stride * (1 << max(0, math.ceil(math.log2(math.sqrt(cnt))))))


def plan(client, q, in_scale: float, K: int = 25, degree: int = 119, double_angle: int = 2, budget: int = 3,
         baby: int = 16, scale0: float = 2.0 ** 54, slots: int | None = None) -> Program:
    """Bootstrapping program for a ciphertext at one limb with scale in_scale;
    q: the q-primes (q[0] is the one removed by ModRaise's lift).

    slots: the number of slots in use, a power of two up to N/2 (default N/2).
    With fewer (sparse packing), the message's slot vector repeats with period
    `slots`, i.e. the message lies in Z[Y], Y = X^(N / (2 slots)).  After
    ModRaise the trace onto that subring -- the sum of the rotations by
    multiples of `slots`, as log2(N / (2 slots)) rotate-and-add steps --
    multiplies its part of t = m + q_0 I by N / (2 slots) and removes the rest
    of I.  The slot transforms are then those of a ring of degree 2 slots:
    the DFT on `slots` points, its diagonals repeated to fill the N/2 slots
    (a rotation by d < slots of a periodic vector is a rotation by d within
    each period), and the trace's factor takes the place of the DFT's
    1 / (N/2) -> 1 / slots normalisation, so the scaling constants stay."""
    N = client.ctx.N
    n = N // 2
    ns = n if slots is None else int(slots)
    assert 2 <= ns <= n and ns & (ns - 1) == 0, "slots must be a power of two in [2, N/2]"
    reps = n // ns
    L = len(q)
    B = _Builder(client, q, scale0)
    x = B.reg(1, in_scale)
    B.prog.in_reg = x
    r = B.emit(MODRAISE, x, arg=L, level=L, scale=scale0)
    # trace onto the subring: r <- r + rot(r, ns 2^k) for k < log2(reps)
    k = 0
    while (ns << k) < n:
        rot = B.emit(ROT, r, arg=ns << k, level=L, scale=B.scale[r])
        if (ns << k) not in B.prog.rot_steps:
            B.prog.rot_steps.append(ns << k)
        r = B.emit(HADD, r, rot, level=L, scale=B.scale[r])
        k += 1

    groups = dft_groups(ns, budget)
    # CoeffToSlot: c F^H = c G_1^H G_2^H ... (the last stages first); the
    # trace's factor reps and the DFT's 1 / ns make 1 / n as before
    c = scale0 / (n * q[0] * 2 * K)
    f = abs(c) ** (1.0 / budget)
    w = r
    for G in reversed(groups):
        D = {d: np.tile(v * f, reps) for d, v in diag_adjoint(G, ns).items()}
        w = B.lt(w, D, _bsgs_n1(sorted(D), ns))

    cj = B.emit(CONJ, w, level=B.level[w], scale=B.scale[w])
    u_re = B.emit(HADD, w, cj, level=B.level[w], scale=B.scale[w])
    dif = B.emit(HSUB, w, cj, level=B.level[w], scale=B.scale[w])
    u_im = B.emit(MULI, dif, arg=-1, level=B.level[w], scale=B.scale[w])

    coeffs = cheb_interp(lambda u: np.cos(2 * np.pi * (K * u - 0.25) / 2 ** double_angle), degree)
    e_re = _evalmod(B, u_re, coeffs, baby, double_angle)
    e_im = _evalmod(B, u_im, coeffs, baby, double_angle)
    e_re, e_im = B.align(e_re, e_im)
    ie = B.emit(MULI, e_im, arg=1, level=B.level[e_im], scale=B.scale[e_im])
    y = B.add(e_re, ie)

    # SlotToCoeff: c' F = c' G_last ... G_1 (the first stages first)
    c2 = q[0] / (2 * np.pi * in_scale)
    f2 = c2 ** (1.0 / budget)
    for G in groups:
        D = {d: np.tile(v * f2, reps) for d, v in G.items()}
        y = B.lt(y, D, _bsgs_n1(sorted(D), ns))
    B.prog.out_reg = y
    B.prog.out_scale = B.scale[y]
    B.prog.rot_steps.sort()
    return B.prog


def _evalmod(B: _Builder, u: int, coeffs, m: int, double_angle: int) -> int:
    d = len(coeffs) - 1
    B.set_base(B.level[u], B.scale[u])
    # baby steps T_1..T_m
    T = {1: u}
    for i in range(2, m + 1):
        if i % 2 == 0:
            t = B.mult(T[i // 2], T[i // 2])
            t = B.cadd(B.add(t, t), -1.0)
        else:
            t = B.mult(T[(i + 1) // 2], T[(i - 1) // 2])
            t = B.sub(B.add(t, t), T[1])
        T[i] = t
    # giant steps T_m, T_2m, T_4m, ...
    G = [T[m]]
    while m * 2 ** len(G) < d + 1:
        g = B.mult(G[-1], G[-1])
        G.append(B.cadd(B.add(g, g), -1.0))

    def leaf(c):
        """sum_b c_b T_b at one level below the lowest T_b used, with scale sigma
        there: one multiply-accumulate over the T_b (each read at its own level)
        with constants c_b q sigma / scale(T_b), then a rescale."""
        terms = [b for b in range(1, len(c)) if c[b] != 0.0] or [1]
        out_nl = min(B.level[T[b]] for b in terms) - 1
        lin = []
        for b in terms:
            cs = B.q[out_nl] * B.sigma[out_nl] / B.scale[T[b]]
            lin.append((T[b], B.const(B.residues((c[b] if b < len(c) else 0.0) * cs, out_nl + 1), cs)))
        B.prog.lins.append(lin)
        k0 = lin[0][1]
        acc = B.emit(CMAC, lin[0][0], out_nl + 1, len(B.prog.lins) - 1, level=out_nl + 1,
                     scale=B.scale[lin[0][0]] * B.prog.const_scale[k0])
        acc = B.rescale(acc)
        return B.cadd(acc, c[0]) if c[0] else acc

    def rec(c, k):
        if len(c) <= m:
            return leaf(c)
        D = m * 2 ** (k - 1)
        qc, rc = cheb_divide(c, D)
        Q = rec(qc, k - 1)
        R = rec(rc, k - 1)
        return B.add(B.mult(Q, G[k - 1]), R)

    x = rec(list(coeffs), len(G))
    for _ in range(double_angle):
        s = B.mult(x, x)
        x = B.cadd(B.add(s, s), -1.0)
    return x


# ---------------------------------------------------------------------------
# interpreter
# ---------------------------------------------------------------------------
def run(ctx, prog: Program, ct, relin_key, conj_key, rot_keys: dict, registers: dict | None = None) -> np.ndarray:
    """Execute a program with the oracle's operations; rot_keys: {steps: key}.
    If `registers` is a dict it receives every register's final value."""
    N = ctx.N
    R = {prog.in_reg: np.asarray(ct, dtype=np.uint64)}
    for op, dst, a, b, arg in prog.instr:
        x = R[a] if op != CMAC else None
        if op == MODRAISE:
            y = ctx.modraise(x, arg)
        elif op == LT:
            t = prog.lts[arg]
            keys = {s: rot_keys[s] for s in _lt_steps(t["diag_idx"], t["n1"], N // 2)}
            y = ctx.linear_transform(x, t["diag_idx"], [p[:x.shape[1]] for p in t["pts"]], t["n1"], keys)
        elif op == RESCALE:
            y = ctx.rescale(x)
        elif op == DROP:
            y = np.ascontiguousarray(x[:, :arg])
        elif op == HADD:
            y = ctx.hadd(x, R[b])
        elif op == HSUB:
            y = ctx.hsub(x, R[b])
        elif op == HMULT:
            y = ctx.hmult(x, R[b], relin_key)
        elif op == CONJ:
            y = ctx.conjugate(x, conj_key)
        elif op == ROT:
            y = ctx.rotate(x, arg, rot_keys[arg])
        elif op == MULI:
            y = ctx.mul_monomial(x, N // 2 if arg > 0 else 3 * N // 2)
        elif op == CMULT:
            y = ctx.scalar_mult(x, prog.consts[arg][:x.shape[1]])
        elif op == CADD:
            y = ctx.scalar_add(x, prog.consts[arg][:x.shape[1]])
        elif op == COPY:
            y = x.copy()
        elif op == CMAC:
            y = None
            for r, k in prog.lins[arg]:
                t = ctx.scalar_mult(np.ascontiguousarray(R[r][:, :b]), prog.consts[k][:b])
                y = t if y is None else ctx.hadd(y, t)
        else:
            raise ValueError("unknown instruction %d" % op)
        R[dst] = y
    if registers is not None:
        registers.update(R)
    return R[prog.out_reg]


def _lt_steps(idx, n1, n):
    s = set()
    for i in idx:
        for v in (i % n1, n1 * (i // n1)):
            if v % n:
                s.add(v)
    return sorted(s)
