"""The library's bootstrapping planner on the CPU: its encoder, its slot DFT
factorisation and its Chebyshev split against their definitions, and the
program it plans, executed with the oracle's operations, refreshes a
ciphertext within 2^-12.  (GPU execution: test_gpu_bootstrap.py.)"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle import bootstrap as obt
from oracle.client import Client
from paper_2507_04775_gb300 import bootstrap as bt


def dense(M, n):
    A = np.zeros((n, n), dtype=complex)
    r = np.arange(n)
    for d, v in M.items():
        A[r, (r + d) % n] += v
    return A


@pytest.mark.parametrize("n", [8, 64, 512])
def test_encoder_inverts_the_slot_evaluation(n):
    """Decoding the integer coefficients by direct evaluation at zeta^(5^j)
    returns the slots, up to the rounding of the coefficients."""
    N = 2 * n
    st = si.Stream(11, n)
    z = st.complex_slots(n)
    scale = 2.0 ** 30
    t = bt.encode_coeffs(z, scale)
    assert t.shape == (N,)
    ex = np.array([pow(5, j, 2 * N) for j in range(n)])
    vals = np.exp(1j * np.pi * np.outer(ex, np.arange(N)) / N) @ t.astype(np.float64)
    assert np.max(np.abs(vals / scale - z)) < n * 2.0 ** -29
    # the oracle's encoder (FFT of the odd-root evaluations) agrees up to the last rounding
    assert np.max(np.abs(t - oracle.encode(z, N, scale))) <= 1


@pytest.mark.parametrize("n,budget", [(16, 3), (128, 3), (64, 2)])
def test_slot_dft_groups_are_the_dft(n, budget):
    N = 2 * n
    U = np.exp(1j * np.pi * np.outer([pow(5, j, 2 * N) for j in range(n)], np.arange(n)) / N)
    bits = n.bit_length() - 1
    Fm = np.eye(n, dtype=complex)
    for G in bt.slot_dft_groups(n, budget):
        Fm = dense(G, n) @ Fm
    perm = [int(format(i, "0%db" % bits)[::-1], 2) for i in range(n)]
    assert np.max(np.abs(Fm[:, perm] - U)) < 1e-12


def test_chebyshev_split():
    c = bt.chebyshev_coeffs(np.cos, 40)
    q, r = bt.chebyshev_split(c, 16)
    u = np.linspace(-1, 1, 501)
    T16 = np.cos(16 * np.arccos(u))
    lhs = np.polynomial.chebyshev.chebval(u, q) * T16 + np.polynomial.chebyshev.chebval(u, r)
    assert np.max(np.abs(lhs - np.cos(u))) < 1e-13


def as_eval_form(ctx, prog):
    """The planned program with its coefficient-form plaintexts moved to
    evaluation-form residues (the oracle interpreter's format)."""
    out = obt.Program(instr=list(prog.instr), consts=list(prog.consts), const_scale=list(prog.const_scale),
                      n_regs=prog.n_regs, in_reg=prog.in_reg, out_reg=prog.out_reg, rot_steps=list(prog.rot_steps),
                      out_scale=prog.out_scale, lins=list(prog.lins))
    for t in prog.lts:
        lvl = t["level"]
        idx = list(range(lvl))
        pts = [ctx.ntt_limbs(ctx.from_signed(cf, idx), idx) for cf in t["coeffs"]]
        out.lts.append({"diag_idx": t["diag_idx"], "pts": pts, "n1": t["n1"], "pt_scale": t["pt_scale"],
                        "level": lvl})
    return out


def test_planned_bootstrap_refreshes_a_ciphertext():
    q0 = oracle.find_primes(12, 60, 1)
    q = q0 + oracle.find_primes(12, 54, 29, exclude=q0)
    p = oracle.find_primes(12, 60, 10, exclude=q)
    ctx = oracle.Context(12, q, p, 3)
    cl = Client(ctx, seed=si.workload_seed(4) + 1, hamming=192)
    prog = bt.plan(ctx.N, q, 2.0 ** 50)
    assert len(prog.lts) == 6 and prog.instr[0][0] == bt.OP["MODRAISE"]
    ev = as_eval_form(ctx, prog)
    rks = {s: cl.rotation_key(s) for s in prog.rot_steps}
    z = cl.random_slots()
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    out = obt.run(ctx, ev, ct, cl.relin_key(), cl.conjugation_key(), rks)
    err = np.max(np.abs(cl.decrypt(out, prog.out_scale) - z)) / max(1.0, np.max(np.abs(z)))
    assert err < 2.0 ** -12, err


def _sparse_setup(seed):
    q0 = oracle.find_primes(12, 60, 1)
    q = q0 + oracle.find_primes(12, 54, 29, exclude=q0)
    p = oracle.find_primes(12, 60, 10, exclude=q)
    ctx = oracle.Context(12, q, p, 3)
    return ctx, Client(ctx, seed=seed, hamming=192), q


@pytest.mark.parametrize("slots", [256, 16])
def test_oracle_sparse_bootstrap_refreshes_a_ciphertext(slots):
    """The oracle planner with fewer slots than N/2: a message whose slot
    vector repeats with period `slots` comes back within 2^-12, after the
    trace (log2(N / 2 slots) rotate-and-add steps) and slots-point transforms."""
    ctx, cl, q = _sparse_setup(si.workload_seed(4) + 11)
    prog = obt.plan(cl, q, 2.0 ** 50, slots=slots)
    n = ctx.N // 2
    reps = n // slots
    assert sum(1 for ins in prog.instr if ins[0] == obt.ROT) == reps.bit_length() - 1
    assert [s for s in prog.rot_steps if s % slots == 0 and s >= slots] == [slots << k for k in range(reps.bit_length() - 1)]
    rks = {s: cl.rotation_key(s) for s in prog.rot_steps}
    z = np.tile(cl.random_slots()[:slots], reps)
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    out = obt.run(ctx, prog, ct, cl.relin_key(), cl.conjugation_key(), rks)
    got = cl.decrypt(out, prog.out_scale)
    err = np.max(np.abs(got - z)) / max(1.0, np.max(np.abs(z)))
    assert err < 2.0 ** -12, err


def test_library_sparse_plan_refreshes_a_ciphertext():
    """The library planner's program with 64 slots, run by the oracle."""
    ctx, cl, q = _sparse_setup(si.workload_seed(4) + 12)
    prog = bt.plan(ctx.N, q, 2.0 ** 50, slots=64)
    ev = as_eval_form(ctx, prog)
    rks = {s: cl.rotation_key(s) for s in prog.rot_steps}
    z = np.tile(cl.random_slots()[:64], ctx.N // 2 // 64)
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    out = obt.run(ctx, ev, ct, cl.relin_key(), cl.conjugation_key(), rks)
    err = np.max(np.abs(cl.decrypt(out, prog.out_scale) - z)) / max(1.0, np.max(np.abs(z)))
    assert err < 2.0 ** -12, err
