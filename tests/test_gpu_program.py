"""GPU program executor: a hand-written program that uses every instruction
(ModRaise, COPY, DROP, CMULT, RESCALE, CADD, MULI, HSUB, HADD, HMULT, CONJ,
CMAC with terms at several levels, LT) gives the oracle interpreter's
residues, and register reuse never lets a result overwrite a live operand."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle import bootstrap as obt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, find_primes, to_device, to_host  # noqa: E402
from paper_2507_04775_gb300 import bootstrap as bt  # noqa: E402


def rand_key(st, o):
    return np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])


def build(o, st):
    P = si.MID
    nl = P.nq
    prog = obt.Program()
    consts = [np.array([st.below(q) for q in o.q], dtype=np.uint64) for _ in range(5)]
    prog.consts, prog.const_scale = consts, [1.0] * 5
    idx = [0, 1, 5]
    prog.lts = [{"diag_idx": idx, "pts": [si.uniform_poly(st, o.q[:7], o.N) for _ in idx], "n1": 2,
                 "pt_scale": 1.0, "level": 7}]
    prog.lins = [[(10, 2), (9, 3), (2, 4)]]
    I = obt
    prog.instr = [
        (I.COPY, 1, 0, -1, 0),
        (I.DROP, 2, 1, -1, 9),
        (I.CMULT, 3, 2, -1, 0),
        (I.RESCALE, 4, 3, -1, 0),          # 8 limbs
        (I.CADD, 5, 4, -1, 1),
        (I.MULI, 6, 5, -1, -1),
        (I.HSUB, 7, 6, 5, 0),
        (I.HMULT, 8, 7, 6, 0),
        (I.RESCALE, 9, 8, -1, 0),          # 7 limbs
        (I.CONJ, 10, 9, -1, 0),
        (I.CMAC, 11, 10, 7, 0),            # r2 (9 limbs) and r9, r10 (7 limbs) read at 7 limbs
        (I.LT, 12, 11, -1, 0),
        (I.HADD, 13, 12, 11, 0),
        (I.MULI, 14, 13, -1, 1),
        (I.HMULT, 15, 14, 14, 0),          # a square: both operands one register
    ]
    prog.n_regs, prog.in_reg, prog.out_reg = 16, 0, 15
    return prog, nl


@pytest.mark.parametrize("nearest", [False, True], ids=["floor", "nearest"])
def test_every_instruction_matches_the_oracle(nearest):
    """In both rounding modes of the context: round-to-nearest reaches the
    program's ModDowns and Rescales (including HMULT+RESCALE pairs run as one
    key switch)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.MID
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    g, o = Context(P.logN, q, p, P.dnum), oracle.Context(P.logN, q, p, P.dnum)
    g.set_rounding(nearest)
    o.set_rounding(nearest)
    st = si.Stream(1101)
    prog, nl = build(o, st)
    rlk, ck = rand_key(st, o), rand_key(st, o)
    rks = {s: rand_key(st, o) for s in (1, 4)}       # baby step 1, giant step n1 * 2 = 4
    a = np.stack([si.uniform_poly(st, o.q, o.N) for _ in range(2)])
    ref = obt.run(o, prog, a, rlk, ck, rks)
    dp = bt.DeviceProgram(g, prog, g.relin_key(to_device(rlk)), g.conjugation_key(to_device(ck)),
                          [g.rotation_key(to_device(k), s) for s, k in rks.items()],
                          in_limbs=nl)
    assert dp.out_limbs == ref.shape[1] == 7
    assert dp.buffers < prog.n_regs                  # registers share buffers
    out = torch.empty(2 * 7 * o.N, dtype=torch.int64, device="cuda")
    dp.run(to_device(a), out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out).reshape(ref.shape), ref)
    # run twice: the program is reusable and its buffers start from any contents
    dp.run(to_device(a), out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out).reshape(ref.shape), ref)
    dp.close()
    g.close()


def test_modraise_program_matches_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.MID
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    g, o = Context(P.logN, q, p, P.dnum), oracle.Context(P.logN, q, p, P.dnum)
    st = si.Stream(1102)
    prog = obt.Program(instr=[(obt.MODRAISE, 1, 0, -1, 12), (obt.RESCALE, 2, 1, -1, 0)], n_regs=3, in_reg=0,
                       out_reg=2)
    a = np.stack([si.uniform_poly(st, o.q[:1], o.N) for _ in range(2)])
    ref = obt.run(o, prog, a, None, None, {})
    dp = bt.DeviceProgram(g, prog, None, None, {}, in_limbs=1)
    out = torch.empty(2 * 11 * o.N, dtype=torch.int64, device="cuda")
    dp.run(to_device(a), out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out).reshape(ref.shape), ref)
    dp.close()
    g.close()


def test_runs_overlap_on_two_streams_of_one_context():
    """Two programs on one context, each with its own work buffer (and so its
    own key-switching scratch), run on two streams at once: each result equals
    the oracle interpreter's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.MID
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    g, o = Context(P.logN, q, p, P.dnum), oracle.Context(P.logN, q, p, P.dnum)
    st = si.Stream(1103)
    prog, nl = build(o, st)
    rlk, ck = rand_key(st, o), rand_key(st, o)
    rks = {s: rand_key(st, o) for s in (1, 4)}
    keys = (g.relin_key(to_device(rlk)), g.conjugation_key(to_device(ck)),
            [g.rotation_key(to_device(k), s) for s, k in rks.items()])
    ins = [np.stack([si.uniform_poly(st, o.q, o.N) for _ in range(2)]) for _ in range(4)]
    refs = [obt.run(o, prog, a, rlk, ck, rks) for a in ins]
    dps = [bt.DeviceProgram(g, prog, *keys, in_limbs=nl) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in dps]
    outs = [torch.empty(2 * 7 * o.N, dtype=torch.int64, device="cuda") for _ in ins]
    dins = [to_device(a) for a in ins]
    torch.cuda.synchronize()
    for k in range(len(ins)):
        dps[k % 2].run(dins[k], outs[k], stream=streams[k % 2])
    torch.cuda.synchronize()
    for k in range(len(ins)):
        assert np.array_equal(to_host(outs[k]).reshape(refs[k].shape), refs[k]), k
    for dp in dps:
        dp.close()
    g.close()
