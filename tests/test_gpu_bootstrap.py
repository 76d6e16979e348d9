"""GPU bootstrapping through the program executor: the oracle's program run on
the device equals the oracle's own run residue for residue (logN=12, all
slots and 256 of 2048); the library's planned program equals the oracle's
execution of the same program and refreshes a ciphertext within 2^-12
(logN=12, 15 and 16, h = 192), also with 2^14, 512 and 64 slots at logN=16
(sparse packing: the message's slot vector repeats with that period)."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle import bootstrap as obt
from oracle.client import Client

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, FidesError, to_device, to_host  # noqa: E402
from paper_2507_04775_gb300 import bootstrap as bt  # noqa: E402
from paper_2507_04775_gb300 import fides as F  # noqa: E402


def boot_primes(logN):
    q0 = oracle.find_primes(logN, 60, 1)
    q = q0 + oracle.find_primes(logN, 54, 29, exclude=q0)
    p = oracle.find_primes(logN, 60, 10, exclude=q)
    return q, p


def setup(logN, seed):
    q, p = boot_primes(logN)
    o = oracle.Context(logN, q, p, 3)
    cl = Client(o, seed=seed, hamming=192)
    return Context(logN, q, p, 3), o, cl, q


def dev_keys(g, cl, steps):
    rlk, ck = cl.relin_key(), cl.conjugation_key()
    rks = {s: cl.rotation_key(s) for s in steps}
    return (rlk, ck, rks), (g.relin_key(to_device(rlk)), g.conjugation_key(to_device(ck)),
                            [g.rotation_key(to_device(k), s) for s, k in rks.items()])


def run_device(g, prog, dkeys, ct, out_limbs):
    dp = bt.DeviceProgram(g, prog, dkeys[0], dkeys[1], dkeys[2])
    assert dp.out_limbs == out_limbs
    out = torch.empty(2 * out_limbs * g.N, dtype=torch.int64, device="cuda")
    sc = dp.run(to_device(ct), out, scale=2.0 ** 50)
    torch.cuda.synchronize()
    res = to_host(out).reshape(2, out_limbs, g.N)
    dp.close()
    return res, sc


def test_oracle_program_on_the_device_is_bit_exact():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o, cl, q = setup(12, si.workload_seed(4))
    prog = obt.plan(cl, q, 2.0 ** 50)
    hkeys, dkeys = dev_keys(g, cl, prog.rot_steps)
    z = cl.random_slots()
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    ref = obt.run(o, prog, ct, *hkeys)
    got, sc = run_device(g, prog, dkeys, ct, ref.shape[1])
    assert np.array_equal(got, ref)
    assert sc == prog.out_scale
    g.close()


def test_planned_program_matches_oracle_and_decrypts_logN12():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o, cl, q = setup(12, si.workload_seed(4) + 2)
    prog = bt.plan(g.N, q, 2.0 ** 50)
    hkeys, dkeys = dev_keys(g, cl, prog.rot_steps)
    z = cl.random_slots()
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    got, sc = run_device(g, prog, dkeys, ct, len(q) - 15)
    # the same program (plaintexts reduced and transformed by the oracle) on the oracle
    from test_bootstrap_plan import as_eval_form
    ref = obt.run(o, as_eval_form(o, prog), ct, *hkeys)
    assert np.array_equal(got, ref)
    err = np.max(np.abs(cl.decrypt(got, sc) - z)) / max(1.0, np.max(np.abs(z)))
    print("bootstrap logN=12 relative slot error 2^%.2f" % np.log2(err))
    assert err < 2.0 ** -12, err
    g.close()


@pytest.mark.parametrize("logN", [15, 16])
def test_bootstrap_decrypts_at_full_size(logN):
    """logN=16 (2^15 slots) and logN=15 (2^14 slots), L=30 (q_0 60-bit, 29 x
    54-bit), K=10, dnum=3, h=192."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o, cl, q = setup(logN, si.workload_seed(4) + 3)
    prog = bt.plan(g.N, q, 2.0 ** 50)
    hkeys, dkeys = dev_keys(g, cl, prog.rot_steps)
    z = cl.random_slots()
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    got, sc = run_device(g, prog, dkeys, ct, len(q) - 15)
    err = np.max(np.abs(cl.decrypt(got, sc) - z)) / max(1.0, np.max(np.abs(z)))
    print("bootstrap logN=%d relative slot error 2^%.2f" % (logN, np.log2(err)))
    assert err < 2.0 ** -12, err
    g.close()


def test_oracle_sparse_program_on_the_device_is_bit_exact():
    """256 of 2048 slots: the trace (three ROT + HADD steps) and 256-point
    transforms, run by the executor, equal the oracle's run residue for
    residue, and the result decrypts to the repeated message."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o, cl, q = setup(12, si.workload_seed(4) + 5)
    prog = obt.plan(cl, q, 2.0 ** 50, slots=256)
    assert sum(1 for ins in prog.instr if ins[0] == obt.ROT) == 3
    hkeys, dkeys = dev_keys(g, cl, prog.rot_steps)
    z = np.tile(cl.random_slots()[:256], 8)
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    ref = obt.run(o, prog, ct, *hkeys)
    got, sc = run_device(g, prog, dkeys, ct, ref.shape[1])
    assert np.array_equal(got, ref)
    err = np.max(np.abs(cl.decrypt(got, sc) - z)) / max(1.0, np.max(np.abs(z)))
    assert err < 2.0 ** -12, err
    g.close()


@pytest.mark.parametrize("slots", [1 << 14, 512, 64])
def test_sparse_bootstrap_decrypts_at_full_size(slots):
    """logN=16 with the slot counts of the paper's Table IV below 2^15: the
    library's planned program refreshes a message repeated with that period
    within 2^-12 (h = 192, L = 30, K = 10, dnum = 3)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o, cl, q = setup(16, si.workload_seed(4) + 6)
    prog = bt.plan(g.N, q, 2.0 ** 50, slots=slots)
    hkeys, dkeys = dev_keys(g, cl, prog.rot_steps)
    z = np.tile(cl.random_slots()[:slots], (g.N // 2) // slots)
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    got, sc = run_device(g, prog, dkeys, ct, len(q) - 15)
    err = np.max(np.abs(cl.decrypt(got, sc) - z)) / max(1.0, np.max(np.abs(z)))
    print("sparse bootstrap logN=16, %d slots: relative slot error 2^%.2f" % (slots, np.log2(err)))
    assert err < 2.0 ** -12, err
    g.close()


def test_program_checks_before_running():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o, cl, q = setup(12, 5)
    prog = bt.BootProgram()
    prog.n_regs, prog.in_reg, prog.out_reg = 3, 0, 2
    prog.instr = [(bt.OP["RESCALE"], 2, 1, -1, 0)]          # reads register 1, never written
    with pytest.raises(FidesError):
        bt.DeviceProgram(g, prog, None, None, {}, in_limbs=5)
    prog.instr = [(bt.OP["HMULT"], 1, 0, 0, 0), (bt.OP["RESCALE"], 2, 1, -1, 0)]
    with pytest.raises(FidesError):                            # no relinearisation key
        bt.DeviceProgram(g, prog, None, None, {}, in_limbs=5)
    prog.instr = [(bt.OP["MODRAISE"], 1, 0, -1, 30), (bt.OP["RESCALE"], 2, 1, -1, 0)]
    with pytest.raises(FidesError):                            # ModRaise of a 5-limb input
        bt.DeviceProgram(g, prog, None, None, {}, in_limbs=5)
    g.close()
