"""GPU parity of the batched path: a batch of HMult / HRotate / Rescale
operations at uneven levels, in two dependent stages, must give the same
residues as the same operations run one by one (single-op path) and as the CPU
oracle, with and without CUDA-graph capture."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import (OP_HMULT, OP_RESCALE, OP_ROTATE, Batch, Context, FidesError, Op,  # noqa: E402
                                    find_primes, to_device, to_host)


def make_pair(P):
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    return Context(P.logN, q, p, P.dnum), oracle.Context(P.logN, q, p, P.dnum)


def rand_ct(st, o, nl):
    return np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])


def rand_key(st, o):
    return np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])


def zeros(o, nl):
    return torch.zeros(2 * nl * o.N, dtype=torch.int64, device="cuda")


class RotKeys:
    """Rotation-key handles over one key buffer, one per rotation (parity does
    not depend on the key's values, only on its Galois element)."""

    def __init__(self, g, t):
        self.g, self.t, self.keys = g, t, {}

    def __call__(self, steps):
        e = self.g.galois_elt(steps)
        if e not in self.keys:
            self.keys[e] = self.g.rotation_key(self.t, steps)
        return self.keys[e]


def build_case(P, levels, seed):
    """Stage 0: HMult of (a_i, b_i) at each level, HRotate of a_i, Rescale of
    a_i; stage 1: HRotate and Rescale of every stage-0 product."""
    g, o = make_pair(P)
    st = si.Stream(seed, 1)
    rlk, rk = rand_key(st, o), rand_key(st, o)
    drlk, drk = g.relin_key(to_device(rlk)), RotKeys(g, to_device(rk))
    host, ops = [], []
    for i, nl in enumerate(levels):
        a, b = rand_ct(st, o, nl), rand_ct(st, o, nl)
        da, db = to_device(a), to_device(b)
        steps = [1, -2, 7, 1 << (P.logN - 2)][i % 4]
        m = Op(OP_HMULT, da, nl, zeros(o, nl), b=db, key=drlk, stage=0, scale_a=2.0**40, scale_b=2.0**40)
        r = Op(OP_ROTATE, da, nl, zeros(o, nl), key=drk(steps), steps=steps, stage=0, scale_a=2.0**40)
        ops += [m, r]
        entry = {"nl": nl, "a": a, "b": b, "steps": steps, "m": m, "r": r}
        if nl >= 2:
            entry["s"] = Op(OP_RESCALE, da, nl, zeros(o, nl - 1), stage=0, scale_a=2.0**40)
            entry["ms"] = Op(OP_RESCALE, m.out, nl, zeros(o, nl - 1), stage=1, scale_a=2.0**80)
            ops += [entry["s"], entry["ms"]]
        entry["mr"] = Op(OP_ROTATE, m.out, nl, zeros(o, nl), key=drk(3), steps=3, stage=1, scale_a=2.0**80)
        ops.append(entry["mr"])
        host.append(entry)
    return g, o, rlk, rk, drlk, drk, host, ops


def single_op_reference(g, host, drlk, drk):
    """The same operations through the single-op entry points."""
    ref = []
    for e in host:
        nl = e["nl"]
        da, db = to_device(e["a"]), to_device(e["b"])
        m, r, mr = zeros(g, nl), zeros(g, nl), zeros(g, nl)
        g.hmult(da, db, nl, drlk, m)
        g.rotate(da, nl, e["steps"], drk(e["steps"]), r)
        g.rotate(m, nl, 3, drk(3), mr)
        d = {"m": m, "r": r, "mr": mr}
        if nl >= 2:
            s, ms = zeros(g, nl - 1), zeros(g, nl - 1)
            g.rescale(da, nl, s)
            g.rescale(m, nl, ms)
            d["s"], d["ms"] = s, ms
        ref.append(d)
    return ref


@pytest.mark.parametrize("P,levels", [(si.MID, [12, 5, 1, 9, 4]), (si.SMALL, [3, 1, 2])],
                         ids=["logN12-L12", "logN12-L3"])
def test_batch_matches_single_op_and_oracle(P, levels):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o, rlk, rk, drlk, drk, host, ops = build_case(P, levels, 501)
    batch = Batch(g, ops)
    info = batch.info()
    assert info["launches"] > 0 and info["scratch_bytes"] > 0
    batch.run()
    torch.cuda.synchronize()
    ref = single_op_reference(g, host, drlk, drk)
    torch.cuda.synchronize()
    for e, r in zip(host, ref):
        for k in ("m", "r", "mr", "s", "ms"):
            if k in r:
                assert np.array_equal(to_host(e[k].out), to_host(r[k])), (e["nl"], k)
        nl = e["nl"]
        assert np.array_equal(to_host(e["m"].out).reshape(2, nl, o.N), o.hmult(e["a"], e["b"], rlk))
        assert np.array_equal(to_host(e["r"].out).reshape(2, nl, o.N), o.rotate(e["a"], e["steps"], rk))
        assert e["m"].out_scale == 2.0**80 and e["r"].out_scale == 2.0**40
        if nl >= 2:
            assert e["ms"].out_scale == 2.0**80 / o.q[nl - 1]
    batch.close()
    g.close()


@pytest.mark.parametrize("group_limbs,tensor_split,prime_order", [(1, 1, 0), (8, 0, 1), (20, 1, 1), (0, 0, 0)])
def test_batch_launch_groups_and_tensor_placement(group_limbs, tensor_split, prime_order):
    """The same batch planned as launch groups of at most group_limbs limbs
    (one op per group at 1; several groups per stage sharing one scratch pool)
    and with the tensor product fused or as its own pass: residues equal the
    single-op path's and the oracle's; smaller groups need less scratch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.MID
    g, o, rlk, rk, drlk, drk, host, ops = build_case(P, [12, 5, 1, 9, 4, 12], 503)
    batch = Batch(g, ops)
    whole = batch.info()
    batch.configure(group_limbs, tensor_split, prime_order)
    info = batch.info()
    assert info["group_limbs"] == group_limbs and info["tensor_split"] == tensor_split
    assert info["prime_order"] == prime_order
    if group_limbs:
        assert info["groups"] > whole["groups"] and info["scratch_bytes"] < whole["scratch_bytes"]
    for op in ops:
        op.out.fill_(-1)
    batch.run()
    torch.cuda.synchronize()
    ref = single_op_reference(g, host, drlk, drk)
    torch.cuda.synchronize()
    for e, r in zip(host, ref):
        for k in ("m", "r", "mr", "s", "ms"):
            if k in r:
                assert np.array_equal(to_host(e[k].out), to_host(r[k])), (e["nl"], k)
    e = host[0]
    assert np.array_equal(to_host(e["m"].out).reshape(2, e["nl"], o.N), o.hmult(e["a"], e["b"], rlk))
    batch.close()
    g.close()


def test_batch_in_round_to_nearest_mode():
    """A batch planned in round-to-nearest mode (centred ModDown conversion,
    centred Rescale lift) equals the single-op path and the oracle in the
    same mode."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.MID
    g, o, rlk, rk, drlk, drk, host, ops = build_case(P, [12, 5, 9, 2], 505)
    g.set_rounding(True)
    o.set_rounding(True)
    batch = Batch(g, ops)
    batch.configure(16, 1, 1)
    batch.run()
    torch.cuda.synchronize()
    ref = single_op_reference(g, host, drlk, drk)
    torch.cuda.synchronize()
    for e, r in zip(host, ref):
        for k in ("m", "r", "mr", "s", "ms"):
            if k in r:
                assert np.array_equal(to_host(e[k].out), to_host(r[k])), (e["nl"], k)
        nl = e["nl"]
        prod = o.hmult(e["a"], e["b"], rlk)
        assert np.array_equal(to_host(e["m"].out).reshape(2, nl, o.N), prod)
        assert np.array_equal(to_host(e["ms"].out).reshape(2, nl - 1, o.N), o.rescale(prod))
        assert np.array_equal(to_host(e["mr"].out).reshape(2, nl, o.N), o.rotate(prod, 3, rk))
    batch.close()
    g.close()


def test_batch_autotune_keeps_results():
    """The autotuner picks a grouping and tensor placement by timing them on
    the batch; the chosen plan still computes the oracle's residues, also
    replayed from a captured graph."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.FULL
    g, o, rlk, rk, drlk, drk, host, ops = build_case(P, [30, 7, 4, 16], 504)
    batch = Batch(g, ops)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ms = batch.autotune(s)
        for op in ops:
            op.out.zero_()
        batch.capture(s)
        batch.run(s)
    s.synchronize()
    info = batch.info()
    assert ms > 0 and info["groups"] >= 2
    e = host[1]
    nl = e["nl"]
    prod = o.hmult(e["a"], e["b"], rlk)
    assert np.array_equal(to_host(e["m"].out).reshape(2, nl, o.N), prod)
    assert np.array_equal(to_host(e["mr"].out).reshape(2, nl, o.N), o.rotate(prod, 3, rk))
    assert np.array_equal(to_host(e["r"].out).reshape(2, nl, o.N), o.rotate(e["a"], e["steps"], rk))
    batch.close()
    g.close()


def test_batch_graph_capture_full_size():
    """logN=16, 30-limb chain at uneven levels, captured in a CUDA graph and
    replayed twice: identical to the oracle and to the uncaptured run."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.FULL
    g, o, rlk, rk, drlk, drk, host, ops = build_case(P, [30, 17, 4], 502)
    batch = Batch(g, ops)
    batch.run()
    torch.cuda.synchronize()
    first = [to_host(op.out).copy() for op in ops]
    for op in ops:
        op.out.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())   # the zeroing above runs on the current stream
    with torch.cuda.stream(s):
        batch.capture(s)
        batch.run(s)
        batch.run(s)
    s.synchronize()
    for op, f in zip(ops, first):
        assert np.array_equal(to_host(op.out), f)
    e = host[1]
    nl = e["nl"]
    prod = o.hmult(e["a"], e["b"], rlk)
    assert np.array_equal(to_host(e["m"].out).reshape(2, nl, o.N), prod)
    assert np.array_equal(to_host(e["mr"].out).reshape(2, nl, o.N), o.rotate(prod, 3, rk))
    assert np.array_equal(to_host(e["ms"].out).reshape(2, nl - 1, o.N), o.rescale(prod))
    batch.close()
    g.close()


def test_batch_rejects_bad_ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = make_pair(si.SMALL)
    a = zeros(o, 3)
    with pytest.raises(FidesError) as e:
        Batch(g, [Op(OP_HMULT, a, 3, zeros(o, 3), b=None, key=None)])
    assert e.value.code == -1
    with pytest.raises(FidesError):
        Batch(g, [Op(OP_RESCALE, a, 1, zeros(o, 1))])
    g.close()


def test_batch_with_more_conversion_jobs_than_sms():
    """72 HMults at logN=12 with 12 limbs (three digits each): the batch's
    ModUp conversion launch has 216 jobs, more than the GPU has SMs, so its
    launcher splits each job's tiles over several CTAs in several waves.
    Every product equals the single-op HMult's, and two equal the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.MID
    g, o = make_pair(P)
    st = si.Stream(503, 1)
    rlk = rand_key(st, o)
    drlk = g.relin_key(to_device(rlk))
    nl, n = P.nq, 72
    pairs = [(rand_ct(st, o, nl), rand_ct(st, o, nl)) for _ in range(n)]
    dev = [(to_device(a), to_device(b)) for a, b in pairs]
    ops = [Op(OP_HMULT, da, nl, zeros(o, nl), b=db, key=drlk, stage=0) for da, db in dev]
    batch = Batch(g, ops)
    batch.run()
    torch.cuda.synchronize()
    for (da, db), op in zip(dev, ops):
        ref = zeros(o, nl)
        g.hmult(da, db, nl, drlk, ref)
        torch.cuda.synchronize()
        assert torch.equal(op.out, ref)
    for i in (0, n - 1):
        a, b = pairs[i]
        assert np.array_equal(to_host(ops[i].out).reshape(2, nl, o.N), o.hmult(a, b, rlk))
    assert g.status() == 0
    batch.close()
    g.close()
