"""GPU: the request server gives every request the same residues alone and in
a mix of concurrent requests at other levels (continuous batching over
several lanes, outputs and scratch reused from the arena), and those residues
are the single-operation path's and the oracle's.  Host-side fault injection
(a failed launch, a hidden completion caught by the watchdog) leaves the
server serving correct results."""
import time

import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import (OP_HMULT, OP_RESCALE, OP_ROTATE, Context, Server, find_primes,  # noqa: E402
                                    to_device, to_host)
from paper_2507_04775_gb300 import fides as F  # noqa: E402

STEPS = (1, -1, 3)


def make_pair(P):
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    return Context(P.logN, q, p, P.dnum), oracle.Context(P.logN, q, p, P.dnum)


def rand_ct(st, o, nl):
    return np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])


def rand_key(st, o):
    return np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])


class Workload:
    """Resident keys and operand ciphertexts (two per level) and a seeded list
    of requests over them."""

    def __init__(self, P, levels, n_req, seed):
        self.g, self.o = make_pair(P)
        st = si.Stream(seed, 1)
        self.rlk = rand_key(st, self.o)
        self.rk = {k: rand_key(st, self.o) for k in STEPS}
        self.d_rlk = self.g.relin_key(to_device(self.rlk))
        self.d_rk = {k: self.g.rotation_key(to_device(v), k) for k, v in self.rk.items()}
        self.pool = {nl: [rand_ct(st, self.o, nl) for _ in range(2)] for nl in levels}
        self.d_pool = {nl: [to_device(c) for c in cts] for nl, cts in self.pool.items()}
        self.reqs = []
        for i in range(n_req):
            nl = levels[st.below(len(levels))]
            kind = (OP_HMULT, OP_ROTATE, OP_RESCALE)[st.below(3)]
            if kind == OP_RESCALE and nl < 2:
                kind = OP_ROTATE
            self.reqs.append((kind, nl, st.below(2), STEPS[st.below(len(STEPS))]))

    def server(self, arena_bytes, **kw):
        s = Server(self.g, arena_bytes, **kw)
        s.set_relin_key(self.d_rlk)
        for k, v in self.d_rk.items():
            s.add_rotation_key(k, v)
        return s

    def submit(self, s, i):
        kind, nl, which, steps = self.reqs[i]
        a, b = self.d_pool[nl][which], self.d_pool[nl][1 - which]
        return s.submit(kind, a, nl, b=b if kind == OP_HMULT else None, steps=steps, tag=i,
                        scale_a=2.0 ** 40, scale_b=2.0 ** 40)

    def single_op(self, i):
        kind, nl, which, steps = self.reqs[i]
        a, b = self.d_pool[nl][which], self.d_pool[nl][1 - which]
        N = self.o.N
        if kind == OP_HMULT:
            out = torch.zeros(2 * nl * N, dtype=torch.int64, device="cuda")
            self.g.hmult(a, b, nl, self.d_rlk, out)
        elif kind == OP_ROTATE:
            out = torch.zeros(2 * nl * N, dtype=torch.int64, device="cuda")
            self.g.rotate(a, nl, steps, self.d_rk[steps], out)
        else:
            out = torch.zeros(2 * (nl - 1) * N, dtype=torch.int64, device="cuda")
            self.g.rescale(a, nl, out)
        torch.cuda.synchronize()
        return to_host(out)

    def oracle(self, i):
        kind, nl, which, steps = self.reqs[i]
        a, b = self.pool[nl][which], self.pool[nl][1 - which]
        if kind == OP_HMULT:
            return self.o.hmult(a, b, self.rlk)
        if kind == OP_ROTATE:
            return self.o.rotate(a, steps, self.rk[steps])
        return self.o.rescale(a)


def collect(s, n, results, timeout=60.0):
    """Polls n completions, copies each output to the host and releases it."""
    t0 = time.time()
    got = []
    while len(got) < n:
        assert time.time() - t0 < timeout, "missing completions"
        for c in s.poll(timeout_us=100000):
            got.append(c)
            if c.status == 0:
                results[c.tag] = to_host(c.tensor().clone())
                s.release(c.id)
    return got


def run_alone(w, s):
    out = {}
    for i in range(len(w.reqs)):
        w.submit(s, i)
        (c,) = collect(s, 1, out)
        assert c.status == 0 and c.group_ops == 1
    return out


def run_mixed(w, s):
    """Half the requests queued while admission is held, then released at
    once (groups of up to max_batch); the other half submitted while those
    groups run."""
    out = {}
    n = len(w.reqs)
    s.pause(True)
    for i in range(n // 2):
        w.submit(s, i)
    s.pause(False)
    for i in range(n // 2, n):
        w.submit(s, i)
    got = collect(s, n, out)
    assert all(c.status == 0 for c in got)
    return out, got


def test_server_results_identical_alone_and_in_the_mix_logN12():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = Workload(si.MID, [12, 11, 7, 4, 2, 1], 36, 601)
    s = w.server(256 << 20, n_lanes=3, max_batch=8)
    alone = run_alone(w, s)
    mixed, got = run_mixed(w, s)
    assert max(c.group_ops for c in got) > 1
    st = s.stats()
    assert st["completed"] == 72 and st["arena_used"] == 0 and st["kernel_launches"] > 0
    for i in range(len(w.reqs)):
        assert np.array_equal(alone[i], mixed[i]), i
        kind, nl = w.reqs[i][:2]
        out_nl = nl - 1 if kind == OP_RESCALE else nl
        assert np.array_equal(mixed[i], w.single_op(i)), i
        assert np.array_equal(mixed[i].reshape(2, out_nl, w.o.N), w.oracle(i)), i
    s.close()
    w.g.close()


def test_server_under_a_tight_budget_reuses_memory_correctly():
    """Room for two 12-limb requests: the queue waits for memory, groups are
    small, and every output still matches the single-op path."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = Workload(si.MID, [12, 9, 3], 24, 602)
    limb = 8 * w.o.N
    one = (2 * 12 + 12 + 12 + 3 * 16 + 2 * 16 + 2 * 4 + 2 * 12) * limb
    s = w.server(2 * one + 4096, n_lanes=3, max_batch=8)
    mixed, got = run_mixed(w, s)
    st = s.stats()
    assert st["arena_peak"] <= st["arena_bytes"] and st["admission_stalls"] >= 1
    for i in range(len(w.reqs)):
        assert np.array_equal(mixed[i], w.single_op(i)), i
    s.close()
    w.g.close()


def test_server_full_size_mix_matches_single_op():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = Workload(si.FULL, [30, 17, 4], 8, 603)
    s = w.server(8 << 30, n_lanes=2, max_batch=4)
    mixed, got = run_mixed(w, s)
    for i in range(len(w.reqs)):
        assert np.array_equal(mixed[i], w.single_op(i)), i
    i = next(k for k, r in enumerate(w.reqs) if r[0] == OP_HMULT)
    nl = w.reqs[i][1]
    assert np.array_equal(mixed[i].reshape(2, nl, w.o.N), w.oracle(i))
    s.close()
    w.g.close()


def test_server_injected_faults_on_the_device_path():
    """A group failed at launch (nothing enqueued) and a group whose completion
    is hidden past the watchdog: both are reported, their memory comes back,
    and the next requests are correct."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = Workload(si.MID, [12, 6], 6, 604)
    s = w.server(256 << 20, n_lanes=1, max_batch=4, timeout_us=20000)
    out = {}
    s.inject(F.FAULT_LAUNCH_ERROR, 1)
    w.submit(s, 0)
    (c,) = collect(s, 1, out)
    assert c.status == F.ERR_CUDA and s.stats()["arena_used"] == 0
    s.inject(F.FAULT_STALL, 200000)
    w.submit(s, 1)
    (c,) = collect(s, 1, out)
    assert c.status == F.ERR_TIMEOUT
    for i in range(2, 6):
        w.submit(s, i)
    collect(s, 4, out)
    for i in range(2, 6):
        assert np.array_equal(out[i], w.single_op(i)), i
    st = s.stats()
    assert st["failed"] == 1 and st["timed_out"] == 1 and st["arena_used"] == 0
    s.close()
    w.g.close()


def test_server_in_round_to_nearest_mode():
    """The context's round-to-nearest mode reaches the server's launch groups:
    every request in a mixed run equals the oracle in that mode (centred
    ModDown conversion, centred Rescale lift) and the single-op path."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = Workload(si.MID, [12, 10, 5, 2], 24, 605)
    w.g.set_rounding(True)
    w.o.set_rounding(True)
    s = w.server(256 << 20, n_lanes=2, max_batch=8)
    mixed, got = run_mixed(w, s)
    assert max(c.group_ops for c in got) > 1
    for i in range(len(w.reqs)):
        kind, nl = w.reqs[i][:2]
        out_nl = nl - 1 if kind == OP_RESCALE else nl
        assert np.array_equal(mixed[i].reshape(2, out_nl, w.o.N), w.oracle(i)), i
        assert np.array_equal(mixed[i], w.single_op(i)), i
    s.close()
    w.g.close()
