"""Request server logic on the CPU (simulation mode: no device, a launch group
"runs" for sim_ns_per_limb x its limbs).  Covers admission by the memory
budget, arrival order, continuous batching across lanes, rejections before
launch, cancellation, the time-out watchdog and injected launch failures.
The same dispatcher drives the GPU executor; results on the device are
checked in test_gpu_server.py."""
import threading
import time

import pytest

from paper_2507_04775_gb300 import build as libbuild
from paper_2507_04775_gb300 import fides as F

LOGN, L, K, DNUM = 16, 30, 10, 3
N = 1 << LOGN
ALPHA = -(-L // DNUM)
A, B, KEY = 0x10000, 0x20000, 0x30000   # stand-in device addresses (never dereferenced in simulation)


@pytest.fixture(scope="module", autouse=True)
def built():
    libbuild.build()


def footprint(kind, nl):
    """Device bytes one request holds while it runs: its output ciphertext and
    the scratch of its key switch (input copy, coefficient form, beta digits
    of nl+K limbs, two accumulators, the 2K special limbs, 2 nl converted
    limbs); a Rescale holds two limbs of scratch.  256-byte granules."""
    limb = 8 * N
    rnd = lambda x: -(-x // 256) * 256
    if kind == F.OP_RESCALE:
        return rnd(2 * (nl - 1) * limb) + rnd(2 * limb)
    beta = -(-nl // ALPHA)
    scratch = (nl + nl + beta * (nl + K) + 2 * (nl + K) + 2 * K + 2 * nl) * limb
    return rnd(2 * nl * limb) + rnd(scratch)


def server(arena, **kw):
    kw.setdefault("n_lanes", 2)
    kw.setdefault("max_batch", 8)
    kw.setdefault("sim_ns_per_limb", 2000)
    s = F.Server(None, arena, simulate=True, shape=(LOGN, L, K, DNUM), **kw)
    s.set_relin_key(KEY)
    for k in (1, 2, 4, -1):
        s.add_rotation_key(k, KEY + k)
    return s


def drain(s, n, timeout=10.0, release=True):
    got, t0 = [], time.time()
    while len(got) < n:
        assert time.time() - t0 < timeout, "completions missing: %d of %d" % (len(got), n)
        for c in s.poll(timeout_us=20000):
            got.append(c)
            if release and c.status == 0:
                s.release(c.id)
    return got


def test_round_trip_and_memory_accounting():
    s = server(1 << 36)
    ids = [s.submit(F.OP_HMULT, A, 30, b=B, scale_a=2.0 ** 40, scale_b=2.0 ** 40),
           s.submit(F.OP_ROTATE, A, 17, steps=4, scale_a=2.0 ** 40),
           s.submit(F.OP_RESCALE, A, 12, scale_a=2.0 ** 80)]
    got = {c.id: c for c in drain(s, 3, release=False)}
    assert sorted(got) == ids
    assert all(c.status == 0 and c.ptr is None for c in got.values())   # simulation computes nothing
    assert [got[i].n_limbs for i in ids] == [30, 17, 11]
    assert [got[i].type for i in ids] == [F.OP_HMULT, F.OP_ROTATE, F.OP_RESCALE]
    st = s.stats()
    outs = 2 * (30 + 17 + 11) * 8 * N
    assert st["held"] == 3 and st["arena_used"] == outs        # outputs stay until released
    assert st["arena_peak"] >= max(footprint(F.OP_HMULT, 30), footprint(F.OP_ROTATE, 17))
    for i in ids:
        s.release(i)
    with pytest.raises(F.FidesError) as e:
        s.release(ids[0])                                       # released twice
    assert e.value.code == F.ERR_ARG
    st = s.stats()
    assert st["arena_used"] == 0 and st["held"] == 0 and st["completed"] == 3
    for c in got.values():
        assert c.t_submit_ns <= c.t_admit_ns <= c.t_launch_ns <= c.t_done_ns
    s.close()


def test_rejections_are_reported_before_anything_is_queued():
    s = F.Server(None, footprint(F.OP_HMULT, 30), simulate=True, shape=(LOGN, L, K, DNUM), max_pending=2)
    cases = [
        (dict(kind=F.OP_HMULT, a=A, n_limbs=10, b=B), F.ERR_KEY),          # no relinearisation key yet
        (dict(kind=F.OP_ROTATE, a=A, n_limbs=10, steps=3), F.ERR_KEY),      # no rotation key
    ]
    for kw, code in cases:
        with pytest.raises(F.FidesError) as e:
            s.submit(**kw)
        assert e.value.code == code
    s.set_relin_key(KEY)
    s.add_rotation_key(3, KEY)
    bad = [
        dict(kind=F.OP_HMULT, a=A, n_limbs=0, b=B),
        dict(kind=F.OP_HMULT, a=A, n_limbs=L + 1, b=B),
        dict(kind=F.OP_HMULT, a=A, n_limbs=5),                              # no b
        dict(kind=F.OP_RESCALE, a=A, n_limbs=1),
        dict(kind=F.OP_RESCALE, a=0, n_limbs=5),                            # NULL input
        dict(kind=7, a=A, n_limbs=5),
    ]
    for kw in bad:
        with pytest.raises(F.FidesError) as e:
            s.submit(**kw)
        assert e.value.code == F.ERR_ARG
    # rotation by 3 + N/2 is the same automorphism as by 3
    s.pause(True)
    s.submit(F.OP_ROTATE, A, 10, steps=3 + N // 2)
    s.submit(F.OP_RESCALE, A, 10)
    with pytest.raises(F.FidesError) as e:
        s.submit(F.OP_RESCALE, A, 10)                                      # max_pending = 2
    assert e.value.code == F.ERR_BUSY
    st = s.stats()
    assert st["pending"] == 2 and st["rejected"] == len(cases) + len(bad) + 1 and st["submitted"] == 2
    s.close()
    # a request larger than the whole arena can never run
    s = server(footprint(F.OP_HMULT, 20))
    with pytest.raises(F.FidesError) as e:
        s.submit(F.OP_HMULT, A, 21, b=B)
    assert e.value.code == F.ERR_NOMEM
    s.submit(F.OP_HMULT, A, 20, b=B)
    drain(s, 1)
    s.close()


def test_budget_bounds_admission_and_the_queue_keeps_arrival_order():
    fp = footprint(F.OP_HMULT, 30)
    s = server(2 * fp + 4096, n_lanes=4, max_batch=8, sim_ns_per_limb=20000)   # room for two requests
    ids = [s.submit(F.OP_HMULT, A, 30, b=B) for _ in range(7)]
    got = drain(s, 7)
    st = s.stats()
    assert st["arena_peak"] <= st["arena_bytes"]
    assert st["admission_stalls"] >= 1
    assert max(c.group_ops for c in got) <= 2
    by_id = sorted(got, key=lambda c: c.id)
    assert [c.id for c in by_id] == ids
    launches = [c.t_launch_ns for c in by_id]
    assert launches == sorted(launches)                                   # no overtaking
    assert st["arena_used"] == 0
    s.close()


def test_groups_form_while_lanes_are_busy():
    s = server(1 << 40, n_lanes=1, max_batch=4, sim_ns_per_limb=0)
    s.pause(True)
    ids = [s.submit(F.OP_ROTATE, A, 8, steps=1) for _ in range(10)]
    s.pause(False)
    got = sorted(drain(s, 10), key=lambda c: c.id)
    assert [c.group_ops for c in got] == [4] * 8 + [2] * 2
    st = s.stats()
    assert st["groups"] == 3 and st["grouped_ops"] == 10 and st["max_group"] == 4
    s.close()


def test_continuous_batching_overlaps_lanes():
    # a group of one 30-limb request runs 30 ms; a request arriving meanwhile
    # starts at once on the second lane; arrivals while both lanes are busy
    # are launched together when the first lane frees
    s = server(1 << 40, n_lanes=2, max_batch=16, sim_ns_per_limb=1_000_000)
    first = s.submit(F.OP_HMULT, A, 30, b=B)
    time.sleep(0.005)
    second = s.submit(F.OP_HMULT, A, 30, b=B)
    time.sleep(0.005)
    rest = [s.submit(F.OP_ROTATE, A, 2, steps=2) for _ in range(5)]
    got = {c.id: c for c in drain(s, 7)}
    assert got[second].t_launch_ns < got[first].t_done_ns                 # overlap on two lanes
    assert got[first].lane != got[second].lane
    assert all(got[r].group_ops == 5 for r in rest)                       # one group for the five
    assert got[rest[0]].t_launch_ns >= got[first].t_done_ns
    assert s.stats()["max_lanes_busy"] == 2
    s.close()


def test_cancel_only_while_queued():
    s = server(1 << 40, n_lanes=1, sim_ns_per_limb=0)
    s.pause(True)
    ids = [s.submit(F.OP_RESCALE, A, 5) for _ in range(3)]
    s.cancel(ids[1])
    with pytest.raises(F.FidesError) as e:
        s.cancel(ids[1])
    assert e.value.code == F.ERR_BUSY
    s.pause(False)
    got = {c.id: c for c in drain(s, 3)}
    assert got[ids[1]].status == F.ERR_CANCELLED and got[ids[1]].lane == -1
    assert got[ids[0]].status == 0 and got[ids[2]].status == 0
    with pytest.raises(F.FidesError):
        s.cancel(ids[0])                                                   # already done
    st = s.stats()
    assert st["cancelled"] == 1 and st["completed"] == 2 and st["arena_used"] == 0
    s.close()


def test_watchdog_reports_a_stalled_group_and_reclaims_it_later():
    s = server(1 << 40, n_lanes=1, timeout_us=3000, sim_ns_per_limb=1000)
    s.inject(F.FAULT_STALL, 60000)                  # the next group's completion is hidden for 60 ms
    rid = s.submit(F.OP_HMULT, A, 10, b=B)
    t0 = time.time()
    c = drain(s, 1, release=False)[0]
    assert c.id == rid and c.status == F.ERR_TIMEOUT and c.ptr is None
    assert time.time() - t0 < 0.05                  # reported by the watchdog, before the stall ends
    assert s.stats()["arena_used"] > 0              # memory held while the device may still use it
    with pytest.raises(F.FidesError):
        s.release(rid)
    nxt = s.submit(F.OP_RESCALE, A, 4)              # queued behind the stalled lane
    c2 = drain(s, 1)[0]
    assert c2.id == nxt and c2.status == 0
    st = s.stats()
    assert st["timed_out"] == 1 and st["arena_used"] == 0
    s.close()


def test_injected_launch_failure_fails_its_group_only():
    s = server(1 << 40, n_lanes=1, sim_ns_per_limb=0)
    s.inject(F.FAULT_LAUNCH_ERROR, 1)
    s.pause(True)
    bad = [s.submit(F.OP_HMULT, A, 6, b=B), s.submit(F.OP_ROTATE, A, 6, steps=-1)]
    s.pause(False)
    got = drain(s, 2)
    assert sorted(c.id for c in got) == bad and all(c.status == F.ERR_CUDA for c in got)
    assert s.stats()["arena_used"] == 0
    ok = s.submit(F.OP_HMULT, A, 6, b=B)
    c = drain(s, 1)[0]
    assert c.id == ok and c.status == 0
    st = s.stats()
    assert st["failed"] == 2 and st["completed"] == 1
    s.close()


def test_concurrent_submitters_and_one_poller():
    s = server(1 << 40, n_lanes=3, max_batch=8, sim_ns_per_limb=200)
    ids, lock = [], threading.Lock()

    def client(k):
        for j in range(50):
            rid = s.submit([F.OP_HMULT, F.OP_ROTATE, F.OP_RESCALE][j % 3], A, 2 + (j + k) % 29, b=B, steps=1,
                           tag=1000 * k + j)
            with lock:
                ids.append(rid)

    th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = drain(s, 200)
    assert len(set(ids)) == 200 and sorted(c.id for c in got) == sorted(ids)
    assert sorted(c.tag for c in got) == sorted(1000 * k + j for k in range(4) for j in range(50))
    assert all(c.status == 0 for c in got)
    st = s.stats()
    assert st["completed"] == 200 and st["arena_used"] == 0 and st["pending"] == 0 and st["in_flight"] == 0
    s.close()


def test_destroy_with_queued_and_running_work_returns():
    s = server(1 << 40, n_lanes=1, sim_ns_per_limb=100000)
    s.submit(F.OP_HMULT, A, 30, b=B)
    s.pause(True)
    for _ in range(5):
        s.submit(F.OP_RESCALE, A, 5)
    t0 = time.time()
    s.close()
    assert time.time() - t0 < 5.0


def test_config_errors():
    with pytest.raises(F.FidesError):
        F.Server(None, 1 << 30)                                             # needs a context unless simulating
    for kw in (dict(n_lanes=0), dict(n_lanes=9), dict(max_batch=0), dict(max_batch=513), dict(max_pending=0)):
        with pytest.raises(F.FidesError):
            F.Server(None, 1 << 30, simulate=True, shape=(LOGN, L, K, DNUM), **kw)
    with pytest.raises(F.FidesError):
        F.Server(None, 1 << 30, simulate=True, shape=(LOGN, L, K, L + 1))
