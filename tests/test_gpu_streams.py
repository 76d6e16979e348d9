"""Single-operation calls of one context on two registered streams at once
(fides_ctx_add_stream): each stream uses its own scratch pool, so HMult+relin
followed by Rescale on one stream and HRotate on the other, all queued before
any synchronisation, give the residues of the same calls made one at a time
on one stream, bit for bit, at logN=16 with 30 limbs.  The first concurrent
results are also compared with the oracle.  Registration is idempotent and
limited to 16 streams per context.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, FidesError, find_primes, to_device, to_host  # noqa: E402


def _pair(P):
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    return Context(P.logN, q, p, P.dnum), oracle.Context(P.logN, q, p, P.dnum)


def _key(st, o):
    return np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])


def test_two_registered_streams_match_one_stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.FULL
    g, o = _pair(P)
    N, nl, reps = o.N, P.nq, 4
    st = si.Stream(si.workload_seed(1), 91)
    rk, kk = _key(st, o), _key(st, o)
    rlk = g.relin_key(to_device(rk))
    steps = [1, 3, 1 << 12, -2]
    rot = {k: g.rotation_key(to_device(kk), k) for k in set(steps)}
    A = [np.stack([si.uniform_poly(st, o.q, N) for _ in range(2)]) for _ in range(reps)]
    B = [np.stack([si.uniform_poly(st, o.q, N) for _ in range(2)]) for _ in range(reps)]
    C = [np.stack([si.uniform_poly(st, o.q, N) for _ in range(2)]) for _ in range(reps)]
    dA, dB, dC = [to_device(x) for x in A], [to_device(x) for x in B], [to_device(x) for x in C]

    def outs():
        m = [torch.full((2 * nl * N,), -1, dtype=torch.int64, device="cuda") for _ in range(reps)]
        r = [torch.full((2 * (nl - 1) * N,), -1, dtype=torch.int64, device="cuda") for _ in range(reps)]
        t = [torch.full((2 * nl * N,), -1, dtype=torch.int64, device="cuda") for _ in range(reps)]
        return m, r, t

    # one at a time, on the current stream (the context's own pool)
    m1, r1, t1 = outs()
    for i in range(reps):
        s = g.hmult(dA[i], dB[i], nl, rlk, m1[i], 1.0, 1.0)
        g.rescale(m1[i], nl, r1[i], s)
        g.rotate(dC[i], nl, steps[i], rot[steps[i]], t1[i])
    torch.cuda.synchronize()

    # both chains queued at once on two registered streams
    s0, s1 = torch.cuda.Stream(), torch.cuda.Stream()
    g.add_stream(s0)
    g.add_stream(s1)
    g.add_stream(s0)                       # registering again is a no-op
    m2, r2, t2 = outs()
    ready = torch.cuda.Event()
    ready.record(torch.cuda.current_stream())   # outputs filled on the current stream
    s0.wait_event(ready)
    s1.wait_event(ready)
    for i in range(reps):
        s = g.hmult(dA[i], dB[i], nl, rlk, m2[i], 1.0, 1.0, stream=s0)
        g.rescale(m2[i], nl, r2[i], s, stream=s0)
        g.rotate(dC[i], nl, steps[i], rot[steps[i]], t2[i], stream=s1)
    torch.cuda.synchronize()
    for i in range(reps):
        assert torch.equal(m1[i], m2[i]), "HMult %d differs between one and two streams" % i
        assert torch.equal(r1[i], r2[i]), "Rescale %d differs between one and two streams" % i
        assert torch.equal(t1[i], t2[i]), "HRotate %d differs between one and two streams" % i
    assert np.array_equal(to_host(r2[0]).reshape(2, nl - 1, N), o.rescale(o.hmult(A[0], B[0], rk)))
    assert np.array_equal(to_host(t2[0]).reshape(2, nl, N), o.rotate(C[0], steps[0], kk))
    assert g.status() == 0
    g.close()


def test_stream_registration_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, _ = _pair(si.SMALL)
    streams = [torch.cuda.Stream() for _ in range(17)]
    for s in streams[:16]:
        g.add_stream(s)
    g.add_stream(streams[3])               # already registered
    with pytest.raises(FidesError):
        g.add_stream(streams[16])
    g.close()
