"""Rescale without allocation, checked against the oracle and the regular Rescale.

fides_rescale_noalloc is for callers that cannot allocate device memory when
they call the library (a host application that owns every allocation, or a
service that reserves all device memory at start-up): its scratch is a static
device array instead of the context's pool.  This test calls it through the C
ABI twice in a row, on different inputs, and requires the residues of the
oracle's Rescale (floor(x / q_l), bit for bit, the tolerance of every parity
test here) and of fides_rescale.  It also checks that the calls change no
device allocation, that a call on a second stream overlapping the regular
Rescale on the first gives correct results on both, and that a ring degree
above the array's size is refused.  It creates its own contexts, so it passes
alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, find_primes, to_device, to_host  # noqa: E402
from paper_2507_04775_gb300.fides import fides_ct, lib  # noqa: E402

ERR_UNSUPPORTED = -2


def _ct(t, n_limbs, scale=1.0):
    return fides_ct(t.data_ptr(), n_limbs, scale)


def _stream_ptr(s):
    return ctypes.c_void_p(s.cuda_stream)


@pytest.mark.parametrize("P", [si.SMALL, si.FULL], ids=lambda P: P.name)
def test_rescale_noalloc_matches_oracle_and_rescale(P):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    ctx = Context(P.logN, q, p, P.dnum)
    orc = oracle.Context(P.logN, q, p, P.dnum)
    N, nl = ctx.N, P.nq
    st = si.Stream(si.workload_seed(0), 77)
    s0 = torch.cuda.current_stream()
    stream = _stream_ptr(s0)
    L = lib()
    for call in range(2):
        a = np.stack([si.uniform_poly(st, q, N) for _ in range(2)])
        da = to_device(a)
        ref = torch.zeros(2 * (nl - 1) * N, dtype=torch.int64, device="cuda")
        got = torch.full_like(ref, -1)
        ca, cr, cg = _ct(da, nl, 2.0**80), _ct(ref, nl - 1), _ct(got, nl - 1)
        assert L.fides_rescale(ctx._h, ctypes.byref(ca), ctypes.byref(cr), stream) == 0
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert L.fides_rescale_noalloc(ctx._h, ctypes.byref(ca), ctypes.byref(cg), stream) == 0, \
            L.fides_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "call %d changed the device's free memory" % call
        assert cg.scale == cr.scale == 2.0**80 / q[nl - 1]
        want = orc.rescale(a)
        assert np.array_equal(to_host(got).reshape(2, nl - 1, N), want), "call %d differs from the oracle" % call
        assert np.array_equal(to_host(got), to_host(ref)), "call %d differs from fides_rescale" % call
    # the context's round-to-nearest mode applies here too
    ctx.set_rounding(True)
    a = np.stack([si.uniform_poly(st, q, N) for _ in range(2)])
    da = to_device(a)
    got = torch.full((2 * (nl - 1) * N,), -1, dtype=torch.int64, device="cuda")
    ca, cg = _ct(da, nl), _ct(got, nl - 1)
    assert L.fides_rescale_noalloc(ctx._h, ctypes.byref(ca), ctypes.byref(cg), stream) == 0, L.fides_last_error()
    torch.cuda.synchronize()
    assert np.array_equal(to_host(got).reshape(2, nl - 1, N), orc.rescale(a, nearest=True))
    ctx.close()


def test_rescale_noalloc_beside_the_regular_rescale():
    """A call on a second stream while the regular Rescale (which uses the
    context's scratch) runs on the first: both results are the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = si.MID
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    ctx = Context(P.logN, q, p, P.dnum)
    orc = oracle.Context(P.logN, q, p, P.dnum)
    N, nl = ctx.N, P.nq
    st = si.Stream(si.workload_seed(0), 78)
    L = lib()
    a = np.stack([si.uniform_poly(st, q, N) for _ in range(2)])
    b = np.stack([si.uniform_poly(st, q, N) for _ in range(2)])
    da, db = to_device(a), to_device(b)
    ra = torch.full((2 * (nl - 1) * N,), -1, dtype=torch.int64, device="cuda")
    rb = torch.full_like(ra, -1)
    s0, s1 = torch.cuda.current_stream(), torch.cuda.Stream()
    ready = torch.cuda.Event()
    ready.record(s0)                 # inputs and outputs are filled on s0
    s1.wait_event(ready)
    ca, cb = _ct(da, nl), _ct(db, nl)
    oa, ob = _ct(ra, nl - 1), _ct(rb, nl - 1)
    for _ in range(4):
        assert L.fides_rescale(ctx._h, ctypes.byref(ca), ctypes.byref(oa), _stream_ptr(s0)) == 0
        assert L.fides_rescale_noalloc(ctx._h, ctypes.byref(cb), ctypes.byref(ob), _stream_ptr(s1)) == 0, \
            L.fides_last_error()
    torch.cuda.synchronize()
    assert np.array_equal(to_host(ra).reshape(2, nl - 1, N), orc.rescale(a))
    assert np.array_equal(to_host(rb).reshape(2, nl - 1, N), orc.rescale(b))
    ctx.close()


def test_rescale_noalloc_refuses_a_ring_above_its_array():
    """N = 2^17 needs 2^18 scratch words; the array holds 2 x 65536."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q = find_primes(17, 54, 3)
    p = find_primes(17, 60, 1, exclude=q)
    ctx = Context(17, q, p, 3)
    N, nl = ctx.N, 3
    x = torch.zeros(2 * nl * N, dtype=torch.int64, device="cuda")
    y = torch.full((2 * (nl - 1) * N,), 7, dtype=torch.int64, device="cuda")
    L = lib()
    cx, cy = _ct(x, nl), _ct(y, nl - 1)
    rc = L.fides_rescale_noalloc(ctx._h, ctypes.byref(cx), ctypes.byref(cy),
                                 _stream_ptr(torch.cuda.current_stream()))
    assert rc == ERR_UNSUPPORTED
    assert b"static array" in L.fides_last_error()
    torch.cuda.synchronize()
    assert bool((y == 7).all()), "a refused call queued work"
    ctx.close()
