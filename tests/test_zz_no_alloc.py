"""Rescale without allocation, checked against the regular Rescale.

fides_rescale_noalloc is for callers that cannot allocate device memory when
they call the library (a host application that owns every allocation, or a
service that reserves all device memory at start-up): its scratch is a static
device array instead of the context's pool.  This test calls it through the C
ABI twice in a row, on different inputs, and requires the same residues as
fides_rescale (bit for bit, the tolerance of every parity test here).  It
creates its own contexts, so it passes alone in a fresh process and after the
other tests.
"""
import ctypes

import numpy as np
import pytest

import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, find_primes, to_device, to_host  # noqa: E402
from paper_2507_04775_gb300.fides import fides_ct, lib  # noqa: E402


def _ct(t, n_limbs, scale=1.0):
    return fides_ct(t.data_ptr(), n_limbs, scale)


@pytest.mark.parametrize("P", [si.SMALL, si.FULL], ids=lambda P: P.name)
def test_rescale_noalloc_matches_rescale(P):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    ctx = Context(P.logN, q, p, P.dnum)
    N, nl = ctx.N, P.nq
    st = si.Stream(si.workload_seed(0), 77)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = lib()
    for call in range(2):
        a = np.stack([si.uniform_poly(st, q, N) for _ in range(2)])
        da = to_device(a)
        ref = torch.zeros(2 * (nl - 1) * N, dtype=torch.int64, device="cuda")
        got = torch.full_like(ref, -1)
        ca, cr, cg = _ct(da, nl, 2.0**80), _ct(ref, nl - 1), _ct(got, nl - 1)
        assert L.fides_rescale(ctx._h, ctypes.byref(ca), ctypes.byref(cr), stream) == 0
        assert L.fides_rescale_noalloc(ctx._h, ctypes.byref(ca), ctypes.byref(cg), stream) == 0, \
            L.fides_last_error()
        torch.cuda.synchronize()
        assert cg.scale == cr.scale == 2.0**80 / q[nl - 1]
        assert np.array_equal(to_host(got), to_host(ref)), "call %d differs" % call
    ctx.close()
