"""GPU parity at the other ring degrees (logN 13, 14, 15, 17: two-pass NTTs
whose passes are not multiples of four stages, so their last register round is
partial): the NTT with every compiled tile variant, and HMult+relin, HRotate,
Rescale and the fused HMult+Rescale, residue for residue against the oracle."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, find_primes, to_device, to_host  # noqa: E402

NQ, NK, DNUM = 6, 2, 3


@pytest.fixture(scope="module", params=[13, 14, 15, 17])
def pair(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    logN = request.param
    q = find_primes(logN, 54, NQ)
    p = find_primes(logN, 60, NK, exclude=q)
    g, o = Context(logN, q, p, DNUM), oracle.Context(logN, q, p, DNUM)
    yield logN, g, o
    g.close()


def rand_key(st, o):
    return np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])


def test_ntt_every_variant(pair):
    logN, g, o = pair
    st = si.Stream(1200 + logN)
    n = len(o.primes)
    a = si.uniform_poly(st, o.primes, o.N)
    idx = list(range(n))
    ref = o.ntt_limbs(a, idx)
    table = g.tune_table()
    for v in range(5):
        g.set_tune_table(bytes([v]) * len(table))
        d = to_device(a)
        g.ntt(d, 0, n)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(d).reshape(n, o.N), ref), "forward, variant %d" % v
        g.intt(d, 0, n)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(d).reshape(n, o.N), a), "inverse, variant %d" % v
    g.set_tune_table(table)


def test_key_switching_ops(pair):
    logN, g, o = pair
    st = si.Stream(1300 + logN)
    rlk, rk = rand_key(st, o), rand_key(st, o)
    drlk, drk = g.relin_key(to_device(rlk)), g.rotation_key(to_device(rk), 3)
    for nl in (NQ, 3):
        a = np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])
        b = np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])
        da, db = to_device(a), to_device(b)
        m, r = torch.empty_like(da), torch.empty_like(da)
        s = torch.empty(2 * (nl - 1) * o.N, dtype=torch.int64, device="cuda")
        hr = torch.empty(2 * (nl - 1) * o.N, dtype=torch.int64, device="cuda")
        g.hmult(da, db, nl, drlk, m)
        g.rotate(da, nl, 3, drk, r)
        g.rescale(da, nl, s)
        g.hmult_rescale(da, db, nl, drlk, hr)
        torch.cuda.synchronize()
        ref_m = o.hmult(a, b, rlk)
        assert np.array_equal(to_host(m).reshape(a.shape), ref_m), nl
        assert np.array_equal(to_host(r).reshape(a.shape), o.rotate(a, 3, rk)), nl
        assert np.array_equal(to_host(s).reshape(2, nl - 1, o.N), o.rescale(a)), nl
        assert np.array_equal(to_host(hr).reshape(2, nl - 1, o.N), o.rescale(ref_m)), nl


def test_autotune_runs(pair):
    logN, g, o = pair
    g.autotune(8)
    st = si.Stream(1400 + logN)
    a = si.uniform_poly(st, o.primes, o.N)
    n = len(o.primes)
    d = to_device(a)
    g.ntt(d, 0, n)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d).reshape(n, o.N), o.ntt_limbs(a, list(range(n))))
