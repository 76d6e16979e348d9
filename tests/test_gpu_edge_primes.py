"""The library at the top of its prime range: every prime just below 2^61,
the bound its lazy ranges rely on (8q < 2^64 in the NTT butterflies; products
of residues below 2q, or sums of two products of canonical residues, below
2^(k+63) in the Barrett reduction of the tensor product and PtMult, k the bit
length of q; in the key inner product sums of up to 2^(63-k) digit products
take it, more take the 128-bit reduction).  At logN=12 (one-pass NTT) and
logN=14 (two passes), with residues drawn uniformly and with every residue at
q - 1 (the largest products), the NTT round trip, HMult+relin, PtMult,
Rescale and HRotate give the oracle's residues exactly.  HMult+relin and
PtMult are also checked at prime sizes from 20 to 49 bits.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, find_primes, to_device, to_host  # noqa: E402

# (logN, q limbs, special primes, dnum); at 61-bit primes the inner product of
# the first two sets (two and three digits) takes the Barrett form, the six
# digits of the third the 128-bit reduction
SETS = [(12, 4, 2, 2), (14, 3, 1, 3), (12, 6, 1, 6)]


@pytest.fixture(scope="module", params=SETS, ids=["logN12-L4-K2", "logN14-L3-K1", "logN12-L6-K1-dnum6"])
def pair(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    logN, nq, nk, dnum = request.param
    q = find_primes(logN, 61, nq)
    p = find_primes(logN, 61, nk, exclude=q)
    assert all((1 << 60) < x < (1 << 61) for x in list(q) + list(p))
    g = Context(logN, q, p, dnum)
    yield g, oracle.Context(logN, q, p, dnum)
    g.close()


def _top(primes, N, polys=None):
    """every residue at q - 1"""
    a = np.stack([np.full(N, int(x) - 1, dtype=np.uint64) for x in primes])
    return a if polys is None else np.stack([a] * polys)


def _inputs(o, st, extreme, nl):
    if extreme:
        ct = lambda: _top(o.q[:nl], o.N, 2)                       # noqa: E731
        key = np.stack([_top(o.primes, o.N, 2) for _ in range(o.dnum)])
        pt = _top(o.q[:nl], o.N)
    else:
        ct = lambda: np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])   # noqa: E731
        key = np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])
        pt = si.uniform_poly(st, o.q[:nl], o.N)
    return ct(), ct(), key, pt


@pytest.mark.parametrize("extreme", [False, True], ids=["uniform", "q-1"])
def test_ntt_round_trip(pair, extreme):
    g, o = pair
    n = len(o.primes)
    a = _top(o.primes, o.N) if extreme else si.uniform_poly(si.Stream(1101, 1), o.primes, o.N)
    d = to_device(a)
    g.ntt(d, 0, n)
    assert np.array_equal(to_host(d).reshape(a.shape), o.ntt_limbs(a, list(range(n))))
    g.intt(d, 0, n)
    assert np.array_equal(to_host(d).reshape(a.shape), a)


@pytest.mark.parametrize("extreme", [False, True], ids=["uniform", "q-1"])
def test_hmult_ptmult_rescale_rotate(pair, extreme):
    g, o = pair
    st = si.Stream(1102, 2)
    nl = len(o.q)
    a, b, key, pt = _inputs(o, st, extreme, nl)
    da, db = to_device(a), to_device(b)
    shape = (2, nl, o.N)

    rlk = g.relin_key(to_device(key))
    out = torch.zeros(2 * nl * o.N, dtype=torch.int64, device="cuda")
    s = g.hmult(da, db, nl, rlk, out, 1.0, 1.0)
    torch.cuda.synchronize()
    m = o.hmult(a, b, key)
    assert np.array_equal(to_host(out).reshape(shape), m)

    res = torch.zeros(2 * (nl - 1) * o.N, dtype=torch.int64, device="cuda")
    g.rescale(out, nl, res, s)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(res).reshape(2, nl - 1, o.N), o.rescale(m))

    pm = torch.zeros(2 * nl * o.N, dtype=torch.int64, device="cuda")
    g.ptmult(da, to_device(pt), nl, pm)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(pm).reshape(shape), o.ptmult(a, pt))

    for step in (1, -3):
        rk = g.rotation_key(to_device(key), step)
        rot = torch.zeros(2 * nl * o.N, dtype=torch.int64, device="cuda")
        g.rotate(da, nl, step, rk, rot)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(rot).reshape(shape), o.rotate(a, step, key)), "step %d" % step
    assert g.status() == 0


# the Barrett reduction shifts by k - 1 and its constant depends on k: one
# context per prime size, q and p primes of the same bit length, so that the
# tensor product, PtMult and the inner product see every shift; 48 and 49
# bits straddle the tensor-core conversion's two epilogues
@pytest.mark.parametrize("bits", [20, 31, 32, 33, 47, 48, 49])
def test_prime_sizes(bits):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    logN, nq, nk, dnum = 12, 4, 2, 2
    q = find_primes(logN, bits, nq)
    p = find_primes(logN, bits, nk, exclude=q)
    g, o = Context(logN, q, p, dnum), oracle.Context(logN, q, p, dnum)
    try:
        for extreme in (False, True):
            st = si.Stream(1103, bits)
            a, b, key, pt = _inputs(o, st, extreme, nq)
            da = to_device(a)
            shape = (2, nq, o.N)
            out = torch.zeros(2 * nq * o.N, dtype=torch.int64, device="cuda")
            g.hmult(da, to_device(b), nq, g.relin_key(to_device(key)), out, 1.0, 1.0)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(out).reshape(shape), o.hmult(a, b, key)), "hmult, %d bits" % bits
            pm = torch.zeros(2 * nq * o.N, dtype=torch.int64, device="cuda")
            g.ptmult(da, to_device(pt), nq, pm)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(pm).reshape(shape), o.ptmult(a, pt)), "ptmult, %d bits" % bits
        assert g.status() == 0
    finally:
        g.close()
