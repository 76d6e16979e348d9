"""GPU parity of the remaining Table I operations and of hoisted rotations:
HAdd, HSub, PtAdd, PtMult, ScalarAdd, ScalarMult (element-wise kernel, 16- and
8-byte-aligned paths, in place), HSquare, Conjugate, and n rotations sharing
one ModUp -- every residue equal to the oracle's."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, FidesError, find_primes, to_device, to_host  # noqa: E402


def make_pair(P):
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    return Context(P.logN, q, p, P.dnum), oracle.Context(P.logN, q, p, P.dnum)


def rand_ct(st, o, nl):
    return np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])


def rand_key(st, o):
    return np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])


def dev_misaligned(x):
    """A device copy of x that starts 8 bytes past a 16-byte boundary."""
    flat = np.ascontiguousarray(x, dtype=np.uint64).reshape(-1)
    buf = torch.zeros(flat.size + 1, dtype=torch.int64, device="cuda")
    buf[1:] = to_device(flat)
    return buf[1:]


CASES = [(si.SMALL, 3), (si.MID, 12), (si.MID, 5), (si.FULL, 30), (si.FULL, 7)]
IDS = ["logN12-L3", "logN12-L12", "logN12-L5of12", "logN16-L30", "logN16-L7of30"]


@pytest.fixture(scope="module")
def pairs():
    cache = {}

    def get(P):
        if P.name not in cache:
            cache[P.name] = make_pair(P)
        return cache[P.name]
    yield get
    for g, _ in cache.values():
        g.close()


@pytest.mark.parametrize("P,nl", CASES, ids=IDS)
def test_elementwise_ops_match_oracle(pairs, P, nl):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = pairs(P)
    st = si.Stream(801, nl)
    a, b = rand_ct(st, o, nl), rand_ct(st, o, nl)
    pt = si.uniform_poly(st, o.q[:nl], o.N)
    k = np.array([int(st.below(q)) for q in o.q[:nl]], dtype=np.uint64)
    da, db, dpt = to_device(a), to_device(b), to_device(pt)
    shape = (2, nl, o.N)

    def run(fn, *args, **kw):
        out = torch.empty(2 * nl * o.N, dtype=torch.int64, device="cuda")
        fn(*args, out=out, **kw)
        torch.cuda.synchronize()
        return to_host(out).reshape(shape)

    assert np.array_equal(run(lambda out: g.hadd(da, db, nl, out)), o.hadd(a, b))
    assert np.array_equal(run(lambda out: g.hsub(da, db, nl, out)), o.hsub(a, b))
    assert np.array_equal(run(lambda out: g.ptadd(da, dpt, nl, out)), o.ptadd(a, pt))
    assert np.array_equal(run(lambda out: g.ptmult(da, dpt, nl, out)), o.ptmult(a, pt))
    assert np.array_equal(run(lambda out: g.scalar_add(da, k, nl, out)), o.scalar_add(a, k))
    assert np.array_equal(run(lambda out: g.scalar_mult(da, k, nl, out)), o.scalar_mult(a, k))
    # 8-byte-aligned buffers take the scalar-load path
    ma, mb, mpt = dev_misaligned(a), dev_misaligned(b), dev_misaligned(pt)
    out = dev_misaligned(np.zeros(shape, dtype=np.uint64))
    g.ptmult(ma, mpt, nl, out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out).reshape(shape), o.ptmult(a, pt))
    g.hsub(ma, mb, nl, out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out).reshape(shape), o.hsub(a, b))
    # in place: out aliases a
    inplace = to_device(a)
    g.hadd(inplace, db, nl, inplace)
    g.scalar_mult(inplace, k, nl, inplace)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(inplace).reshape(shape), o.scalar_mult(o.hadd(a, b), k))


def test_scale_bookkeeping_and_argument_errors(pairs):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = pairs(si.SMALL)
    nl = o.nq
    x = torch.zeros(2 * nl * o.N, dtype=torch.int64, device="cuda")
    pt = torch.zeros(nl * o.N, dtype=torch.int64, device="cuda")
    assert g.ptmult(x, pt, nl, x.clone(), scale=2.0 ** 40, pt_scale=2.0 ** 30) == 2.0 ** 70
    assert g.scalar_mult(x, 3, nl, x.clone(), scale=2.0 ** 40, k_scale=1.0) == 2.0 ** 40
    assert g.hadd(x, x, nl, x.clone(), scale=2.0 ** 40) == 2.0 ** 40
    with pytest.raises(FidesError):
        g.scalar_add(x, [o.q[0], 0, 0], nl, x.clone())          # residue not below q_0
    with pytest.raises(FidesError):
        g.hadd(x, x, 0, x.clone())                               # no limbs


@pytest.mark.parametrize("P,nl", [(si.SMALL, 3), (si.MID, 9), (si.FULL, 30)], ids=["logN12-L3", "logN12-L9", "logN16-L30"])
def test_hsquare_and_conjugate_match_oracle(pairs, P, nl):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = pairs(P)
    st = si.Stream(802, nl)
    a = rand_ct(st, o, nl)
    rlk, ck = rand_key(st, o), rand_key(st, o)
    da = to_device(a)
    sq, cj = torch.empty_like(da), torch.empty_like(da)
    g.hsquare(da, nl, g.relin_key(to_device(rlk)), sq)
    g.conjugate(da, nl, g.conjugation_key(to_device(ck)), cj)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(sq).reshape(a.shape), o.hsquare(a, rlk))
    assert np.array_equal(to_host(cj).reshape(a.shape), o.conjugate(a, ck))


@pytest.mark.parametrize("P,nl,steps", [(si.SMALL, 3, [1, 2, -1]), (si.MID, 12, [3, -7, 1, 0]), (si.MID, 5, [2, 9]),
                                        (si.MID, 1, [1]), (si.FULL, 30, [1, 4, -3]), (si.FULL, 11, [1 << 13, 5])],
                         ids=["logN12-L3", "logN12-L12", "logN12-L5", "logN12-L1", "logN16-L30", "logN16-L11"])
def test_hoisted_rotations_match_oracle(pairs, P, nl, steps):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = pairs(P)
    st = si.Stream(803, nl)
    a = rand_ct(st, o, nl)
    keys = [rand_key(st, o) for _ in steps]
    da = to_device(a)
    outs = [torch.empty_like(da) for _ in steps]
    g.rotate_hoisted(da, nl, steps, [g.rotation_key(to_device(k), s) for k, s in zip(keys, steps)], outs)
    torch.cuda.synchronize()
    ref = o.rotate_hoisted(a, steps, keys)
    for i in range(len(steps)):
        assert np.array_equal(to_host(outs[i]).reshape(a.shape), ref[i]), steps[i]
    with pytest.raises(FidesError):
        g.rotate_hoisted(da, nl, [], [], [])


@pytest.mark.parametrize("P,nl", [(si.SMALL, 3), (si.MID, 12), (si.MID, 4), (si.FULL, 30), (si.FULL, 13)],
                         ids=["logN12-L3", "logN12-L12", "logN12-L4", "logN16-L30", "logN16-L13"])
def test_modraise_and_mul_i_match_oracle(pairs, P, nl):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = pairs(P)
    st = si.Stream(804, nl)
    a1 = np.stack([si.uniform_poly(st, o.q[:1], o.N) for _ in range(2)])
    raised = torch.empty(2 * nl * o.N, dtype=torch.int64, device="cuda")
    g.modraise(to_device(a1), raised, nl)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(raised).reshape(2, nl, o.N), o.modraise(a1, nl))
    a = np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])
    da = to_device(a)
    for sign, k in ((1, o.N // 2), (-1, 3 * o.N // 2)):
        out = torch.empty_like(da)
        g.mul_i(da, nl, out, sign=sign)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(out).reshape(a.shape), o.mul_monomial(a, k)), sign


def test_autotune_cache_round_trip(pairs, tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = pairs(si.FULL)
    path = str(tmp_path / "tune.json")
    g.autotune(16, cache=path)
    first = g.tune_table()
    g.set_tune_table(bytes(len(first)))           # all variant 0
    assert g.tune_table() == bytes(len(first))
    g.autotune(16, cache=path)                    # loaded from the cache, not re-timed
    assert g.tune_table() == first
    with pytest.raises(FidesError):
        g.set_tune_table(bytes([9]) * len(first))
    assert g.tune_table() == first
