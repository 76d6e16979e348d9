"""GPU parity: every entry point of the C ABI against the CPU oracle, residue
for residue (bit-exact), on seeded inputs.

Sizes: the logN=12 workload (3 limbs, K=1, dnum=3) and a logN=12 set with 12
limbs (K=4, alpha=4: several digits, a ragged last digit) run in full; the
logN=16 workload (30 limbs, K=10, dnum=3) runs in full at the top level and
at ragged levels; a logN=12 set with the most primes a context takes (48 q +
16 special = 64; digits of 16 limbs, beyond the unrolled conversion sizes)
covers the generic paths.  Keys are uniform residues (parity does not depend on key
structure); decryption through real keys is checked separately.
"""
import ctypes

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


@pytest.fixture(scope="module", params=["SMALL", "MID", "FULL", "WIDE"])
def pair(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = getattr(si, request.param)
    g, o = make_pair(P)
    yield P, g, o
    g.close()


def rand_poly(st, primes, N, npoly=None):
    if npoly is None:
        return si.uniform_poly(st, primes, N)
    return np.stack([si.uniform_poly(st, primes, N) for _ in range(npoly)])


def rand_key(st, o):
    return np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])


def levels(P):
    # top level, a ragged level inside a digit, and the bottom
    return sorted({P.nq, max(1, P.nq - 3), max(1, (P.nq + 1) // 2), 1})


def test_ntt_intt_all_primes(pair):
    P, g, o = pair
    st = si.Stream(1000 + P.logN, 1)
    n = len(o.primes)
    a = rand_poly(st, o.primes, o.N)
    d = to_device(a)
    g.ntt(d, 0, n)
    A = o.ntt_limbs(a, list(range(n)))
    assert np.array_equal(to_host(d).reshape(a.shape), A)
    g.intt(d, 0, n)
    assert np.array_equal(to_host(d).reshape(a.shape), a)


def test_ntt_batch_and_offset(pair):
    P, g, o = pair
    st = si.Stream(1001, 2)
    first, nl, batch = 1, min(3, len(o.primes) - 1), 3
    prim = o.primes[first:first + nl]
    a = np.stack([rand_poly(st, prim, o.N) for _ in range(batch)])
    d = to_device(a)
    g.ntt(d, first, nl, batch)
    got = to_host(d).reshape(a.shape)
    for b in range(batch):
        assert np.array_equal(got[b], o.ntt_limbs(a[b], list(range(first, first + nl))))
    g.intt(d, first, nl, batch)
    assert np.array_equal(to_host(d).reshape(a.shape), a)


def test_modup(pair):
    P, g, o = pair
    st = si.Stream(1002, 3)
    for nl in levels(P):
        d = rand_poly(st, o.q[:nl], o.N)
        beta = g.beta(nl)
        ext = torch.zeros(beta * (nl + o.nk) * o.N, dtype=torch.int64, device="cuda")
        g.modup(to_device(d), nl, ext)
        got = to_host(ext).reshape(beta, nl + o.nk, o.N)
        assert np.array_equal(got, o.modup(d)), "modup differs at nl=%d" % nl


def test_moddown(pair):
    P, g, o = pair
    st = si.Stream(1003, 4)
    for nl in levels(P):
        x = rand_poly(st, o.q[:nl] + o.p, o.N)
        out = torch.zeros(nl * o.N, dtype=torch.int64, device="cuda")
        g.moddown(to_device(x), nl, out)
        assert np.array_equal(to_host(out).reshape(nl, o.N), o.moddown(x)), "moddown differs at nl=%d" % nl


def test_keyswitch(pair):
    P, g, o = pair
    st = si.Stream(1004, 5)
    key = rand_key(st, o)
    dk = g.register_key(to_device(key), 0)
    for nl in levels(P):
        d = rand_poly(st, o.q[:nl], o.N)
        o0 = torch.zeros(nl * o.N, dtype=torch.int64, device="cuda")
        o1 = torch.zeros_like(o0)
        g.keyswitch(to_device(d), nl, dk, o0, o1)
        w0, w1 = o.keyswitch(d, key)
        assert np.array_equal(to_host(o0).reshape(nl, o.N), w0), "ks0 differs at nl=%d" % nl
        assert np.array_equal(to_host(o1).reshape(nl, o.N), w1), "ks1 differs at nl=%d" % nl


def test_hmult(pair):
    P, g, o = pair
    st = si.Stream(1005, 6)
    key = rand_key(st, o)
    dk = g.relin_key(to_device(key))
    for nl in levels(P):
        a, b = rand_poly(st, o.q[:nl], o.N, 2), rand_poly(st, o.q[:nl], o.N, 2)
        out = torch.zeros(2 * nl * o.N, dtype=torch.int64, device="cuda")
        scale = g.hmult(to_device(a), to_device(b), nl, dk, out, 2.0**40, 2.0**40)
        assert scale == 2.0**80
        assert np.array_equal(to_host(out).reshape(2, nl, o.N), o.hmult(a, b, key)), "hmult differs at nl=%d" % nl


def test_key_written_just_before_the_call(pair):
    """The key switch reads its key before it waits for the kernels queued
    ahead of it, and every library kernel lets the next one start early; a key
    produced on the same stream right before the call by the library's own
    NTT (from its coefficient form) and registered at once is still the one
    used, on two back-to-back calls with different keys in one buffer."""
    P, g, o = pair
    st = si.Stream(1014, 15)
    k1, k2 = rand_key(st, o), rand_key(st, o)
    nl = P.nq
    a, b = rand_poly(st, o.q[:nl], o.N, 2), rand_poly(st, o.q[:nl], o.N, 2)
    da, db = to_device(a), to_device(b)
    ne, allp = len(o.primes), list(range(len(o.primes)))
    coeff = [to_device(np.stack([np.stack([o.intt_limbs(k[j, t], allp) for t in range(2)]) for j in range(o.dnum)]))
             for k in (k1, k2)]
    dk = torch.zeros_like(coeff[0])
    out1 = torch.empty(2 * nl * o.N, dtype=torch.int64, device="cuda")
    out2 = torch.empty_like(out1)
    for c, out in zip(coeff, (out1, out2)):
        dk.copy_(c)                                # a copy on the current stream
        g.ntt(dk, 0, ne, batch=2 * o.dnum)         # the library's NTT, same stream
        key = g.relin_key(dk)
        g.hmult(da, db, nl, key, out)
        torch.cuda.synchronize()
        key.close()
    assert np.array_equal(to_host(out1).reshape(2, nl, o.N), o.hmult(a, b, k1))
    assert np.array_equal(to_host(out2).reshape(2, nl, o.N), o.hmult(a, b, k2))


def test_key_handles_are_checked(pair):
    """A key is refused (FIDES_ERR_KEY) before anything is queued when its
    Galois element is not the one the operation needs, or it belongs to
    another context; registration refuses elements that are not 0 or odd
    below 2N."""
    P, g, o = pair
    nl = P.nq
    st = si.Stream(1015, 16)
    a = rand_poly(st, o.q[:nl], o.N, 2)
    da = to_device(a)
    buf = to_device(rand_key(st, o))
    rlk, rk1, ck = g.relin_key(buf), g.rotation_key(buf, 1), g.conjugation_key(buf)
    assert (rlk.galois, rk1.galois, ck.galois) == (0, 5, 2 * o.N - 1)
    out = torch.full((2 * nl * o.N,), 7, dtype=torch.int64, device="cuda")
    for call in (lambda: g.rotate(da, nl, 1, rlk, out),        # the relinearisation key for a rotation
                 lambda: g.rotate(da, nl, 2, rk1, out),        # the key of another rotation
                 lambda: g.conjugate(da, nl, rk1, out),
                 lambda: g.hmult(da, da, nl, rk1, out),
                 lambda: g.hsquare(da, nl, ck, out)):
        with pytest.raises(FidesError) as e:
            call()
        assert e.value.code == -7
    torch.cuda.synchronize()
    assert bool((out == 7).all()), "a refused call queued work"
    for bad in (2, 2 * o.N + 1, 4 * o.N):
        with pytest.raises(FidesError) as e:
            g.register_key(buf, bad)
        assert e.value.code == -1
    q2 = find_primes(12, 40, 2)
    other = Context(12, q2, find_primes(12, 50, 1, exclude=q2), 2)
    try:
        with pytest.raises(FidesError) as e:
            g.rotate(da, nl, 1, other.rotation_key(torch.zeros(other.key_words(), dtype=torch.int64,
                                                                device="cuda"), 1), out)
        assert e.value.code == -7
    finally:
        other.close()


def test_rotate(pair):
    P, g, o = pair
    st = si.Stream(1006, 7)
    key = rand_key(st, o)
    buf = to_device(key)
    nl = P.nq
    a = rand_poly(st, o.q[:nl], o.N, 2)
    da = to_device(a)
    steps_list = [1, 2, 1 << (P.logN - 3), -1, o.N // 2, 3 * o.N]
    for steps in steps_list:
        out = torch.zeros(2 * nl * o.N, dtype=torch.int64, device="cuda")
        g.rotate(da, nl, steps, g.rotation_key(buf, steps), out)
        assert np.array_equal(to_host(out).reshape(2, nl, o.N), o.rotate(a, steps, key)), "rotate %d" % steps
    nl2 = max(1, nl - 3)
    a2 = rand_poly(st, o.q[:nl2], o.N, 2)
    out = torch.zeros(2 * nl2 * o.N, dtype=torch.int64, device="cuda")
    g.rotate(to_device(a2), nl2, 5, g.rotation_key(buf, 5), out)
    assert np.array_equal(to_host(out).reshape(2, nl2, o.N), o.rotate(a2, 5, key))


def test_rescale(pair):
    P, g, o = pair
    st = si.Stream(1007, 8)
    for nl in sorted({P.nq, 2, max(2, P.nq // 2)}):
        a = rand_poly(st, o.q[:nl], o.N, 2)
        out = torch.zeros(2 * (nl - 1) * o.N, dtype=torch.int64, device="cuda")
        scale = g.rescale(to_device(a), nl, out, 2.0**80)
        assert scale == 2.0**80 / o.q[nl - 1]
        assert np.array_equal(to_host(out).reshape(2, nl - 1, o.N), o.rescale(a)), "rescale differs at nl=%d" % nl


def test_rescale_round(pair):
    """Round-to-nearest Rescale against the oracle's, with the dropped limb's
    coefficients at the rounding boundary (q_l -+ 1) / 2, at 0, 1 and q_l - 1,
    and random; the floor Rescale of the same input differs from it."""
    P, g, o = pair
    st = si.Stream(1013, 14)
    for nl in sorted({P.nq, 2, max(2, P.nq // 2 + 1)}):
        a = rand_poly(st, o.q[:nl], o.N, 2)
        ql = o.q[nl - 1]
        edges = np.array([0, 1, (ql - 1) // 2, (ql + 1) // 2, ql - 1], dtype=np.uint64)
        for poly in range(2):
            coef = o.intt(a[poly, nl - 1], nl - 1)
            coef[::7] = np.resize(edges, coef[::7].shape)
            a[poly, nl - 1] = o.ntt(coef, nl - 1)
        out = torch.zeros(2 * (nl - 1) * o.N, dtype=torch.int64, device="cuda")
        scale = g.rescale(to_device(a), nl, out, 2.0**80, nearest=True)
        assert scale == 2.0**80 / ql
        want = o.rescale(a, nearest=True)
        assert np.array_equal(to_host(out).reshape(2, nl - 1, o.N), want), "rescale_round differs at nl=%d" % nl
        assert not np.array_equal(want, o.rescale(a))


def test_hmult_on_8_byte_aligned_buffers(pair):
    """Buffers that are only 8-byte aligned take the tensor product fused into
    the first INTT pass instead of its own 16-byte pass; the residues are the
    same."""
    P, g, o = pair
    st = si.Stream(1012, 13)
    key = rand_key(st, o)
    dk = g.relin_key(to_device(key))
    nl = P.nq
    a, b = rand_poly(st, o.q[:nl], o.N, 2), rand_poly(st, o.q[:nl], o.N, 2)
    w = 2 * nl * o.N
    pool = torch.zeros(3 * w + 5, dtype=torch.int64, device="cuda")
    da, db, out = pool[1:1 + w], pool[w + 3:2 * w + 3], pool[2 * w + 5:3 * w + 5]   # odd word offsets
    da.copy_(to_device(a).reshape(-1))
    db.copy_(to_device(b).reshape(-1))
    g.hmult(da, db, nl, dk, out)
    ref = o.hmult(a, b, key)
    assert np.array_equal(to_host(out).reshape(ref.shape), ref)
    out2 = torch.zeros(2 * (nl - 1) * o.N + 1, dtype=torch.int64, device="cuda")[1:]
    g.hmult_rescale(da, db, nl, dk, out2)
    assert np.array_equal(to_host(out2).reshape(2, nl - 1, o.N), o.rescale(ref))


def test_hmult_rescale(pair):
    """The fused HMult+Rescale against the oracle's HMult then Rescale, at
    every level the other tests use (2 and up); the plain HMult on the same
    inputs is unchanged."""
    P, g, o = pair
    st = si.Stream(1011, 12)
    key = rand_key(st, o)
    dk = g.relin_key(to_device(key))
    for nl in sorted({n for n in levels(P) if n >= 2} | {2}):
        a, b = rand_poly(st, o.q[:nl], o.N, 2), rand_poly(st, o.q[:nl], o.N, 2)
        out = torch.zeros(2 * (nl - 1) * o.N, dtype=torch.int64, device="cuda")
        scale = g.hmult_rescale(to_device(a), to_device(b), nl, dk, out, 2.0**40, 2.0**40)
        assert scale == 2.0**80 / o.q[nl - 1]
        ref = o.rescale(o.hmult(a, b, key))
        assert np.array_equal(to_host(out).reshape(2, nl - 1, o.N), ref), "hmult_rescale differs at nl=%d" % nl


def test_round_to_nearest_mode(pair):
    """Both contexts in round-to-nearest mode (ModDown converts centred
    residues, Rescale lifts the centred one): ModDown, KeySwitch, HMult,
    HRotate, Rescale and the fused HMult+Rescale equal the oracle's, at the
    top level and a ragged one, and differ from the floor results."""
    P, g, o = pair
    st = si.Stream(1016, 17)
    key = rand_key(st, o)
    buf = to_device(key)
    rlk = g.relin_key(buf)
    g.set_rounding(True)
    o.set_rounding(True)
    try:
        assert g.nearest
        for nl in sorted({P.nq, max(2, P.nq - 3)}):
            ne = nl + len(o.p)
            x = rand_poly(st, o.q[:nl] + o.p, o.N)
            out = torch.zeros(nl * o.N, dtype=torch.int64, device="cuda")
            g.moddown(to_device(x), nl, out)
            want = o.moddown(x)
            assert np.array_equal(to_host(out).reshape(nl, o.N), want), "moddown nl=%d" % nl
            o.set_rounding(False)
            assert not np.array_equal(want, o.moddown(x))
            o.set_rounding(True)
            a, b = rand_poly(st, o.q[:nl], o.N, 2), rand_poly(st, o.q[:nl], o.N, 2)
            da, db = to_device(a), to_device(b)
            m = torch.zeros(2 * nl * o.N, dtype=torch.int64, device="cuda")
            g.hmult(da, db, nl, rlk, m)
            ref_m = o.hmult(a, b, key)
            assert np.array_equal(to_host(m).reshape(2, nl, o.N), ref_m), "hmult nl=%d" % nl
            r = torch.zeros_like(m)
            g.rotate(da, nl, 3, g.rotation_key(buf, 3), r)
            assert np.array_equal(to_host(r).reshape(2, nl, o.N), o.rotate(a, 3, key)), "rotate nl=%d" % nl
            o0, o1 = (torch.zeros(nl * o.N, dtype=torch.int64, device="cuda") for _ in range(2))
            g.keyswitch(da, nl, rlk, o0, o1)
            w0, w1 = o.keyswitch(a[0], key)
            assert np.array_equal(to_host(o0).reshape(nl, o.N), w0) and np.array_equal(to_host(o1).reshape(nl, o.N), w1)
            rs = torch.zeros(2 * (nl - 1) * o.N, dtype=torch.int64, device="cuda")
            g.rescale(m, nl, rs)
            assert np.array_equal(to_host(rs).reshape(2, nl - 1, o.N), o.rescale(ref_m)), "rescale nl=%d" % nl
            fu = torch.zeros_like(rs)
            g.hmult_rescale(da, db, nl, rlk, fu)
            assert np.array_equal(to_host(fu).reshape(2, nl - 1, o.N), o.rescale(ref_m)), "hmult_rescale nl=%d" % nl
    finally:
        g.set_rounding(False)
        o.set_rounding(False)


def test_galois_and_psi(pair):
    P, g, o = pair
    for i in range(len(o.primes)):
        assert g.psi(i) == o.psi(i)
    for s in [0, 1, 7, -1, -5, o.N, 12345]:
        assert g.galois_elt(s) == o.galois_elt(s)


def test_argument_errors(pair):
    P, g, o = pair
    d = torch.zeros(2 * o.N, dtype=torch.int64, device="cuda")
    with pytest.raises(FidesError) as e:
        g.rescale(d, 1, d)
    assert e.value.code == -1
    with pytest.raises(FidesError) as e:
        g.rescale(d, 1, d, nearest=True)
    assert e.value.code == -1
    with pytest.raises(FidesError):
        g.ntt(d, len(o.primes), 1)
    with pytest.raises(ValueError):
        g.ntt(d, 0, 3)
    # fused HMult+Rescale: one limb cannot be rescaled; the ABI checks the
    # output level before queueing anything
    key = g.relin_key(torch.zeros(g.key_words(), dtype=torch.int64, device="cuda"))
    with pytest.raises(FidesError) as e:
        g.hmult_rescale(d, d, 1, key, d)
    assert e.value.code == -1
    from paper_2507_04775_gb300 import fides as F
    ct = F.fides_ct(d.data_ptr(), 2, 1.0)
    bad = F.fides_ct(d.data_ptr(), 2, 0.0)      # out must have n_limbs - 1 = 1 limb
    rc = F.lib().fides_hmult_rescale(g._h, ctypes.byref(ct), ctypes.byref(ct), key.handle, ctypes.byref(bad), None)
    assert rc == -1
    # a raw buffer where a key handle belongs is refused by the binding
    with pytest.raises(TypeError):
        g.hmult(d, d, 1, key.tensor, d)


def test_boundary_refuses_bad_descriptors_before_queueing():
    """Through the C ABI: zero limbs, more limbs than the context has, a level
    mismatch between operands, an output aliasing an input and a NULL
    descriptor are each refused with FIDES_ERR_ARG, and no work is queued (a
    sentinel output stays as it was)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_04775_gb300 import fides as F
    P = si.SMALL
    g, o = make_pair(P)
    st = si.Stream(1020, 1)
    L, N = P.nq, o.N
    key = rand_key(st, o)
    rlk = g.relin_key(to_device(key))
    rk = g.rotation_key(to_device(key), 1)
    a = to_device(rand_poly(st, o.q, N, 2))
    b = to_device(rand_poly(st, o.q, N, 2))
    sentinel = torch.full((2 * (L + 1) * N,), 12345, dtype=torch.int64, device="cuda")
    lib = F.lib()

    def ct(t, n):
        return F.fides_ct(t.data_ptr(), n, 1.0)

    cases = [
        ("hmult, 0 limbs", lambda: lib.fides_hmult(g._h, ctypes.byref(ct(a, 0)), ctypes.byref(ct(b, 0)),
                                                   rlk.handle, ctypes.byref(ct(sentinel, 0)), None)),
        ("hmult, L + 1 limbs", lambda: lib.fides_hmult(g._h, ctypes.byref(ct(a, L + 1)), ctypes.byref(ct(b, L + 1)),
                                                       rlk.handle, ctypes.byref(ct(sentinel, L + 1)), None)),
        ("hmult, level mismatch", lambda: lib.fides_hmult(g._h, ctypes.byref(ct(a, L)), ctypes.byref(ct(b, L - 1)),
                                                          rlk.handle, ctypes.byref(ct(sentinel, L)), None)),
        ("hmult, out aliases a", lambda: lib.fides_hmult(g._h, ctypes.byref(ct(sentinel, L)),
                                                         ctypes.byref(ct(b, L)), rlk.handle,
                                                         ctypes.byref(ct(sentinel, L)), None)),
        ("hmult, NULL b", lambda: lib.fides_hmult(g._h, ctypes.byref(ct(a, L)), None, rlk.handle,
                                                  ctypes.byref(ct(sentinel, L)), None)),
        ("rotate, out level", lambda: lib.fides_rotate(g._h, ctypes.byref(ct(a, L)), 1, rk.handle,
                                                       ctypes.byref(ct(sentinel, L - 1)), None)),
        ("rotate, out aliases a", lambda: lib.fides_rotate(g._h, ctypes.byref(ct(sentinel, L)), 1, rk.handle,
                                                           ctypes.byref(ct(sentinel, L)), None)),
        ("rescale, 1 limb", lambda: lib.fides_rescale(g._h, ctypes.byref(ct(a, 1)), ctypes.byref(ct(sentinel, 0)),
                                                      None)),
        ("rescale, out level", lambda: lib.fides_rescale(g._h, ctypes.byref(ct(a, L)), ctypes.byref(ct(sentinel, L)),
                                                         None)),
    ]
    for name, call in cases:
        assert call() == -1, name
        torch.cuda.synchronize()
        assert bool((sentinel == 12345).all()), "%s queued work" % name
    assert g.status() == 0
    g.close()
