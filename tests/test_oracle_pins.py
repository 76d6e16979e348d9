"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks an oracle function against one of: a closed form, brute force
on tiny inputs in pure Python integers, a big-integer CRT identity, a library
routine (sympy), or a decryption-error bound.  Together they are meant to fail
on a dropped term, a wrong sign or index, or a transposed operand anywhere in
``oracle/``.
"""
import random

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.client import Client

sympy = pytest.importorskip("sympy")


def brv(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2) if bits else 0


def make_ctx(logN, nq, q_bits, nk, p_bits, dnum):
    q = oracle.find_primes(logN, q_bits, nq)
    p = oracle.find_primes(logN, p_bits, nk, exclude=q)
    return oracle.Context(logN, q, p, dnum)


@pytest.fixture(scope="module")
def tiny():
    # N = 16, four 30-bit q, two 40-bit p, dnum = 2 (alpha = 2)
    return make_ctx(4, 4, 30, 2, 40, 2)


@pytest.fixture(scope="module")
def small():
    P = si.SMALL
    return make_ctx(P.logN, P.nq, P.q_bits, P.nk, P.p_bits, P.dnum)


@pytest.fixture(scope="module")
def mid():
    P = si.MID
    return make_ctx(P.logN, P.nq, P.q_bits, P.nk, P.p_bits, P.dnum)


# ---------------------------------------------------------------- modmul
def test_mul_mod_edges_and_random():
    rng = random.Random(1)
    for q in [3, 97, (1 << 40) - 87, 1152921504606830593, (1 << 61) - 1]:
        vals = [0, 1, q - 1, q - 2, q // 2, 2 * q - 1 if 2 * q - 1 < 2**64 else q]
        for a in vals:
            for b in vals:
                assert oracle.mul_mod(a, b, q) == (a * b) % q
        for _ in range(2000):
            a, b = rng.randrange(2**64), rng.randrange(2**64)
            assert oracle.mul_mod(a, b, q) == (a * b) % q


# ---------------------------------------------------------------- primes
def test_is_prime_matches_sympy():
    rng = random.Random(2)
    cands = [561, 1105, 1729, 2465, 2821, 6601, 3215031751, 2**61 - 1, 2**64 - 59, 2**62 + 1]
    cands += [rng.randrange(2**64) | 1 for _ in range(300)]
    for n in cands:
        assert oracle.is_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("logN,bits,count", [(12, 40, 3), (12, 50, 1), (16, 54, 30), (16, 60, 10)])
def test_find_primes_is_the_downward_walk(logN, bits, count):
    ps = oracle.find_primes(logN, bits, count)
    step = 2 << logN
    # brute force: every candidate of the form k*2N+1 below 2^bits, descending
    want, q = [], (1 << bits) - step + 1
    while len(want) < count:
        if sympy.isprime(q):
            want.append(q)
        q -= step
    assert ps == want
    for q in ps:
        assert q % step == 1 and q.bit_length() == bits


def test_smallest_generator_matches_sympy():
    for q in [97, 257, 7681, 12289] + oracle.find_primes(12, 40, 2) + oracle.find_primes(16, 54, 2):
        assert oracle.smallest_generator(q) == sympy.primitive_root(q)


def test_psi_is_primitive_2n_root(small, mid):
    for ctx in (small, mid):
        for i, q in enumerate(ctx.primes):
            psi = ctx.psi(i)
            g = sympy.primitive_root(q)
            assert psi == pow(g, (q - 1) // (2 * ctx.N), q)
            assert pow(psi, ctx.N, q) == q - 1


# ---------------------------------------------------------------- NTT
def _eval_at(a, x, q):
    acc = 0
    for c in reversed(a):
        acc = (acc * x + c) % q
    return acc


def test_ntt_is_evaluation_at_odd_roots(tiny):
    """NTT slot j = a(psi^(2 brv(j)+1)) (bit-reversed order), by Horner."""
    rng = random.Random(3)
    N, bits = tiny.N, tiny.logN
    for i, q in enumerate(tiny.primes):
        a = [rng.randrange(q) for _ in range(N)]
        psi = tiny.psi(i)
        want = [_eval_at(a, pow(psi, 2 * brv(j, bits) + 1, q), q) for j in range(N)]
        assert tiny.ntt_naive(np.array(a, dtype=np.uint64), i).tolist() == want
        assert tiny.ntt(np.array(a, dtype=np.uint64), i).tolist() == want


@pytest.mark.parametrize("logN", [6, 8, 10])
def test_radix2_ntt_matches_definition(logN):
    ctx = make_ctx(logN, 2, 50, 1, 59, 1)
    st = si.Stream(5, logN)
    for i, q in enumerate(ctx.primes):
        a = st.uniform_mod(q, ctx.N)
        A = ctx.ntt_naive(a, i)
        assert np.array_equal(ctx.ntt(a, i), A)
        assert np.array_equal(ctx.intt_naive(A, i), a)
        assert np.array_equal(ctx.intt(A, i), a)


def _negacyclic(a, b, q):
    N = len(a)
    c = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                c[k] += a[i] * b[j]
            else:
                c[k - N] -= a[i] * b[j]
    return [x % q for x in c]


@pytest.mark.parametrize("logN", [4, 6])
def test_convolution_theorem(logN):
    """INTT(NTT(a) . NTT(b)) equals the schoolbook product mod X^N + 1."""
    ctx = make_ctx(logN, 2, 40, 1, 50, 1)
    st = si.Stream(7, logN)
    for i, q in enumerate(ctx.primes):
        a, b = st.uniform_mod(q, ctx.N), st.uniform_mod(q, ctx.N)
        A, B = ctx.ntt(a, i), ctx.ntt(b, i)
        C = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64)
        assert ctx.intt(C, i).tolist() == _negacyclic(a.tolist(), b.tolist(), q)


def test_ntt_special_inputs(small):
    N = small.N
    for i, q in enumerate(small.primes):
        one = np.zeros(N, dtype=np.uint64); one[0] = 1
        assert np.all(small.ntt(one, i) == 1)
        x = np.zeros(N, dtype=np.uint64); x[1] = 1
        psi = small.psi(i)
        want = [pow(psi, 2 * brv(j, small.logN) + 1, q) for j in range(N)]
        assert small.ntt(x, i).tolist() == want
        # inverse at full size is an identity on random data
        a = si.Stream(9, i).uniform_mod(q, N)
        assert np.array_equal(small.intt(small.ntt(a, i), i), a)


# ---------------------------------------------------------------- base conversion
def _crt_int(res, primes):
    return oracle.crt(np.asarray(res, dtype=np.uint64).reshape(len(primes), -1), primes)


def test_bconv_is_x_plus_u_Q(mid):
    """y_p = x + u Q_src (mod p) with one integer 0 <= u < |src| for all p."""
    st = si.Stream(11)
    src = [0, 1, 2, 3]
    dst = list(range(4, len(mid.primes)))
    x = si.uniform_poly(st, [mid.primes[i] for i in src], mid.N)
    y = mid.bconv(x, src, dst)
    sp = [mid.primes[i] for i in src]
    Qs = 1
    for q in sp:
        Qs *= q
    X = oracle.crt(x, sp)
    for n in range(0, mid.N, 97):
        us = set()
        for k, di in enumerate(dst):
            p = mid.primes[di]
            # find u in [0, |src|) with X + u Qs = y (mod p)
            cand = [u for u in range(len(src)) if (X[n] + u * Qs - int(y[k, n])) % p == 0]
            assert len(cand) == 1
            us.add(cand[0])
        assert len(us) == 1


def _coeff(ctx, x, pidx):
    return ctx.intt_limbs(x, pidx)


def test_modup_digits(mid):
    nl = 11                                 # ragged: digits of 4, 4 and 3 limbs
    st = si.Stream(12)
    d = si.uniform_poly(st, mid.q[:nl], mid.N)
    ext = mid.modup(d)
    alpha = mid.alpha
    assert alpha == 4 and ext.shape == (3, nl + mid.nk, mid.N)
    dc = _coeff(mid, d, list(range(nl)))
    ep = list(range(nl)) + [mid.nq + k for k in range(mid.nk)]
    for j in range(3):
        lo, hi = j * alpha, min((j + 1) * alpha, nl)
        assert np.array_equal(ext[j, lo:hi], d[lo:hi])      # digit limbs copied
        ec = _coeff(mid, ext[j], ep)
        sp = mid.q[lo:hi]
        Qj = 1
        for q in sp:
            Qj *= q
        X = oracle.crt(dc[lo:hi], sp)
        for n in range(0, mid.N, 131):
            for z in range(nl + mid.nk):
                if lo <= z < hi:
                    continue
                p = mid.primes[ep[z]]
                assert any((X[n] + u * Qj - int(ec[z, n])) % p == 0 for u in range(hi - lo))


def test_moddown_is_floor_division_by_P(mid):
    nl = 7
    st = si.Stream(13)
    ep = list(range(nl)) + [mid.nq + k for k in range(mid.nk)]
    x = si.uniform_poly(st, [mid.primes[i] for i in ep], mid.N)
    out = mid.moddown(x)
    xc = _coeff(mid, x, ep)
    oc = _coeff(mid, out, list(range(nl)))
    Ql, P = 1, 1
    for q in mid.q[:nl]:
        Ql *= q
    for p in mid.p:
        P *= p
    X = oracle.crt(xc, mid.q[:nl] + mid.p)
    xP = oracle.crt(xc[nl:], mid.p)
    O = oracle.crt(oc, mid.q[:nl])
    for n in range(mid.N):
        assert (X[n] - xP[n]) % P == 0
        u = ((X[n] - xP[n]) // P - O[n]) % Ql
        assert 0 <= u < mid.nk


def test_bconv_centred_is_x_plus_u_Q_with_centred_u(mid):
    """The conversion from centred residues: y_p = X + u Q_src (mod p) with
    one integer u, |u| <= |src| / 2 + 1, for every target p; and it differs
    from the canonical conversion by exactly -c Q_src, c the number of
    residues [x_i qhat_i^-1]_{q_i} above (q_i - 1) / 2."""
    st = si.Stream(31)
    src = [0, 1, 2, 3]
    dst = list(range(4, len(mid.primes)))
    sp = [mid.primes[i] for i in src]
    x = si.uniform_poly(st, sp, mid.N)
    yc = mid.bconv(x, src, dst, centred=True)
    yf = mid.bconv(x, src, dst)
    Qs = 1
    for q in sp:
        Qs *= q
    X = oracle.crt(x, sp)
    lo, hi = -(len(src) // 2) - 1, len(src) // 2 + 1
    for n in range(0, mid.N, 89):
        us = set()
        for k, di in enumerate(dst):
            p = mid.primes[di]
            cand = [u for u in range(lo, hi + 1) if (X[n] + u * Qs - int(yc[k, n])) % p == 0]
            assert len(cand) == 1
            us.add(cand[0])
        assert len(us) == 1
        cnt = 0
        for i, q in enumerate(sp):
            qhat = Qs // q
            v = int(x[i, n]) * pow(qhat % q, -1, q) % q
            cnt += v > (q - 1) // 2
        for k, di in enumerate(dst):
            p = mid.primes[di]
            assert (int(yf[k, n]) - cnt * Qs - int(yc[k, n])) % p == 0


def test_moddown_nearest_is_round_within_K_over_2(mid):
    """Nearest ModDown: out P = X - S (mod Q_l P) with S = X (mod P) and
    |S| < K P / 2, so out is within K/2 of X / P; its error S / P has mean
    about 0, where floor's has mean about K / 2 (the floor's 1/2 and the
    conversion term u in [0, K) with mean (K - 1) / 2)."""
    nl = 7
    st = si.Stream(32)
    ep = list(range(nl)) + [mid.nq + k for k in range(mid.nk)]
    x = si.uniform_poly(st, [mid.primes[i] for i in ep], mid.N)
    xc = _coeff(mid, x, ep)
    Ql, P = 1, 1
    for q in mid.q[:nl]:
        Ql *= q
    for p in mid.p:
        P *= p
    X = oracle.crt(xc, mid.q[:nl] + mid.p)
    means = {}
    for nearest in (False, True):
        mid.set_rounding(nearest)
        try:
            oc = _coeff(mid, mid.moddown(x), list(range(nl)))
        finally:
            mid.set_rounding(False)
        O = oracle.crt(oc, mid.q[:nl])
        errs = []
        for n in range(mid.N):
            S = oracle.centered([(X[n] - O[n] * P) % (Ql * P)], Ql * P)[0]
            assert (S - X[n]) % P == 0
            if nearest:
                assert abs(S) < mid.nk * P // 2
            else:
                assert 0 <= S < (mid.nk + 1) * P
            errs.append(S / P)
        means[nearest] = float(np.mean(errs))
    assert abs(means[True]) < 0.1, means
    assert abs(means[False] - mid.nk / 2) < 0.25, means


def test_rescale_is_exact_floor(mid):
    nl = 9
    st = si.Stream(14)
    a = np.stack([si.uniform_poly(st, mid.q[:nl], mid.N) for _ in range(2)])
    out = mid.rescale(a)
    ql = mid.q[nl - 1]
    for poly in range(2):
        X = oracle.crt(_coeff(mid, a[poly], list(range(nl))), mid.q[:nl])
        O = oracle.crt(_coeff(mid, out[poly], list(range(nl - 1))), mid.q[:nl - 1])
        assert O == [x // ql for x in X]


def test_rescale_nearest_is_exact_round(mid):
    """Round-to-nearest Rescale: round(x / q_l) = floor((2x + q_l) / (2 q_l))
    (q_l odd, so no ties), reduced mod Q_{l-1} (x just below Q_l rounds up to
    Q_{l-1} = 0), on random x and on x whose remainder mod q_l sits at the
    rounding boundary ((q_l -+ 1) / 2), at 0 and at q_l - 1."""
    nl = 9
    ql = mid.q[nl - 1]
    Ql, Ql1 = 1, 1
    for q in mid.q[:nl]:
        Ql *= q
    Ql1 = Ql // ql
    rng = random.Random(19)
    X = [[rng.randrange(Ql) for _ in range(mid.N)] for _ in range(2)]
    edges = [0, 1, (ql - 1) // 2, (ql + 1) // 2, ql - 1]
    for n in range(0, mid.N, 3):
        k = rng.randrange(Ql1)
        X[0][n] = k * ql + edges[(n // 3) % len(edges)]
    X[1][0], X[1][1], X[1][2] = Ql - 1, Ql - (ql - 1) // 2, Ql - (ql + 1) // 2
    a = np.stack([mid.ntt_limbs(np.array([[x % q for x in Xp] for q in mid.q[:nl]], dtype=np.uint64),
                                list(range(nl))) for Xp in X])
    out = mid.rescale(a, nearest=True)
    for poly in range(2):
        O = oracle.crt(_coeff(mid, out[poly], list(range(nl - 1))), mid.q[:nl - 1])
        assert O == [((2 * x + ql) // (2 * ql)) % Ql1 for x in X[poly]]
    # floor and nearest differ exactly where the remainder passes (q_l - 1) / 2
    fl = mid.rescale(a)
    for poly in range(2):
        F = oracle.crt(_coeff(mid, fl[poly], list(range(nl - 1))), mid.q[:nl - 1])
        O = oracle.crt(_coeff(mid, out[poly], list(range(nl - 1))), mid.q[:nl - 1])
        for x, f, o in zip(X[poly], F, O):
            assert o == (f + (1 if x % ql > (ql - 1) // 2 else 0)) % Ql1


# ---------------------------------------------------------------- automorphism
def test_automorphism_coeff_is_substitution(tiny):
    N = tiny.N
    st = si.Stream(15)
    a = si.uniform_poly(st, tiny.q, N)
    for steps in [1, 2, 3, -1]:
        g = tiny.galois_elt(steps)
        assert g == pow(5, steps % (N // 2), 2 * N)
        out = tiny.automorph_coeff(a, g)
        for z, q in enumerate(tiny.q):
            want = [0] * N
            for i in range(N):
                e = (i * g) % (2 * N)
                if e < N:
                    want[e] = (want[e] + int(a[z, i])) % q
                else:
                    want[e - N] = (want[e - N] - int(a[z, i])) % q
            assert out[z].tolist() == want


def test_automorphism_eval_matches_coeff(small):
    st = si.Stream(16)
    a = si.uniform_poly(st, small.q, small.N)
    idx = list(range(small.nq))
    A = small.ntt_limbs(a, idx)
    for steps in [1, 5, 1000, -3]:
        g = small.galois_elt(steps)
        assert np.array_equal(small.automorph_eval(A, g), small.ntt_limbs(small.automorph_coeff(a, g), idx))
    assert small.galois_elt(small.N // 2) == 1


# ---------------------------------------------------------------- encoding
def test_encode_fft_matches_direct_and_roundtrips():
    N = 256
    z = si.Stream(17).complex_slots(N // 2)
    m = oracle.encode(z, N, 2.0**40)
    assert np.array_equal(m, oracle.encode_direct(z, N, 2.0**40))
    assert np.max(np.abs(oracle.decode(m, N, 2.0**40) - z)) < 2.0**-30
    assert np.max(np.abs(oracle.decode(m, N, 2.0**40) - oracle.decode_direct(m, N, 2.0**40))) < 2.0**-40


def test_encode_is_multiplicative_and_rotates():
    N = 64
    st = si.Stream(18)
    z1, z2 = st.complex_slots(N // 2), st.complex_slots(N // 2)
    m1, m2 = oracle.encode(z1, N, 2.0**30), oracle.encode(z2, N, 2.0**30)
    prod = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                prod[k] += int(m1[i]) * int(m2[j])
            else:
                prod[k - N] -= int(m1[i]) * int(m2[j])
    assert np.max(np.abs(oracle.decode(prod, N, 2.0**60) - z1 * z2)) < 2.0**-20
    # m(X^5) holds the slots rotated left by one
    rot = [0] * N
    for i in range(N):
        e = (5 * i) % (2 * N)
        if e < N:
            rot[e] += int(m1[i])
        else:
            rot[e - N] -= int(m1[i])
    assert np.max(np.abs(oracle.decode(rot, N, 2.0**30) - np.roll(z1, -1))) < 2.0**-20


# ---------------------------------------------------------------- scheme level
def _rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(1.0, np.max(np.abs(ref))))


@pytest.fixture(scope="module")
def small_client(small):
    return Client(small, seed=si.workload_seed(0))


def test_encrypt_decrypt_roundtrip(small, small_client):
    z = small_client.random_slots()
    ct = small_client.encrypt(z, small.nq, 2.0**40)
    assert _rel_err(small_client.decrypt(ct, 2.0**40), z) < 2.0**-25


def test_keyswitch_noise_bound(small, small_client):
    """decrypt(KeySwitch(d)) - d s' is small: bounded by
    K (1 + ||s||_1) + N alpha B_e max_j Q_j / P (B_e = 6 sigma, rounded up)."""
    c = small
    rk = small_client.rotation_key(1)
    g = c.galois_elt(1)
    sp = c.automorph_eval(small_client.s_eval, g)
    nl = c.nq
    d = si.uniform_poly(si.Stream(19), c.q[:nl], c.N)
    ks0, ks1 = c.keyswitch(d, rk)
    # ks0 + ks1 s - d s' in coefficient form, centred
    idx = list(range(nl))
    lhs = np.stack([ks0, ks1])
    dec = oracle.crt(small_client.ctx.decrypt_residues(lhs, small_client.s_eval[:nl]), c.q[:nl])
    dsp = oracle.crt(c.intt_limbs(c.pointwise_mul(d, sp[:nl], idx), idx), c.q[:nl])
    Q = 1
    for q in c.q[:nl]:
        Q *= q
    diff = oracle.centered([(a - b) % Q for a, b in zip(dec, dsp)], Q)
    P = 1
    for p in c.p:
        P *= p
    Qj = max(c.q[j * c.alpha] for j in range(c.beta(nl)))   # alpha = 1 here
    s1 = int(np.sum(np.abs(small_client.s_coeff)))
    bound = c.nk * (1 + s1) + c.N * c.alpha * 20 * Qj // P + 1
    worst = max(abs(x) for x in diff)
    assert worst <= bound, (worst, bound)


def test_hmult_relin_decrypts_to_product(small, small_client):
    z1, z2 = small_client.random_slots(), small_client.random_slots()
    a = small_client.encrypt(z1, small.nq, 2.0**40)
    b = small_client.encrypt(z2, small.nq, 2.0**40)
    rlk = small_client.relin_key()
    out = small.hmult(a, b, rlk)
    assert _rel_err(small_client.decrypt(out, 2.0**80), z1 * z2) < 2.0**-20
    # and after Rescale by q_2 (scale 2^80 / q_2)
    rs = small.rescale(out)
    assert _rel_err(small_client.decrypt(rs, 2.0**80 / small.q[2]), z1 * z2) < 2.0**-20


def test_hmult_relin_catches_a_wrong_key(small, small_client):
    """A rotation key in place of the relinearisation key must not decrypt."""
    z1, z2 = small_client.random_slots(), small_client.random_slots()
    a = small_client.encrypt(z1, small.nq, 2.0**40)
    b = small_client.encrypt(z2, small.nq, 2.0**40)
    out = small.hmult(a, b, small_client.rotation_key(1))
    assert _rel_err(small_client.decrypt(out, 2.0**80), z1 * z2) > 1.0


def test_hrotate_decrypts_to_rotation(small, small_client):
    z = small_client.random_slots()
    ct = small_client.encrypt(z, small.nq, 2.0**40)
    r1, r2, r3 = small_client.rotation_key(1), small_client.rotation_key(2), small_client.rotation_key(3)
    o1 = small.rotate(ct, 1, r1)
    assert _rel_err(small_client.decrypt(o1, 2.0**40), np.roll(z, -1)) < 2.0**-20
    o12 = small.rotate(o1, 2, r2)
    o3 = small.rotate(ct, 3, r3)
    assert _rel_err(small_client.decrypt(o12, 2.0**40), small_client.decrypt(o3, 2.0**40)) < 2.0**-20
    assert _rel_err(small_client.decrypt(o3, 2.0**40), np.roll(z, -3)) < 2.0**-20


def test_nearest_rounding_meets_the_bound_at_logN16():
    """At logN=16 (30 x 54-bit q, K = 10, dnum = 3, scale 2^40) floor rounding
    leaves a same-sign error on every coefficient of the key-switch output
    (the conversion term u in [0, K) and the floor), which the decoding sums
    coherently into the slots whose evaluation point is near 1 (Galois
    exponents 1, 5, ..., 2N - 3 of the slot group): the rotation misses 2^-20
    there.  Round-to-nearest removes the mean and meets
    it; HMult+relin at scale 2^80 meets it either way."""
    P = si.FULL
    o = make_ctx(P.logN, P.nq, P.q_bits, P.nk, P.p_bits, P.dnum)
    cl = Client(o, seed=si.workload_seed(1) + 7)
    z1, z2 = cl.random_slots(), cl.random_slots()
    a, b = cl.encrypt(z1, P.nq, 2.0**40), cl.encrypt(z2, P.nq, 2.0**40)
    rk, rlk = cl.rotation_key(1), cl.relin_key()
    errs = {}
    for nearest in (False, True):
        o.set_rounding(nearest)
        d = cl.decrypt(o.rotate(a, 1, rk), 2.0**40) - np.roll(z1, -1)
        errs[nearest] = np.abs(d)
        assert _rel_err(cl.decrypt(o.hmult(a, b, rlk), 2.0**80), z1 * z2) < 2.0**-20
    assert errs[False].max() > 2.0**-19
    assert errs[True].max() < 2.0**-20
    # elsewhere the two agree to well below the bound
    assert np.median(errs[False]) < 2.0**-22 and np.median(errs[True]) < 2.0**-22


def test_rotation_by_half_the_ring_is_the_identity(small, small_client):
    """5 has order N/2 modulo 2N, so a rotation by N/2 slots is sigma_1: the
    Galois element is 1, the evaluation-form automorphism leaves every limb as
    it is, and the ciphertext decrypts to the same slots."""
    N = small.N
    assert sympy.n_order(5, 2 * N) == N // 2
    assert small.galois_elt(N // 2) == 1 and small.galois_elt(-(N // 2)) == 1
    st = si.Stream(21)
    a = si.uniform_poly(st, small.q, N)
    assert np.array_equal(small.automorph_eval(a, 1), a)
    z = small_client.random_slots()
    ct = small_client.encrypt(z, small.nq, 2.0**40)
    o = small.rotate(ct, N // 2, small_client.rotation_key(N // 2))
    assert _rel_err(small_client.decrypt(o, 2.0**40), z) < 2.0**-20


def test_lower_level_hmult(mid):
    """Ragged digits: HMult at 5 of 12 limbs (digits of 4 and 1 limbs)."""
    cl = Client(mid, seed=21)
    z1, z2 = cl.random_slots(), cl.random_slots()
    a = cl.encrypt(z1, 5, 2.0**40)
    b = cl.encrypt(z2, 5, 2.0**40)
    out = mid.hmult(a, b, cl.relin_key())
    assert _rel_err(cl.decrypt(out, 2.0**80), z1 * z2) < 2.0**-20


# ------------------------------------------- Table I element-wise ops, Conjugate, HSquare
def _negacyclic(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            if i + j < N:
                out[i + j] += a[i] * b[j]
            else:
                out[i + j - N] -= a[i] * b[j]
    return [x % q for x in out]


def test_ptmult_is_the_negacyclic_ring_product(tiny):
    """In evaluation form the slot-wise product is the product in
    Z_q[X]/(X^N + 1): checked against the schoolbook product of the
    coefficient forms, in Python integers."""
    c = tiny
    st = si.Stream(71)
    a = np.stack([si.uniform_poly(st, c.q, c.N) for _ in range(2)])
    pt = si.uniform_poly(st, c.q, c.N)
    out = c.ptmult(a, pt)
    idx = list(range(c.nq))
    cp = c.intt_limbs(pt, idx)
    for t in range(2):
        ca, co = c.intt_limbs(a[t], idx), c.intt_limbs(out[t], idx)
        for i in range(c.nq):
            assert [int(x) for x in co[i]] == _negacyclic([int(x) for x in ca[i]], [int(x) for x in cp[i]], c.q[i])


def test_additive_and_scalar_ops_are_crt_identities(mid):
    """Each limb is the residue of one big integer modulo Q = prod q_i:
    HAdd/HSub/PtAdd/ScalarAdd/ScalarMult must act on those integers."""
    c = mid
    nl = 7
    st = si.Stream(72)
    a = np.stack([si.uniform_poly(st, c.q[:nl], c.N) for _ in range(2)])
    b = np.stack([si.uniform_poly(st, c.q[:nl], c.N) for _ in range(2)])
    pt = si.uniform_poly(st, c.q[:nl], c.N)
    Q = 1
    for q in c.q[:nl]:
        Q *= q
    K = random.Random(5).randrange(Q)
    k = np.array([K % q for q in c.q[:nl]], dtype=np.uint64)
    cols = range(0, c.N, 97)

    def big(x):
        return oracle.crt(x[:, cols], c.q[:nl])

    A0, A1, B0, B1, PT = big(a[0]), big(a[1]), big(b[0]), big(b[1]), big(pt)
    h, s = c.hadd(a, b), c.hsub(a, b)
    assert big(h[0]) == [(x + y) % Q for x, y in zip(A0, B0)] and big(h[1]) == [(x + y) % Q for x, y in zip(A1, B1)]
    assert big(s[0]) == [(x - y) % Q for x, y in zip(A0, B0)] and big(s[1]) == [(x - y) % Q for x, y in zip(A1, B1)]
    p = c.ptadd(a, pt)
    assert big(p[0]) == [(x + y) % Q for x, y in zip(A0, PT)] and np.array_equal(p[1], a[1])
    sa = c.scalar_add(a, k)
    assert big(sa[0]) == [(x + K) % Q for x in A0] and np.array_equal(sa[1], a[1])
    sm = c.scalar_mult(a, k)
    assert big(sm[0]) == [x * K % Q for x in A0] and big(sm[1]) == [x * K % Q for x in A1]
    pm = c.ptmult(a, pt)
    assert big(pm[1]) == [x * y % Q for x, y in zip(A1, PT)]


def test_elementwise_ops_decrypt_to_slot_arithmetic(small, small_client):
    cl, D = small_client, 2.0 ** 40
    nl = small.nq
    z1, z2 = cl.random_slots(), cl.random_slots()
    a, b = cl.encrypt(z1, nl, D), cl.encrypt(z2, nl, D)
    assert _rel_err(cl.decrypt(small.hadd(a, b), D), z1 + z2) < 2.0 ** -20
    assert _rel_err(cl.decrypt(small.hsub(a, b), D), z1 - z2) < 2.0 ** -20
    pt = cl.encode_eval(z2, nl, D)
    assert _rel_err(cl.decrypt(small.ptadd(a, pt), D), z1 + z2) < 2.0 ** -20
    pm = small.ptmult(a, pt)
    assert _rel_err(cl.decrypt(pm, D * D), z1 * z2) < 2.0 ** -20
    assert _rel_err(cl.decrypt(small.rescale(pm), D * D / small.q[nl - 1]), z1 * z2) < 2.0 ** -20
    x = 0.3711
    assert _rel_err(cl.decrypt(small.scalar_add(a, cl.const_residues(x, nl, D)), D), z1 + x) < 2.0 ** -20
    assert _rel_err(cl.decrypt(small.scalar_mult(a, cl.const_residues(3, nl, 1.0)), D), 3 * z1) < 2.0 ** -20
    assert _rel_err(cl.decrypt(small.scalar_mult(a, cl.const_residues(x, nl, D)), D * D), x * z1) < 2.0 ** -20
    assert _rel_err(cl.decrypt(small.hsquare(a, cl.relin_key()), D * D), z1 * z1) < 2.0 ** -20
    assert _rel_err(cl.decrypt(small.conjugate(a, cl.conjugation_key()), D), np.conj(z1)) < 2.0 ** -20


# ------------------------------------------------------------- hoisted rotations
def test_hoisted_rotation_without_automorphism_is_the_key_switch(small, small_client):
    """steps = 0 (g = 1): one shared ModUp, inner product, ModDown and + c0 are
    exactly the single rotation's key switch, residue for residue."""
    cl = small_client
    z = cl.random_slots()
    ct = cl.encrypt(z, small.nq, 2.0 ** 40)
    rk0 = cl.rotation_key(0)
    (h,) = small.rotate_hoisted(ct, [0], [rk0])
    assert np.array_equal(h, small.rotate(ct, 0, rk0))


def test_hoisted_rotations_decrypt_to_rotations(small, small_client):
    cl, D = small_client, 2.0 ** 40
    z = cl.random_slots()
    ct = cl.encrypt(z, small.nq, D)
    steps = [1, 2, -1, 5]
    keys = [cl.rotation_key(k) for k in steps]
    outs = small.rotate_hoisted(ct, steps, keys)
    for k, o, rk in zip(steps, outs, keys):
        assert _rel_err(cl.decrypt(o, D), np.roll(z, -k)) < 2.0 ** -20, k
        # same message as the unhoisted rotation, different residues
        plain = small.rotate(ct, k, rk)
        assert _rel_err(cl.decrypt(o, D), cl.decrypt(plain, D)) < 2.0 ** -20


def test_hoisted_rotation_at_ragged_levels(mid):
    cl = Client(mid, seed=23)
    D = 2.0 ** 40
    z = cl.random_slots()
    for nl in (12, 6, 1):
        ct = cl.encrypt(z, nl, D)
        steps = [3, -7]
        outs = mid.rotate_hoisted(ct, steps, [cl.rotation_key(k) for k in steps])
        for k, o in zip(steps, outs):
            assert _rel_err(cl.decrypt(o, D), np.roll(z, -k)) < 2.0 ** -20, (nl, k)


# ------------------------------------------------------- BSGS linear transform
def _lt_keys(cl, diag_idx, n1):
    steps = {i % n1 for i in diag_idx if i % n1} | {n1 * (i // n1) for i in diag_idx if i // n1}
    return {k: cl.rotation_key(k) for k in sorted(steps)}


def test_linear_transform_decrypts_to_matrix_product(small, small_client):
    """y = M z for a matrix given by 8 of its 2048 diagonals, against numpy."""
    cl, D = small_client, 2.0 ** 40
    n = small.N // 2
    st = si.Stream(81)
    idx = [0, 1, 3, 8, 9, 21, 100, n - 1]
    diags = {i: st.complex_slots(n) for i in idx}
    z = cl.random_slots()
    ct = cl.encrypt(z, small.nq, D)
    ref = sum(diags[i] * np.roll(z, -i) for i in idx)
    outs = []
    for n1 in (8, 1, 4096):
        di, pts = cl.encode_diagonals(diags, n1, small.nq, D)
        out = small.linear_transform(ct, di, pts, n1, _lt_keys(cl, idx, n1))
        got = cl.decrypt(out, D * D)
        assert _rel_err(got, ref) < 2.0 ** -20, n1
        outs.append(got)
    assert _rel_err(outs[0], outs[1]) < 2.0 ** -20


def test_linear_transform_needs_its_keys(small, small_client):
    cl = small_client
    ct = cl.encrypt(cl.random_slots(), small.nq, 2.0 ** 40)
    diags = {0: np.ones(small.N // 2), 9: np.ones(small.N // 2)}
    di, pts = cl.encode_diagonals(diags, 8, small.nq, 2.0 ** 40)
    with pytest.raises(KeyError):
        small.linear_transform(ct, di, pts, 8, {1: cl.rotation_key(1)})     # giant step 8 missing


# ----------------------------------------------------------- bootstrapping steps
def test_modraise_is_the_centred_lift(mid):
    """Each coefficient of the raised ciphertext is the centred representative
    of the one-limb coefficient (big-integer CRT over the raised limbs)."""
    c = mid
    st = si.Stream(91)
    a = np.stack([si.uniform_poly(st, c.q[:1], c.N) for _ in range(2)])
    nl = 9
    r = c.modraise(a, nl)
    idx = list(range(nl))
    Q = 1
    for q in c.q[:nl]:
        Q *= q
    q0 = c.q[0]
    for t in range(2):
        src = c.intt(a[t][0], 0)
        got = oracle.centered(oracle.crt(c.intt_limbs(r[t], idx), c.q[:nl]), Q)
        want = [int(v) - q0 if int(v) > q0 // 2 else int(v) for v in src]
        assert got == want


def test_modraise_decrypts_to_m_plus_q0_I(small, small_client):
    cl = small_client
    z = cl.random_slots()
    ct = cl.encrypt(z, 1, 2.0 ** 30)
    raised = small.modraise(ct, small.nq)
    d1 = cl.decrypt_coeffs(ct)
    dr = cl.decrypt_coeffs(raised)
    q0 = small.q[0]
    I = [(x - y) // q0 for x, y in zip(dr, d1)]
    assert all((x - y) % q0 == 0 for x, y in zip(dr, d1))
    s1 = int(np.sum(np.abs(cl.s_coeff)))
    assert max(abs(v) for v in I) <= s1 + 1 and any(I)


def test_monomial_multiplication_rotates_the_phase(small, small_client):
    cl, D = small_client, 2.0 ** 40
    z = cl.random_slots()
    ct = cl.encrypt(z, small.nq, D)
    N = small.N
    assert _rel_err(cl.decrypt(small.mul_monomial(ct, N // 2), D), 1j * z) < 2.0 ** -20
    assert _rel_err(cl.decrypt(small.mul_monomial(ct, 3 * N // 2), D), -1j * z) < 2.0 ** -20
    # X^(N/2) twice is X^N = -1, exactly
    twice = small.mul_monomial(small.mul_monomial(ct, N // 2), N // 2)
    neg = np.stack([np.stack([(q - x) % q for x, q in zip(ct[t], small.q)]) for t in range(2)]).astype(np.uint64)
    assert np.array_equal(twice, neg)


# ------------------------------------------------------------- bootstrapping
def _dense(M, n):
    A = np.zeros((n, n), dtype=complex)
    r = np.arange(n)
    for d, v in M.items():
        A[r, (r + d) % n] += v
    return A


@pytest.mark.parametrize("n,budget", [(16, 3), (64, 3), (32, 2)])
def test_slot_dft_factorisation(n, budget):
    """The grouped butterfly stages times the bit reversal are the slot DFT
    U[j][i] = zeta^(5^j i) (zeta = exp(i pi / 2n)), and the adjoint of the
    diagonal form is the conjugate transpose."""
    from oracle import bootstrap as bt
    N = 2 * n
    U = np.exp(1j * np.pi * np.outer([pow(5, j, 2 * N) for j in range(n)], np.arange(n)) / N)
    bits = n.bit_length() - 1
    P = np.zeros((n, n))
    for i in range(n):
        P[i, brv(i, bits)] = 1
    F = np.eye(n, dtype=complex)
    for G in bt.dft_groups(n, budget):
        assert len(G) <= 2 ** (bits // budget + 2) - 1
        F = _dense(G, n) @ F
    assert np.max(np.abs(F @ P - U)) < 1e-12
    G = bt.dft_groups(n, budget)[0]
    assert np.max(np.abs(_dense(bt.diag_adjoint(G, n), n) - _dense(G, n).conj().T)) < 1e-14


def test_coefficients_to_slots_identity():
    """With real coefficients t, (1/n) U^H U t = t_lo + i t_hi (the reading
    CoeffToSlot relies on)."""
    n = 32
    N = 2 * n
    ex = np.array([pow(5, j, 2 * N) for j in range(n)])
    Ufull = np.exp(1j * np.pi * np.outer(ex, np.arange(N)) / N)
    t = np.random.default_rng(3).normal(size=N)
    Ulo = Ufull[:, :n]
    w = Ulo.conj().T @ (Ufull @ t) / n
    assert np.max(np.abs(w - (t[:n] + 1j * t[n:]))) < 1e-12


def test_chebyshev_interpolation_and_division():
    from oracle import bootstrap as bt
    f = lambda u: np.cos(2 * np.pi * (25 * u - 0.25) / 4)
    c = bt.cheb_interp(f, 119)
    u = np.linspace(-1, 1, 2001)
    assert np.max(np.abs(np.polynomial.chebyshev.chebval(u, c) - f(u))) < 1e-12
    qc, rc = bt.cheb_divide(c, 64)
    T64 = np.cos(64 * np.arccos(u))
    lhs = np.polynomial.chebyshev.chebval(u, qc) * T64 + np.polynomial.chebyshev.chebval(u, rc)
    assert np.max(np.abs(lhs - np.polynomial.chebyshev.chebval(u, c))) < 1e-12


@pytest.fixture(scope="module")
def boot12():
    """logN=12 bootstrapping context: q_0 of 60 bits, 29 q_i of 54 bits, K=10 x 60 bits, dnum=3, h=192."""
    from oracle import bootstrap as bt
    q0 = oracle.find_primes(12, 60, 1)
    q = q0 + oracle.find_primes(12, 54, 29, exclude=q0)
    p = oracle.find_primes(12, 60, 10, exclude=q)
    ctx = oracle.Context(12, q, p, 3)
    cl = Client(ctx, seed=si.workload_seed(4), hamming=192)
    prog = bt.plan(cl, q, 2.0 ** 50)
    keys = (cl.relin_key(), cl.conjugation_key(), {s: cl.rotation_key(s) for s in prog.rot_steps})
    return ctx, cl, prog, keys


def test_bootstrap_refreshes_the_ciphertext(boot12):
    """ModRaise -> CoeffToSlot -> EvalMod -> SlotToCoeff on a one-limb
    ciphertext: the result has limbs again and decrypts to the message within
    2^-12 (sparse ternary secret, h = 192)."""
    from oracle import bootstrap as bt
    ctx, cl, prog, (rlk, ck, rks) = boot12
    z = cl.random_slots()
    ct = cl.encrypt(z, 1, 2.0 ** 50)
    out = bt.run(ctx, prog, ct, rlk, ck, rks)
    assert out.shape[1] >= 12
    assert _rel_err(cl.decrypt(out, prog.out_scale), z) < 2.0 ** -12
