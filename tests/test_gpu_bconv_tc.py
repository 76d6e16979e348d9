"""Base conversion on the tensor cores (Eq. 1 as an exact byte-matrix product,
fp16 x fp16 -> fp32): residue for residue against the oracle on extreme
inputs, on contexts where only one of ModUp / ModDown has tensor-core images
(the other converts on the integer kernel), with the device status word left
clear, and a bounded device wait that runs out.  The standard parameter sets
(SMALL, MID, FULL, WIDE) run every conversion on the tensor cores; their
ModUp / ModDown / key-switching parity at every level is in test_gpu_parity."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, find_primes, to_device, to_host  # noqa: E402


def contexts(logN, nq, nk, dnum, q_bits=54, p_bits=60):
    q = find_primes(logN, q_bits, nq)
    p = find_primes(logN, p_bits, nk, exclude=q)
    return Context(logN, q, p, dnum), oracle.Context(logN, q, p, dnum)


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def check_modup_moddown(g, o, d_host, x_host, nl, what):
    beta = g.beta(nl)
    ext = torch.zeros(beta * (nl + o.nk) * o.N, dtype=torch.int64, device="cuda")
    g.modup(to_device(d_host), nl, ext)
    out = torch.zeros(nl * o.N, dtype=torch.int64, device="cuda")
    g.moddown(to_device(x_host), nl, out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(ext).reshape(beta, nl + o.nk, o.N), o.modup(d_host)), "modup, %s, nl=%d" % (what, nl)
    assert np.array_equal(to_host(out).reshape(nl, o.N), o.moddown(x_host)), "moddown, %s, nl=%d" % (what, nl)


@pytest.mark.parametrize("name", ["SMALL", "MID", "FULL", "WIDE"])
def test_standard_sets_convert_on_tensor_cores(name):
    need_gpu()
    P = getattr(si, name)
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    g = Context(P.logN, q, p, P.dnum)
    assert g.tensor_bconv
    g.close()


@pytest.mark.parametrize("name", ["SMALL", "MID", "WIDE"])
def test_extreme_residues(name):
    """Every residue q_i - 1 (the largest bytes a residue has), every residue
    0, and alternating rows: the largest partial sums of the byte product."""
    need_gpu()
    P = getattr(si, name)
    g, o = contexts(P.logN, P.nq, P.nk, P.dnum, P.q_bits, P.p_bits)
    for nl in sorted({P.nq, max(1, P.nq - 1)}):
        top = np.stack([np.full(o.N, qi - 1, dtype=np.uint64) for qi in o.q[:nl]])
        topx = np.stack([np.full(o.N, qi - 1, dtype=np.uint64) for qi in o.q[:nl] + o.p])
        check_modup_moddown(g, o, top, topx, nl, "q - 1")
        check_modup_moddown(g, o, np.zeros_like(top), np.zeros_like(topx), nl, "zero")
        alt = top.copy()
        alt[:, 1::2] = 0
        altx = topx.copy()
        altx[:, ::2] = 0
        check_modup_moddown(g, o, alt, altx, nl, "alternating")
    assert g.status() == 0
    g.close()


@pytest.mark.parametrize("shape", [(34, 3, 2), (20, 17, 2)], ids=["modup-integer", "moddown-integer"])
def test_one_conversion_on_the_integer_kernel(shape):
    """(L, K, dnum) = (34, 3, 2): digits of 17 primes, ModUp on the integer
    kernel, ModDown (K = 3) on the tensor cores; (20, 17, 2): the reverse."""
    need_gpu()
    nq, nk, dnum = shape
    g, o = contexts(12, nq, nk, dnum)
    assert not g.tensor_bconv
    st = si.Stream(1500 + nq, 1)
    rlk = np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])
    drlk = g.relin_key(to_device(rlk))
    for nl in (nq, nq - 5):
        d = si.uniform_poly(st, o.q[:nl], o.N)
        x = si.uniform_poly(st, o.q[:nl] + o.p, o.N)
        check_modup_moddown(g, o, d, x, nl, "random")
        a = np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])
        b = np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])
        m = torch.empty(2 * nl * o.N, dtype=torch.int64, device="cuda")
        g.hmult(to_device(a), to_device(b), nl, drlk, m)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(m).reshape(a.shape), o.hmult(a, b, rlk)), nl
    # round-to-nearest: the centred ModDown conversion on the same kernels
    g.set_rounding(True)
    o.set_rounding(True)
    for nl in (nq, nq - 5):
        d = si.uniform_poly(st, o.q[:nl], o.N)
        x = si.uniform_poly(st, o.q[:nl] + o.p, o.N)
        check_modup_moddown(g, o, d, x, nl, "random, nearest")
    assert g.status() == 0
    g.close()


@pytest.mark.parametrize("name", ["SMALL", "FULL", "WIDE"])
def test_centred_conversion_on_extreme_residues(name):
    """Round-to-nearest ModDown on special limbs whose converted residues sit
    at the centring boundary ((p - 1) / 2 and (p + 1) / 2), at p - 1 and at 0
    (every source in the upper half: the largest correction the tensor-core
    sums carry)."""
    need_gpu()
    P = getattr(si, name)
    g, o = contexts(P.logN, P.nq, P.nk, P.dnum, P.q_bits, P.p_bits)
    g.set_rounding(True)
    o.set_rounding(True)
    nl = P.nq
    st = si.Stream(1600, 2)
    d = si.uniform_poly(st, o.q[:nl], o.N)
    pidx = [o.nq + k for k in range(o.nk)]
    for what in ("boundary", "all upper", "zero"):
        x = si.uniform_poly(st, o.q[:nl] + o.p, o.N)
        # choose the coefficient form of the special limbs so that the
        # conversion's sources [x_k Phat_k^-1]_{p_k} take the wanted values
        coef = np.empty((o.nk, o.N), dtype=np.uint64)
        for k, p in enumerate(o.p):
            Phat = 1
            for m, pm in enumerate(o.p):
                if m != k:
                    Phat *= pm
            if what == "boundary":
                want = [(p - 1) // 2, (p + 1) // 2, p - 1, 0, 1]
                vals = np.resize(np.array(want, dtype=object), o.N)
            elif what == "all upper":
                vals = np.full(o.N, p - 1, dtype=object)
            else:
                vals = np.zeros(o.N, dtype=object)
            coef[k] = np.array([int(v) * (Phat % p) % p for v in vals], dtype=np.uint64)
        x[nl:] = o.ntt_limbs(coef, pidx)
        check_modup_moddown(g, o, d, x, nl, what)
    assert g.status() == 0
    g.close()


def test_full_size_ragged_levels_and_status():
    """logN=16, 30 limbs, K=10, dnum=3: HMult at a level whose last digit has
    one prime (nl = 21) and at one with an odd target count (nl = 28), then
    the status word."""
    need_gpu()
    P = si.FULL
    g, o = contexts(P.logN, P.nq, P.nk, P.dnum, P.q_bits, P.p_bits)
    st = si.Stream(1510, 2)
    rlk = np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])
    drlk = g.relin_key(to_device(rlk))
    for nl in (21, 28):
        a = np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])
        b = np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])
        m = torch.empty(2 * nl * o.N, dtype=torch.int64, device="cuda")
        g.hmult(to_device(a), to_device(b), nl, drlk, m)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(m).reshape(a.shape), o.hmult(a, b, rlk)), nl
    assert g.status() == 0
    g.close()


def test_a_wait_that_runs_out_is_reported_and_the_context_stays_usable():
    """The bounded-wait machinery of the tensor-core conversion: a device wait
    that nothing completes gives up after its limit (1 ms here), sets the
    status bit, and the context then runs a key switch bit-exactly."""
    need_gpu()
    P = si.MID
    g, o = contexts(P.logN, P.nq, P.nk, P.dnum, P.q_bits, P.p_bits)
    assert g.status() == 0
    g.selftest_wait(1000)
    assert g.status() == 1            # reported once ...
    assert g.status() == 0            # ... and cleared
    st = si.Stream(1520, 1)
    d = si.uniform_poly(st, o.q, o.N)
    x = si.uniform_poly(st, o.q + o.p, o.N)
    check_modup_moddown(g, o, d, x, P.nq, "after a timeout")
    assert g.status() == 0
    g.close()


@pytest.mark.parametrize("name", ["MID", "FULL"])
def test_a_stalled_conversion_aborts_frees_its_tensor_memory_and_reports(name):
    """The conversion's abort path: one CTA never receives its first tile, its
    waits (limited to 5 ms here) run out, every role of it leaves, and it frees
    its tensor memory; the status bit is set once.  Then two rounds of ModUp
    and ModDown conversions, which allocate tensor memory on every SM, are
    bit-exact with the oracle and report nothing."""
    need_gpu()
    P = getattr(si, name)
    g, o = contexts(P.logN, P.nq, P.nk, P.dnum, P.q_bits, P.p_bits)
    assert g.status() == 0
    g.selftest_conversion(5000)
    assert g.status() == 1            # reported once ...
    assert g.status() == 0            # ... and cleared
    st = si.Stream(1521, 1)
    for rnd in range(2):
        d = si.uniform_poly(st, o.q, o.N)
        x = si.uniform_poly(st, o.q + o.p, o.N)
        check_modup_moddown(g, o, d, x, P.nq, "after a stalled conversion, round %d" % rnd)
    assert g.status() == 0
    g.close()
