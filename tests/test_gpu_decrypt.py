"""Decryption of GPU results made with real keys: the slot error against the
FP64 result, stated as a number (relative: max |dec - ref| / max(1, max |ref|)).

Keys, encryption and decryption come from the oracle's client (RLWE keys of a
uniform ternary secret, Gaussian errors sigma = 3.2); the HMult+relin,
HRotate and Rescale are the library's.  Two parameter sets:
  - logN=12, 3 x 40-bit q, K=1, dnum=3, scale 2^40 (q ~ scale);
  - logN=16, 30 x 54-bit q, K=10, dnum=3, scale 2^40 -- the bench workload --
    with HRotate by 1 and 2^14 slots, and again at scale 2^54 (q ~ scale,
    Table II), where Rescale keeps the precision;
each under both rounding modes of the context (fides_ctx_set_rounding).

Floor rounding leaves an error of nonzero mean on every coefficient of a
key-switch output (the conversion term u in [0, K) plus the floor) and of a
Rescale output (the floor); decoding sums it coherently into the few slots
whose evaluation point is near 1, so at logN=16 a rotation decrypts only to
about 2^-14 and a Rescale at scale 2^40 to about 2^-4 there (the median slot
is at 2^-25 and 2^-13).  Round-to-nearest removes the mean.  Bounds checked:
  - HMult+relin (scale 2^80): 2^-20 in both modes;
  - HRotate (scale 2^40): 2^-20 with nearest (and at logN=12 with floor);
    with floor at logN=16 the number is stated and checked below 2^-12;
  - Rescale from scale 2^80 by a 54-bit prime leaves scale 2^26: about 2^-10
    with nearest, checked below 2^-8 (floor: stated, below 2^-2); at scale
    2^54 (and at logN=12, where q ~ scale) 2^-20 with nearest.
The errors are printed (pytest -s shows them).
"""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle.client import Client

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2507_04775_gb300 import Context, find_primes, to_device, to_host  # noqa: E402


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(1.0, float(np.max(np.abs(ref)))))


def log2(x):
    return math.log2(x) if x > 0 else float("-inf")


@pytest.mark.parametrize("nearest", [False, True], ids=["floor", "nearest"])
@pytest.mark.parametrize("P", [si.SMALL, si.FULL], ids=lambda P: P.name)
def test_decrypts_through_gpu_with_real_keys(P, nearest):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q = find_primes(P.logN, P.q_bits, P.nq)
    p = find_primes(P.logN, P.p_bits, P.nk, exclude=q)
    g, o = Context(P.logN, q, p, P.dnum), oracle.Context(P.logN, q, p, P.dnum)
    g.set_rounding(nearest)
    cl = Client(o, seed=si.workload_seed(0 if P is si.SMALL else 1))
    N, nl = o.N, P.nq
    full = P is si.FULL
    rot_steps = [1, 1 << 14] if full else [3]
    rlk = g.relin_key(to_device(cl.relin_key()))
    rks = {k: g.rotation_key(to_device(cl.rotation_key(k)), k) for k in rot_steps}
    report = {}
    for delta in [2.0**40] + ([2.0**54] if full else []):
        z1, z2 = cl.random_slots(), cl.random_slots()
        a, b = cl.encrypt(z1, nl, delta), cl.encrypt(z2, nl, delta)
        da, db = to_device(a), to_device(b)
        ref = z1 * z2
        out = torch.zeros(2 * nl * N, dtype=torch.int64, device="cuda")
        s = g.hmult(da, db, nl, rlk, out, delta, delta)
        e_hm = rel_err(cl.decrypt(to_host(out).reshape(2, nl, N), s), ref)
        rs = torch.zeros(2 * (nl - 1) * N, dtype=torch.int64, device="cuda")
        s2 = g.rescale(out, nl, rs, s)
        e_rs = rel_err(cl.decrypt(to_host(rs).reshape(2, nl - 1, N), s2), ref)
        fused = torch.zeros_like(rs)
        s4 = g.hmult_rescale(da, db, nl, rlk, fused, delta, delta)
        assert s4 == s2
        e_fu = rel_err(cl.decrypt(to_host(fused).reshape(2, nl - 1, N), s4), ref)
        tag = "scale 2^%d" % round(math.log2(delta))
        report[tag] = {"hmult": e_hm, "rescale": e_rs, "hmult_rescale": e_fu}
        assert e_hm < 2.0**-20, (tag, "hmult", log2(e_hm))
        q_like = delta >= q[nl - 1] / 2          # Rescale lands back near the scale
        if nearest:
            bound_rs = 2.0**-20 if q_like else 2.0**-8
        else:
            bound_rs = 2.0**-20 if (q_like and not full) else (2.0**-16 if q_like else 2.0**-2)
        for name in ("rescale", "hmult_rescale"):
            assert report[tag][name] < bound_rs, (tag, name, log2(report[tag][name]))
        if delta == 2.0**40:
            for k, key in rks.items():
                rot = torch.zeros_like(out)
                g.rotate(da, nl, k, key, rot)
                e = rel_err(cl.decrypt(to_host(rot).reshape(2, nl, N), delta), np.roll(z1, -k))
                report[tag]["rotate_%d" % k] = e
                bound = 2.0**-20 if (nearest or not full) else 2.0**-12
                assert e < bound, (tag, "rotate", k, log2(e))
    print("\ndecryption error, %s, %s rounding (log2 of relative slot error):"
          % (P.name, "nearest" if nearest else "floor"))
    for tag, r in report.items():
        print("  %s: %s" % (tag, ", ".join("%s %.1f" % (k, log2(v)) for k, v in r.items())))
    for key in [rlk, *rks.values()]:
        key.close()
    g.close()
