"""GPU parity of the baby-step giant-step linear transform (hoisted baby
steps, plaintext multiply-accumulate per giant step, HRotate, HAdd) with the
oracle's, residue for residue, for several splits n1 and levels."""
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


def rand_key(st, o):
    return np.stack([np.stack([si.uniform_poly(st, o.primes, o.N) for _ in range(2)]) for _ in range(o.dnum)])


def needed_steps(idx, n1):
    return sorted({i % n1 for i in idx if i % n1} | {n1 * (i // n1) for i in idx if i // n1})


@pytest.mark.parametrize("P,nl,idx,n1", [
    (si.MID, 12, [0, 1, 3, 8, 9, 21, 100, 2047], 8),
    (si.MID, 5, [0, 1, 3, 8, 9, 21, 100, 2047], 1),
    (si.MID, 7, [2, 5, 11], 4096),
    (si.MID, 12, [1], 8),
    (si.FULL, 30, [0, 1, 2, 16, 17, 300, 32767], 16),
], ids=["logN12-L12-n1_8", "logN12-L5-n1_1", "logN12-L7-baby-only", "logN12-one-diag", "logN16-L30-n1_16"])
def test_linear_transform_matches_oracle(P, nl, idx, n1):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = make_pair(P)
    st = si.Stream(901, nl)
    a = np.stack([si.uniform_poly(st, o.q[:nl], o.N) for _ in range(2)])
    pts = [si.uniform_poly(st, o.q[:nl], o.N) for _ in idx]
    keys = {k: rand_key(st, o) for k in needed_steps(idx, n1)}
    ref = o.linear_transform(a, idx, pts, n1, keys)
    da = to_device(a)
    out = torch.empty_like(da)
    sc = g.linear_transform(da, nl, idx, [to_device(p) for p in pts], n1,
                            [g.rotation_key(to_device(v), k) for k, v in keys.items()],
                            out, scale=2.0 ** 40, pt_scale=2.0 ** 30)
    torch.cuda.synchronize()
    assert sc == 2.0 ** 70
    assert np.array_equal(to_host(out).reshape(a.shape), ref)
    g.close()


def test_linear_transform_rejects_before_queueing():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, o = make_pair(si.SMALL)
    nl = o.nq
    st = si.Stream(902)
    da = to_device(np.stack([si.uniform_poly(st, o.q, o.N) for _ in range(2)]))
    pt = to_device(si.uniform_poly(st, o.q, o.N))
    buf = to_device(rand_key(st, o))
    out = torch.empty_like(da)
    with pytest.raises(FidesError) as e:
        g.linear_transform(da, nl, [0, 9], [pt, pt], 8, [g.rotation_key(buf, 1)], out)   # giant step 8 has no key
    assert e.value.code == -7
    with pytest.raises(FidesError) as e:                                 # a key of step 8 registered as step 9
        g.linear_transform(da, nl, [0, 8], [pt, pt], 8, [g.register_key(buf, g.galois_elt(9))], out)
    assert e.value.code == -7
    with pytest.raises(FidesError):
        g.linear_transform(da, nl, [3, 3], [pt, pt], 8, [g.rotation_key(buf, 3)], out)   # repeated diagonal
    with pytest.raises(FidesError):
        g.linear_transform(da, nl, [o.N // 2], [pt], 8, [], out)         # out of range
    g.close()
