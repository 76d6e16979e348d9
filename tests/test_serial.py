"""Ciphertext and key files: round trips, and every mismatch refused."""
import types

import numpy as np
import pytest

import seeded_inputs as si
from paper_2507_04775_gb300 import serial

torch = pytest.importorskip("torch")


def ctx_like(q, p, logN=4, dnum=2):
    return types.SimpleNamespace(logN=logN, N=1 << logN, q=list(q), p=list(p), dnum=dnum)


Q, P = [97, 193, 257], [353, 449]


def test_ciphertext_round_trip(tmp_path):
    c = ctx_like(Q, P)
    st = si.Stream(3)
    ct = np.stack([si.uniform_poly(st, Q, c.N) for _ in range(2)])
    f = tmp_path / "a.ct"
    serial.save_ciphertext(f, c, ct, 3, 2.0 ** 40)
    back, nl, scale = serial.load_ciphertext(f, c)
    assert np.array_equal(back, ct) and nl == 3 and scale == 2.0 ** 40
    # a torch int64 tensor with the same bits writes the same file
    g = tmp_path / "b.ct"
    serial.save_ciphertext(g, c, torch.from_numpy(ct.view(np.int64).copy()), 3, 2.0 ** 40)
    assert f.read_bytes() == g.read_bytes()
    assert len(f.read_bytes()) == 48 + 8 * ct.size


def test_key_round_trip(tmp_path):
    c = ctx_like(Q, P)
    st = si.Stream(4)
    key = np.stack([np.stack([si.uniform_poly(st, Q + P, c.N) for _ in range(2)]) for _ in range(c.dnum)])
    f = tmp_path / "k.key"
    serial.save_key(f, c, key)
    assert np.array_equal(serial.load_key(f, c), key)
    with pytest.raises(ValueError):
        serial.load_ciphertext(f, c)                      # a key is not a ciphertext


def test_mismatches_are_refused(tmp_path):
    c = ctx_like(Q, P)
    ct = np.zeros((2, 3, c.N), dtype=np.uint64)
    f = tmp_path / "a.ct"
    serial.save_ciphertext(f, c, ct, 3, 1.0)
    with pytest.raises(ValueError):
        serial.load_ciphertext(f, ctx_like([97, 193, 769], P))        # other primes
    with pytest.raises(ValueError):
        serial.load_ciphertext(f, ctx_like(Q, P, logN=5))              # other ring
    raw = f.read_bytes()
    (tmp_path / "t.ct").write_bytes(raw[:-8])
    with pytest.raises(ValueError):
        serial.load_ciphertext(tmp_path / "t.ct", c)                   # truncated
    with pytest.raises(ValueError):
        serial.save_ciphertext(tmp_path / "x.ct", c, ct[:, :2], 3, 1.0)  # wrong size
