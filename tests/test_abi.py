"""Host-side checks of the C ABI (no GPU needed): every symbol declared in
include/*.h is exported by the library, host helpers agree with the oracle's
independent implementation, and argument errors are reported before any
device work."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_2507_04775_gb300 import build as libbuild
from paper_2507_04775_gb300 import fides

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return fides.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fides_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "fides_hmult" in names and "fides_ctx_create" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(fides.EXPORTS) <= set(names)


@pytest.mark.parametrize("logN,bits,count", [(12, 40, 3), (12, 50, 1), (16, 54, 30), (16, 60, 10)])
def test_find_primes_agrees_with_oracle(L, logN, bits, count):
    assert fides.find_primes(logN, bits, count) == oracle.find_primes(logN, bits, count)
    q = fides.find_primes(logN, bits, count)
    assert fides.find_primes(logN, bits, 2, exclude=q[:1]) == q[1:3] if count > 2 else True


def _create(L, logN, q, p, dnum):
    arr = np.ascontiguousarray(q + p, dtype=np.uint64)
    h = ctypes.c_void_p()
    rc = L.fides_ctx_create(logN, len(q), dnum, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(p),
                            ctypes.byref(h))
    return rc, h


def test_ctx_create_rejects_bad_parameters_before_device_work(L):
    q = fides.find_primes(12, 40, 3)
    p = fides.find_primes(12, 50, 1, exclude=q)
    for logN in (11, 18):                                         # ring degrees outside 2^12..2^17
        rc, h = _create(L, logN, q, p, 3)
        assert rc == -2 and not h.value and b"logN" in L.fides_last_error()
    rc, h = _create(L, 12, q[:2] + [q[2] + 2], p, 3)          # not prime
    assert rc == -6 and not h.value
    rc, h = _create(L, 12, q, [q[0]], 3)                        # repeated prime
    assert rc == -6
    rc, h = _create(L, 12, q, p, 4)                             # dnum > L
    assert rc == -1
    q16 = fides.find_primes(12, 54, 2)
    rc, h = _create(L, 16, q16, p, 1)                           # 2N = 2^17 does not divide q - 1
    assert rc == -6


def test_find_primes_argument_errors(L):
    with pytest.raises(fides.FidesError):
        fides.find_primes(16, 62, 1)
    with pytest.raises(fides.FidesError):
        fides.find_primes(16, 10, 1)


def test_key_handle_argument_errors_on_the_host(L):
    """Key registration refuses missing arguments before touching a device;
    the handle helpers accept NULL."""
    h = ctypes.c_void_p(1)
    assert L.fides_key_register(None, ctypes.c_void_p(4096), 0, ctypes.byref(h)) == -1
    assert h.value is None
    assert L.fides_key_register(None, None, 0, None) == -1
    assert L.fides_key_galois(None) == 0
    L.fides_key_destroy(None)
    assert L.fides_keyswitch(None, None, 1, None, None, None, None) == -1
    assert L.fides_rotate(None, None, 1, None, None, None) == -1


def test_version(L):
    assert "sm_103a" in fides.version()
