"""Host-side serialisation of ciphertexts and switching keys.

A file is a 48-byte little-endian header followed by the residues as
little-endian u64 words, limb-major, exactly the device layout:

  magic     8 bytes   b"FIDESCT1" (ciphertext) or b"FIDESKY1" (switching key)
  logN      u32
  n_limbs   u32       ciphertext limbs, or L + K for a key
  n_polys   u32       2 for a ciphertext, 2 * dnum for a key
  reserved  u32       0
  scale     f64       the ciphertext's scale (0 for a key)
  primes    16 bytes  SHA-256 prefix of the context's primes (q then p, u64 LE)

Loading checks the magic, the ring degree, the primes and the file size, and
raises ValueError on any mismatch, so a ciphertext cannot be read into a
context with other moduli.
"""
from __future__ import annotations

import hashlib
import struct

import numpy as np

_HEADER = struct.Struct("<8sIIIId16s")
CT_MAGIC, KEY_MAGIC = b"FIDESCT1", b"FIDESKY1"


def primes_digest(ctx) -> bytes:
    return hashlib.sha256(np.asarray(list(ctx.q) + list(ctx.p), dtype="<u8").tobytes()).digest()[:16]


def _as_host(x) -> np.ndarray:
    """The residues as a host uint64 array (int64 input keeps its bits)."""
    if hasattr(x, "detach"):                       # a torch tensor (device or host)
        x = x.detach().cpu().contiguous().numpy()
    x = np.ascontiguousarray(x)
    if x.dtype == np.int64:
        return x.view(np.uint64)
    return x.astype(np.uint64, copy=False)


def _write(path, magic, ctx, data, n_limbs, n_polys, scale):
    arr = _as_host(data).reshape(-1)
    if arr.size != n_polys * n_limbs * ctx.N:
        raise ValueError("data holds %d words, expected %d" % (arr.size, n_polys * n_limbs * ctx.N))
    with open(path, "wb") as f:
        f.write(_HEADER.pack(magic, ctx.logN, n_limbs, n_polys, 0, float(scale), primes_digest(ctx)))
        f.write(arr.astype("<u8", copy=False).tobytes())


def _read(path, magic, ctx):
    with open(path, "rb") as f:
        head = f.read(_HEADER.size)
        if len(head) != _HEADER.size:
            raise ValueError("%s: truncated header" % path)
        mg, logN, n_limbs, n_polys, _, scale, dig = _HEADER.unpack(head)
        if mg != magic:
            raise ValueError("%s: not a %s file" % (path, magic.decode()))
        if logN != ctx.logN or dig != primes_digest(ctx):
            raise ValueError("%s: written for another ring or other primes" % path)
        words = n_polys * n_limbs * (1 << logN)
        body = f.read()
    if len(body) != 8 * words:
        raise ValueError("%s: %d data bytes, expected %d" % (path, len(body), 8 * words))
    arr = np.frombuffer(body, dtype="<u8").astype(np.uint64).reshape(n_polys, n_limbs, 1 << logN)
    return arr, n_limbs, scale


def save_ciphertext(path, ctx, ct, n_limbs: int, scale: float):
    """ct: [2][n_limbs][N] residues (numpy or torch, int64 or uint64 bits)."""
    _write(path, CT_MAGIC, ctx, ct, n_limbs, 2, scale)


def load_ciphertext(path, ctx):
    """(array [2][n_limbs][N] uint64, n_limbs, scale)."""
    return _read(path, CT_MAGIC, ctx)


def save_key(path, ctx, key):
    """key: [dnum][2][L+K][N]."""
    _write(path, KEY_MAGIC, ctx, key, len(ctx.q) + len(ctx.p), 2 * ctx.dnum, 0.0)


def load_key(path, ctx) -> np.ndarray:
    arr, _, _ = _read(path, KEY_MAGIC, ctx)
    return arr.reshape(ctx.dnum, 2, len(ctx.q) + len(ctx.p), ctx.N)
