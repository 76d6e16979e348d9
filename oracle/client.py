"""Client side of CKKS for tests: keys, encryption, decryption to slots.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper leaves these
steps to OpenFHE (Sec. III-A); here they are built from the oracle's own
arithmetic and the seeded samplers, so that a decryption-error check never
depends on the CUDA library.
"""
from __future__ import annotations

import numpy as np

import seeded_inputs as si
from oracle import Context, crt, centered, decode, encode


class Client:
    """Secret key and helpers for one oracle context.

    ``hamming`` selects a sparse ternary secret of that weight; the default is
    a uniform ternary secret.  Streams: 1 secret, 2 key randomness, 3
    encryption randomness, 4 messages.
    """

    def __init__(self, ctx: Context, seed: int, hamming: int | None = None, sigma: float = 3.2):
        self.ctx = ctx
        self.seed = seed
        self.sigma = sigma
        st = si.Stream(seed, 1)
        N = ctx.N
        self.s_coeff = st.sparse_ternary(N, hamming) if hamming else st.ternary(N)
        self.s_eval = ctx.to_eval_full(self.s_coeff)
        self._keys = si.Stream(seed, 2)
        self._enc = si.Stream(seed, 3)
        self.msgs = si.Stream(seed, 4)
        self.all_idx = list(range(len(ctx.primes)))

    # -- keys ------------------------------------------------------------
    def _switch_key(self, sp_eval: np.ndarray) -> np.ndarray:
        c = self.ctx
        a = np.stack([si.uniform_poly(self._keys, c.primes, c.N) for _ in range(c.dnum)])
        e = np.stack([self._keys.gaussian(c.N, self.sigma) for _ in range(c.dnum)])
        return c.keygen(self.s_eval, sp_eval, a, e)

    def relin_key(self) -> np.ndarray:
        """Switching key from s^2 to s."""
        s2 = self.ctx.pointwise_mul(self.s_eval, self.s_eval, self.all_idx)
        return self._switch_key(s2)

    def rotation_key(self, steps: int) -> np.ndarray:
        """Switching key from s(X^g) to s, g = 5^steps mod 2N."""
        g = self.ctx.galois_elt(steps)
        return self._switch_key(self.ctx.automorph_eval(self.s_eval, g))

    def conjugation_key(self) -> np.ndarray:
        """Switching key from s(X^(2N-1)) to s."""
        return self._switch_key(self.ctx.automorph_eval(self.s_eval, 2 * self.ctx.N - 1))

    # -- plaintexts and constants ------------------------------------------
    def encode_eval(self, z: np.ndarray, nl: int, scale: float) -> np.ndarray:
        """Plaintext of slots z at `scale` in evaluation form under q_0..q_{nl-1}."""
        c = self.ctx
        idx = list(range(nl))
        return c.ntt_limbs(c.from_signed(encode(z, c.N, scale), idx), idx)

    def encode_diagonals(self, diags: dict, n1: int, nl: int, scale: float):
        """Plaintexts of a diagonal-method linear transform with baby step n1:
        diagonal i (slots d_i, y = sum_i d_i * rot_i(z)) is encoded pre-rotated
        by -n1 floor(i / n1).  Returns (indices, plaintexts)."""
        idx = sorted(diags)
        pts = [self.encode_eval(np.roll(np.asarray(diags[i]), n1 * (i // n1)), nl, scale) for i in idx]
        return idx, pts

    def const_residues(self, x: float, nl: int, scale: float) -> np.ndarray:
        """Residues of round(x * scale) modulo q_0..q_{nl-1}."""
        v = int(round(x * scale))
        return np.array([v % q for q in self.ctx.q[:nl]], dtype=np.uint64)

    # -- encryption --------------------------------------------------------
    def encrypt(self, z: np.ndarray, nl: int, scale: float) -> np.ndarray:
        c = self.ctx
        m = encode(z, c.N, scale)
        e = self._enc.gaussian(c.N, self.sigma)
        a = si.uniform_poly(self._enc, c.q[:nl], c.N)
        return c.encrypt(m, e, a, self.s_eval[:nl])

    def decrypt_coeffs(self, ct: np.ndarray) -> list[int]:
        """Centred integer coefficients of c0 + c1 s modulo Q_l."""
        nl = ct.shape[1]
        r = self.ctx.decrypt_residues(ct, self.s_eval[:nl])
        Q = 1
        for q in self.ctx.q[:nl]:
            Q *= q
        return centered(crt(r, self.ctx.q[:nl]), Q)

    def decrypt(self, ct: np.ndarray, scale: float) -> np.ndarray:
        return decode(self.decrypt_coeffs(ct), self.ctx.N, scale)

    def random_slots(self) -> np.ndarray:
        return self.msgs.complex_slots(self.ctx.N // 2)
