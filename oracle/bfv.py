"""BFV primitives of the oracle (Sec. 2.3): batch encoding, symmetric
encryption, decryption, HAdd / CMult / PMult and hoisted rotation.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Random draws: every random polynomial comes from a SplitMix64 stream keyed
by (seed, tag, a, b); the tags below name which quantity a stream feeds.
"""
from __future__ import annotations

import numpy as np

from . import _clib
from .params import Params, centred, slot_exponents

TAG_SECRET = 1  # secret key s, ternary
TAG_ENC_A = 2  # ciphertext mask a, per ciphertext index
TAG_ENC_E = 3  # ciphertext error e, per ciphertext index
TAG_KSK_A = 4  # Galois-key mask, per (Galois element, digit)
TAG_KSK_E = 5  # Galois-key error, per (Galois element, digit)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _qarr(P: Params):
    return _u64(P.q), _u64(P.psi)


# ------------------------------------------------------------------ sampling
def stream_key(seed: int, tag: int, a: int = 0, b: int = 0) -> int:
    return int(_clib.lib().orc_stream_key(seed, tag, a, b))


def sample_ternary(P: Params, key: int) -> np.ndarray:
    out = np.zeros(P.N, dtype=np.int64)
    _clib.lib().orc_sample_ternary(key, P.N, out)
    return out


def sample_uniform(P: Params, key: int) -> np.ndarray:
    q, _ = _qarr(P)
    out = np.zeros(P.L * P.N, dtype=np.uint64)
    _clib.lib().orc_sample_uniform(key, P.L, P.N, q, out)
    return out.reshape(P.L, P.N)


def sample_gauss(P: Params, key: int, n: int | None = None) -> np.ndarray:
    n = P.N if n is None else n
    out = np.zeros(n, dtype=np.int64)
    _clib.lib().orc_sample_gauss(key, n, P.sigma2[0], P.sigma2[1], P.bound, out)
    return out


# ------------------------------------------------------------------ encoding
def _slot_ntt_index(P: Params) -> np.ndarray:
    """NTT position (natural order, A[k] = m(zeta^(2k+1))) of every flat slot."""
    return (np.array(slot_exponents(P.N), dtype=np.int64) - 1) // 2


def encode(P: Params, slots) -> np.ndarray:
    """Batch encoding (Sec. 2.3): slot values (length N, flat index r*N/2+i)
    -> plaintext polynomial coefficients in [0, t)."""
    v = np.zeros(P.N, dtype=np.uint64)
    v[_slot_ntt_index(P)] = np.mod(np.asarray(slots, dtype=np.int64), P.t).astype(np.uint64)
    _clib.lib().orc_ntt_inv(v, P.N, P.t, P.zeta)
    return v


def decode(P: Params, m) -> np.ndarray:
    v = _u64(np.mod(np.asarray(m, dtype=np.int64), P.t))
    _clib.lib().orc_ntt_fwd(v, P.N, P.t, P.zeta)
    return v[_slot_ntt_index(P)].astype(np.int64)


# ------------------------------------------------------------------ keys
def keygen(P: Params, seed: int) -> np.ndarray:
    """Secret key s: ternary coefficients in {-1, 0, 1}."""
    return sample_ternary(P, stream_key(seed, TAG_SECRET))


def galois_key(P: Params, s: np.ndarray, g: int, seed: int) -> np.ndarray:
    """Key-switching key for sigma_g: [L*l][2][L][N] (b, a) per digit."""
    Ll = P.L * P.l
    a_all = np.zeros((Ll, P.L, P.N), dtype=np.uint64)
    e_all = np.zeros((Ll, P.N), dtype=np.int64)
    for dd in range(Ll):
        a_all[dd] = sample_uniform(P, stream_key(seed, TAG_KSK_A, g, dd))
        e_all[dd] = sample_gauss(P, stream_key(seed, TAG_KSK_E, g, dd))
    q, psi = _qarr(P)
    out = np.zeros((Ll, 2, P.L, P.N), dtype=np.uint64)
    _clib.lib().orc_galois_key(_i64(s), g, a_all, e_all, q, psi, P.L, P.N, P.w, P.l, out)
    return out


# ------------------------------------------------------------------ enc / dec
def delta_mod(P: Params) -> np.ndarray:
    return _u64([P.delta % qi for qi in P.q])


def encrypt(P: Params, s: np.ndarray, m: np.ndarray, seed: int, index: int) -> np.ndarray:
    """Symmetric BFV encryption (Sec. 2.3): (c0, c1) = ([Delta m + a s + e]_q, [-a]_q).
    `index` picks the random streams for this ciphertext."""
    a = sample_uniform(P, stream_key(seed, TAG_ENC_A, index))
    e = sample_gauss(P, stream_key(seed, TAG_ENC_E, index))
    q, psi = _qarr(P)
    ct = np.zeros((2, P.L, P.N), dtype=np.uint64)
    _clib.lib().orc_encrypt(_u64(m), _i64(s), a, e, delta_mod(P), q, psi, P.L, P.N, ct)
    return ct


def crt_lift(P: Params, residues: np.ndarray) -> list[int]:
    """Residues [L][N] -> centred integers in (-Q/2, Q/2] (Chinese remaindering)."""
    Q = P.Q
    basis = []
    for qi in P.q:
        Qi = Q // qi
        basis.append(Qi * pow(Qi, -1, qi))
    out = []
    for n in range(P.N):
        x = 0
        for k in range(P.L):
            x += int(residues[k, n]) * basis[k]
        out.append(centred(x, Q))
    return out


def phase(P: Params, s: np.ndarray, ct: np.ndarray) -> list[int]:
    """[c0 + c1 s]_q as centred integers (= Delta m + v, Sec. 2.3)."""
    q, psi = _qarr(P)
    out = np.zeros((P.L, P.N), dtype=np.uint64)
    _clib.lib().orc_dot_secret(_u64(ct), _i64(s), q, psi, P.L, P.N, out)
    return crt_lift(P, out)


def decrypt(P: Params, s: np.ndarray, ct: np.ndarray) -> np.ndarray:
    """Dec(c) = [ round(t [c0 + c1 s]_q / q) ]_t (Sec. 2.3), rounding half up."""
    Q, t = P.Q, P.t
    x = phase(P, s, ct)
    return np.array([((2 * t * xi + Q) // (2 * Q)) % t for xi in x], dtype=np.int64)


def noise(P: Params, s: np.ndarray, ct: np.ndarray, m) -> int:
    """||v||_inf with [c0 + c1 s]_q = Delta m + v (Sec. 2.3); m the expected plaintext."""
    Q = P.Q
    x = phase(P, s, ct)
    d = P.delta
    return max(abs(centred(xi - d * int(mi), Q)) for xi, mi in zip(x, np.asarray(m).tolist()))


# ------------------------------------------------------------------ operations
def hadd(P: Params, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """HAdd: coefficient-wise sum mod q_k."""
    q = np.array(P.q, dtype=object).reshape(1, P.L, 1)
    return ((a.astype(object) + b.astype(object)) % q).astype(np.uint64)


def cmult_add(P: Params, acc: np.ndarray, x: np.ndarray, scalar: int) -> None:
    """acc <- acc + CMult(x, scalar), reduced at once."""
    q, _ = _qarr(P)
    _clib.lib().orc_cmult_add(acc, _u64(x), int(scalar), q, P.L, P.N)


def cmult(P: Params, x: np.ndarray, scalar: int) -> np.ndarray:
    acc = np.zeros_like(x, dtype=np.uint64)
    cmult_add(P, acc, x, scalar)
    return acc


def pmult(P: Params, ct: np.ndarray, pt_centred) -> np.ndarray:
    """PMult: multiply both polynomials by the plaintext polynomial, given
    with centred integer coefficients."""
    q, psi = _qarr(P)
    out = np.zeros((2, P.L, P.N), dtype=np.uint64)
    _clib.lib().orc_pmult(_u64(ct), _i64(pt_centred), q, psi, P.L, P.N, out)
    return out


def decompose(P: Params, ct: np.ndarray) -> np.ndarray:
    """Hoisting step 1: digits of c1 in base 2^w, [L*l][N]."""
    d = np.zeros((P.L * P.l, P.N), dtype=np.uint64)
    _clib.lib().orc_decompose(_u64(ct[1]), P.L, P.N, P.w, P.l, d)
    return d


def rotate_hoisted(P: Params, ct: np.ndarray, digits: np.ndarray, ksk: np.ndarray, g: int) -> np.ndarray:
    """Hoisting step 2: automorphism sigma_g of c0 and of the digits, then key product."""
    q, psi = _qarr(P)
    out = np.zeros((2, P.L, P.N), dtype=np.uint64)
    _clib.lib().orc_rotate_hoisted(_u64(ct), _u64(digits), _u64(ksk), g, q, psi, P.L, P.N, P.l, out)
    return out


def hrot(P: Params, ct: np.ndarray, ksk: np.ndarray, g: int) -> np.ndarray:
    """HRot by the Galois element g (no hoisting across calls)."""
    return rotate_hoisted(P, ct, decompose(P, ct), ksk, g)


def rotation_element(P: Params, step: int) -> int:
    """Galois element of a left rotation of both slot rows by `step`: 3^step mod 2N."""
    return pow(3, step % (P.N // 2), 2 * P.N)


def row_swap_element(P: Params) -> int:
    """Galois element exchanging the two slot rows: 2N - 1."""
    return 2 * P.N - 1


def hadamard_plaintext(P: Params) -> np.ndarray:
    """The [k, -k] plaintext (row 0 = k, row 1 = -k), centred coefficients."""
    half = P.N // 2
    m = encode(P, [P.k] * half + [-P.k] * half)
    return np.array([centred(int(x), P.t) for x in m], dtype=np.int64)


def noise_of(P: Params, s: np.ndarray, ct: np.ndarray) -> int:
    """||v||_inf measured against the message the ciphertext decrypts to."""
    return noise(P, s, ct, decrypt(P, s, ct))
