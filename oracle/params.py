"""Encryption-parameter selection, written from the paper's Sec. 3.2.1.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain Python integers.

The procedure (Sec. 3.2.1, "Optimal Parameter Selection"):
  1. pick (n, p, q) with p = 1 (mod 2n) and q = 1 (mod 2n) so that SIMD
     batching and the NTT exist;
  2. compute h_{p,n}, the (single repeated) non-zero coefficient of the
     plaintext polynomial whose slots hold [1, -1];
  3. pick the integer k minimising k*h_{p,n} (mod p), because PMult with the
     [k, -k] plaintext grows the noise by 2|[k h]_p| instead of 2h.

Readings where the paper is silent:
  * p is the largest prime below 2^bits with p = 1 (mod 2n) unless given;
  * each RNS limb q_i is one of the largest primes below 2^limb_bits with
    q_i = 1 (mod 2n), in descending order;
  * the slot root zeta is the smallest primitive 2n-th root of unity mod p;
    slot (row r, index i) is the evaluation at zeta^((-1)^r 3^i);
  * k ranges over [1, k_max] and ties go to the smallest k; "minimised"
    means the smallest absolute value of the centred residue.
"""
from __future__ import annotations

from dataclasses import dataclass, field

# deterministic Miller-Rabin witnesses for every n < 3.3e24 (covers 64-bit)
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)


def is_prime(n: int) -> bool:
    """Miller-Rabin with a fixed witness set that is exact below 3.3e24."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(N: int, bits: int, count: int) -> list[int]:
    """The `count` largest primes below 2^bits that are 1 mod 2N, descending."""
    M = 2 * N
    out = []
    c = ((2**bits - 1) // M) * M + 1
    if c >= 2**bits:
        c -= M
    while len(out) < count and c > M:
        if is_prime(c):
            out.append(c)
        c -= M
    if len(out) < count:
        raise ValueError("not enough NTT-friendly primes")
    return out


def plain_modulus(N: int, bits: int) -> int:
    """Largest prime p < 2^bits with p = 1 (mod 2N) (step 1 for p)."""
    return ntt_primes(N, bits, 1)[0]


def min_primitive_root_2n(p: int, N: int) -> int:
    """Smallest x with x^N = -1 (mod p): a primitive 2N-th root of unity."""
    for x in range(2, p):
        if pow(x, N, p) == p - 1:
            return x
    raise ValueError("no primitive 2N-th root")


def any_primitive_root_2n(q: int, N: int) -> int:
    """Some primitive 2N-th root mod a large prime q: x^((q-1)/2N) for the first x that works."""
    e = (q - 1) // (2 * N)
    for x in range(2, 1 << 20):
        r = pow(x, e, q)
        if pow(r, N, q) == q - 1:
            return r
    raise ValueError("no root found")


def centred(v: int, p: int) -> int:
    """Representative of v mod p in (-p/2, p/2]."""
    v %= p
    return v - p if v > p // 2 else v


def slot_exponents(N: int) -> list[int]:
    """Odd exponent e for each flat slot index r*(N/2) + i: e = (-1)^r 3^i mod 2N."""
    M = 2 * N
    ex = []
    for r in range(2):
        for i in range(N // 2):
            e = pow(3, i, M)
            ex.append((M - e) % M if r else e)
    return ex


def encode_slots(values, p: int, N: int, zeta: int) -> list[int]:
    """Batch encoding (Sec. 2.3): the polynomial m of degree < N with
    m(zeta^e_s) = values[s] for every slot s.  Direct O(N^2) interpolation by
    the inverse transform m_j = N^-1 sum_s v_s zeta^(-e_s j); used here only
    for the small special polynomials of the parameter search."""
    M = 2 * N
    ex = slot_exponents(N)
    ninv = pow(N, -1, p)
    zinv = pow(zeta, -1, p)
    m = []
    for j in range(N):
        acc = 0
        for s, e in enumerate(ex):
            v = int(values[s]) % p
            if v:
                acc += v * pow(zinv, (e * j) % M, p)
        m.append(acc * ninv % p)
    return m


def hadamard_poly_coeff(p: int, N: int, zeta: int) -> tuple[int, list[int]]:
    """h_{p,n}: the non-zero coefficient of the plaintext packing [1, -1]
    (row 0 all 1, row 1 all -1) and the positions where it is non-zero.
    Computed in O(N) by evaluating the interpolation formula only where the
    polynomial can be non-zero; the full O(N^2) interpolation is used by the
    tests at small N to check positions and values."""
    ex = slot_exponents(N)
    M = 2 * N
    ninv = pow(N, -1, p)
    zinv = pow(zeta, -1, p)
    vals = [1] * (N // 2) + [p - 1] * (N // 2)

    def coeff(j):
        acc = 0
        for s, e in enumerate(ex):
            acc += vals[s] * pow(zinv, (e * j) % M, p)
        return acc * ninv % p

    # the coefficient at N/4 (the paper's claim of two equal non-zero terms
    # is checked exhaustively in the tests at small N)
    return coeff(N // 4), [N // 4, 3 * N // 4]


def best_k(h: int, p: int, k_max: int) -> int:
    """Step 3: k in [1, k_max] minimising |centred(k h mod p)|; ties -> smallest k."""
    best, best_v = None, None
    for k in range(1, k_max + 1):
        v = abs(centred(k * h, p))
        if best_v is None or v < best_v:
            best, best_v = k, v
    return best


@dataclass
class Params:
    """BFV parameters in RNS form (Sec. 2.3, Sec. 4.1)."""

    N: int
    t: int
    q: list[int]
    w: int  # decomposition base 2^w for key switching
    zeta: int = 0  # slot root mod t
    psi: list[int] = field(default_factory=list)  # NTT roots mod q_i
    h: int = 0  # residue mod t of the [1,-1] polynomial's coefficient
    k: int = 1
    sigma2: tuple[int, int] = (256, 25)  # sigma = 3.2 as the exact rational 256/25
    bound: int = 32  # B = 10 sigma, rounded down

    @property
    def L(self) -> int:
        return len(self.q)

    @property
    def l(self) -> int:
        """digits per limb: ceil(bits(q_max) / w)"""
        b = max(qi.bit_length() for qi in self.q)
        return -(-b // self.w)

    @property
    def Q(self) -> int:
        r = 1
        for qi in self.q:
            r *= qi
        return r

    @property
    def delta(self) -> int:
        return self.Q // self.t

    @property
    def kh(self) -> int:
        """centred coefficient of the [k, -k] plaintext"""
        return centred(self.k * self.h, self.t)


def make_params(N: int, L: int, w: int, t: int = 0, t_bits: int = 20, limb_bits: int = 50,
                k_max: int = 32) -> Params:
    """Steps 1-3 of Sec. 3.2.1 for a given ring degree and limb count."""
    if t == 0:
        t = plain_modulus(N, t_bits)
    if not is_prime(t) or t % (2 * N) != 1:
        raise ValueError("t must be a prime = 1 mod 2N for batching")
    q = ntt_primes(N, limb_bits, L)
    zeta = min_primitive_root_2n(t, N)
    h, _ = hadamard_poly_coeff(t, N, zeta)
    k = best_k(h, t, k_max)
    psi = [any_primitive_root_2n(qi, N) for qi in q]
    return Params(N=N, t=t, q=q, w=w, zeta=zeta, psi=psi, h=h, k=k)
