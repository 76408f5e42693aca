"""Pins for the oracle's parameter selection (Sec. 3.2.1).

The worked example of Sec. 3.2.1 (tests/golden/worked_example.json), the
closed form h^2 = -1/2 (mod p) derived from the slot structure, exhaustive
interpolation at small n, and sympy's independent primality test.
"""
import json
import os

import pytest
import sympy

from oracle import params as prm

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))


def test_worked_example_h_and_k():
    n, p = GOLD["n"], GOLD["p"]
    assert sympy.isprime(p) and p % (2 * n) == 1
    zeta = prm.min_primitive_root_2n(p, n)
    h, pos = prm.hadamard_poly_coeff(p, n, zeta)
    assert abs(prm.centred(h, p)) == GOLD["h_abs"]
    assert abs(prm.centred(h, p)).bit_length() == GOLD["h_bits"]
    assert prm.best_k(h, p, 32) == GOLD["k"]
    # Noise growth bits quoted next to the example: weights of 8 bits times
    # 2|[k h]_p| (Sec. 3.2.1: PMult grows noise by a factor (f0+f1+2(f0-f1)h)/2).
    wb = GOLD["weight_bits"]
    grow_k1 = (2 ** wb * 2 * abs(prm.centred(h, p))).bit_length() - 1
    grow_k = (2 ** wb * 2 * abs(prm.centred(GOLD["k"] * h, p))).bit_length() - 1
    assert grow_k1 == GOLD["pmult_growth_bits_k1"]
    assert grow_k == GOLD["pmult_growth_bits_k"]


@pytest.mark.parametrize("n,p", [(2048, 307201), (4096, 1032193), (8192, 1032193), (16384, 786433), (16, 97),
                                 (32, 193), (64, 257)])
def test_h_closed_form(n, p):
    # [1,-1] = c (X^{n/4} + X^{3n/4}) with c (w + w^3) = 1, w = zeta^{n/4} a primitive
    # 8th root of unity; (w + w^3)^2 = -2, hence h^2 = -1/2 (mod p), for any root choice.
    zeta = prm.min_primitive_root_2n(p, n)
    h, _ = prm.hadamard_poly_coeff(p, n, zeta)
    assert (h * h * 2 + 1) % p == 0


@pytest.mark.parametrize("n,p", [(16, 97), (32, 193), (64, 257), (64, 641)])
def test_hadamard_poly_is_two_equal_terms(n, p):
    """Full interpolation: exactly two non-zero coefficients, equal, at n/4 and 3n/4 (Sec. 3.2.1)."""
    zeta = prm.min_primitive_root_2n(p, n)
    m = prm.encode_slots([1] * (n // 2) + [p - 1] * (n // 2), p, n, zeta)
    nz = [i for i, c in enumerate(m) if c]
    assert nz == [n // 4, 3 * n // 4]
    assert m[n // 4] == m[3 * n // 4]
    h, _ = prm.hadamard_poly_coeff(p, n, zeta)
    assert h == m[n // 4]
    # scaling the slot pattern by k scales the coefficients by k (the [k,-k] plaintext)
    k = 5
    mk = prm.encode_slots([k] * (n // 2) + [p - k] * (n // 2), p, n, zeta)
    assert mk == [(k * c) % p for c in m]


@pytest.mark.parametrize("n,bits,count", [(4096, 50, 3), (8192, 50, 3), (16384, 50, 6), (2048, 20, 2)])
def test_ntt_primes(n, bits, count):
    qs = prm.ntt_primes(n, bits, count)
    assert qs == sorted(qs, reverse=True) and len(set(qs)) == count
    for q in qs:
        assert sympy.isprime(q) and q % (2 * n) == 1 and q < 2 ** bits
    # nothing was skipped: every c = 1 mod 2n in (qs[-1], 2^bits) that is not listed is composite
    c = qs[-1] + 2 * n
    while c < 2 ** bits:
        assert (c in qs) == sympy.isprime(c)
        c += 2 * n


def test_plain_modulus_readings():
    # largest prime below 2^20 that is 1 mod 2N (reading of t = 2^20)
    assert prm.plain_modulus(4096, 20) == 1032193
    assert prm.plain_modulus(8192, 20) == 1032193
    assert prm.plain_modulus(16384, 20) == 786433
    for n, t in [(4096, 1032193), (16384, 786433)]:
        assert all(not sympy.isprime(c) for c in range(t + 2 * n, 2 ** 20, 2 * n))


@pytest.mark.parametrize("p,n", [(97, 16), (1032193, 4096), (786433, 16384)])
def test_min_root(p, n):
    z = prm.min_primitive_root_2n(p, n)
    assert sympy.n_order(z, p) == 2 * n
    assert all(sympy.n_order(x, p) != 2 * n for x in range(2, z))


def test_best_k_is_argmin():
    p, h = 307201, 84248
    for kmax in (1, 5, 11, 40, 61, 100):
        k = prm.best_k(h, p, kmax)
        vals = [abs(prm.centred(j * h, p)) for j in range(1, kmax + 1)]
        assert abs(prm.centred(k * h, p)) == min(vals)
        assert k == 1 + vals.index(min(vals))


def test_make_params_fields():
    P = prm.make_params(N=4096, L=2, w=25)
    assert P.t == 1032193 and P.l == 2 and P.L == 2
    assert P.Q == P.q[0] * P.q[1] and P.delta == P.Q // P.t
    for qi, psi in zip(P.q, P.psi):
        assert pow(psi, P.N, qi) == qi - 1
