"""Pins for the oracle's ring arithmetic and samplers.

Independent references: direct evaluation of the NTT's definition, the
schoolbook negacyclic product, the ring-homomorphism property of the
automorphism, published SplitMix64 outputs and sampler moments.
"""
import numpy as np
import pytest

from oracle import _clib, bfv
from oracle import params as prm


def _schoolbook(a, b, q):
    N = len(a)
    c = [0] * N
    for i in range(N):
        for j in range(N):
            if i + j < N:
                c[i + j] += a[i] * b[j]
            else:
                c[i + j - N] -= a[i] * b[j]
    return [x % q for x in c]


def _rand(rng, N, q):
    return np.array([int(x) % q for x in rng.integers(0, 2**62, N)], dtype=np.uint64)


@pytest.mark.parametrize("N,bits", [(8, 30), (16, 50), (64, 50), (64, 61)])
def test_ntt_matches_definition(N, bits):
    q = prm.ntt_primes(N, bits, 1)[0]
    psi = prm.any_primitive_root_2n(q, N)
    rng = np.random.default_rng(N)
    a = _rand(rng, N, q)
    A = a.copy()
    _clib.lib().orc_ntt_fwd(A, N, q, psi)
    for k in range(N):
        e = 2 * k + 1
        ref = sum(int(a[i]) * pow(psi, e * i, q) for i in range(N)) % q
        assert int(A[k]) == ref
    _clib.lib().orc_ntt_inv(A, N, q, psi)
    assert (A == a).all()


@pytest.mark.parametrize("N,bits", [(8, 30), (16, 50), (64, 50), (64, 60)])
def test_negacyclic_product_vs_schoolbook(N, bits):
    q = prm.ntt_primes(N, bits, 1)[0]
    psi = prm.any_primitive_root_2n(q, N)
    rng = np.random.default_rng(7 + N)
    a, b = _rand(rng, N, q), _rand(rng, N, q)
    c = np.zeros(N, dtype=np.uint64)
    _clib.lib().orc_negacyclic_mul(a, b, c, N, q, psi)
    assert [int(x) for x in c] == _schoolbook([int(x) for x in a], [int(x) for x in b], q)


def test_ntt_round_trip_large():
    N = 16384
    q = prm.ntt_primes(N, 50, 1)[0]
    psi = prm.any_primitive_root_2n(q, N)
    a = _rand(np.random.default_rng(3), N, q)
    A = a.copy()
    _clib.lib().orc_ntt_fwd(A, N, q, psi)
    _clib.lib().orc_ntt_inv(A, N, q, psi)
    assert (A == a).all()


@pytest.mark.parametrize("g", [3, 9, 31, 127, 27])
def test_automorphism_is_evaluation_substitution(g):
    # sigma_g(a)(x) = a(x^g) at every root x of X^N + 1
    N = 64
    q = prm.ntt_primes(N, 40, 1)[0]
    psi = prm.any_primitive_root_2n(q, N)
    a = _rand(np.random.default_rng(g), N, q)
    out = np.zeros(N, dtype=np.uint64)
    _clib.lib().orc_automorphism(a, out, N, q, g % (2 * N))
    for e in (1, 3, 5, 77):
        x = pow(psi, e, q)
        lhs = sum(int(out[i]) * pow(x, i, q) for i in range(N)) % q
        rhs = sum(int(a[i]) * pow(x, g * i, q) for i in range(N)) % q
        assert lhs == rhs


def test_automorphism_composes():
    N = 32
    q = prm.ntt_primes(N, 40, 1)[0]
    a = _rand(np.random.default_rng(1), N, q)
    t1, t2, t3 = (np.zeros(N, dtype=np.uint64) for _ in range(3))
    L = _clib.lib()
    L.orc_automorphism(a, t1, N, q, 3)
    L.orc_automorphism(t1, t2, N, q, 5)
    L.orc_automorphism(a, t3, N, q, 15)
    assert (t2 == t3).all()


def _small_params(N=64):
    return prm.make_params(N=N, L=2, w=25)


def test_encode_decode_and_slot_product():
    P = _small_params()
    rng = np.random.default_rng(5)
    u = rng.integers(0, P.t, P.N)
    v = rng.integers(0, P.t, P.N)
    assert (bfv.decode(P, bfv.encode(P, u)) == u).all()
    # multiplication of polynomials mod t is slot-wise multiplication
    mu, mv = bfv.encode(P, u), bfv.encode(P, v)
    prod = _schoolbook([int(x) for x in mu], [int(x) for x in mv], P.t)
    assert (bfv.decode(P, prod) == (u * v) % P.t).all()
    # the oracle's fast encode agrees with direct interpolation
    assert [int(x) for x in mu] == prm.encode_slots(list(u), P.t, P.N, P.zeta)


@pytest.mark.parametrize("step", [1, 2, 5, -1, -9, 31])
def test_rotation_and_row_swap_on_slots(step):
    P = _small_params()
    half = P.N // 2
    u = np.random.default_rng(step % 97).integers(0, P.t, P.N)
    m = bfv.encode(P, u)
    out = np.zeros(P.N, dtype=np.uint64)
    _clib.lib().orc_automorphism(m, out, P.N, P.t, bfv.rotation_element(P, step))
    ref = np.concatenate([np.roll(u[:half], -step), np.roll(u[half:], -step)])
    assert (bfv.decode(P, out) == ref).all()
    _clib.lib().orc_automorphism(m, out, P.N, P.t, bfv.row_swap_element(P))
    assert (bfv.decode(P, out) == np.concatenate([u[half:], u[:half]])).all()


def test_splitmix_published_outputs():
    # SplitMix64 from state 0: first three outputs of the published generator
    L = _clib.lib()
    assert L.orc_splitmix_at(0, 0) == 0xE220A8397B1DCDAF
    assert L.orc_splitmix_at(0, 1) == 0x6E789E6AA1B965F4
    assert L.orc_splitmix_at(0, 2) == 0x06C45D188009454F


def test_samplers():
    P = prm.make_params(N=16384, L=2, w=25)
    s = bfv.sample_ternary(P, 123)
    assert set(np.unique(s)) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs((s == v).mean() - 1 / 3) < 0.02
    e = np.concatenate([bfv.sample_gauss(P, k) for k in range(4)]).astype(float)
    assert abs(e.mean()) < 0.1
    assert abs(e.var() - 10.24) < 0.4  # sigma = 3.2
    assert np.abs(e).max() <= 32
    # discrete Gaussian shape: P(0)/P(1) = exp(1/(2 sigma^2))
    r = (e == 0).mean() / ((e == 1).mean())
    assert abs(np.log(r) - 1 / (2 * 10.24)) < 0.03
    a = bfv.sample_uniform(P, 99)
    for k in range(P.L):
        x = a[k].astype(float) / P.q[k]
        assert (a[k] < P.q[k]).all() and abs(x.mean() - 0.5) < 0.01
