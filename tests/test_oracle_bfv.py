"""Pins for the oracle's BFV operations (Sec. 2.3) and the Hadamard identity (Eq. 1)."""
import numpy as np
import pytest

from oracle import bfv
from oracle import params as prm

HALF = None


@pytest.fixture(scope="module")
def P():
    return prm.make_params(N=256, L=2, w=25)


@pytest.fixture(scope="module")
def s(P):
    return bfv.keygen(P, 11)


def _m(P, seed):
    return np.random.default_rng(seed).integers(0, P.t, P.N)


def test_encrypt_decrypt(P, s):
    for i in range(3):
        u = _m(P, i)
        ct = bfv.encrypt(P, s, bfv.encode(P, u), 2, i)
        assert (bfv.decode(P, bfv.decrypt(P, s, ct)) == u).all()
        # fresh noise is the error e itself (plus nothing else): |v| <= B = 32
        assert bfv.noise(P, s, ct, bfv.encode(P, u)) <= P.bound
        # c1 = -a is uniform: different ciphertext indices give different masks
    c0 = bfv.encrypt(P, s, bfv.encode(P, _m(P, 0)), 2, 0)
    c1 = bfv.encrypt(P, s, bfv.encode(P, _m(P, 0)), 2, 1)
    assert not (c0[1] == c1[1]).all()


def test_hadd_cmult_pmult(P, s):
    u, v = _m(P, 1), _m(P, 2)
    cu = bfv.encrypt(P, s, bfv.encode(P, u), 2, 0)
    cv = bfv.encrypt(P, s, bfv.encode(P, v), 2, 1)
    dec = lambda c: bfv.decode(P, bfv.decrypt(P, s, c))
    assert (dec(bfv.hadd(P, cu, cv)) == (u + v) % P.t).all()
    assert (dec(bfv.cmult(P, cu, -7)) == (-7 * u) % P.t).all()
    w = np.random.default_rng(3).integers(0, 16, P.N)
    pt = [prm.centred(int(x), P.t) for x in bfv.encode(P, w)]
    assert (dec(bfv.pmult(P, cu, pt)) == (u * w) % P.t).all()


@pytest.mark.parametrize("step", [1, 4, -3, 17])
def test_hrot(P, s, step):
    u = _m(P, 5)
    half = P.N // 2
    ct = bfv.encrypt(P, s, bfv.encode(P, u), 2, 0)
    g = bfv.rotation_element(P, step)
    r = bfv.hrot(P, ct, bfv.galois_key(P, s, g, 9), g)
    ref = np.concatenate([np.roll(u[:half], -step), np.roll(u[half:], -step)])
    assert (bfv.decode(P, bfv.decrypt(P, s, r)) == ref).all()


def test_hoisted_rotations_share_one_decomposition(P, s):
    u = _m(P, 6)
    half = P.N // 2
    ct = bfv.encrypt(P, s, bfv.encode(P, u), 2, 0)
    digits = bfv.decompose(P, ct)
    # the digits recombine to c1: sum_j d_ij 2^(w j) = c1 mod q_i
    for i in range(P.L):
        rec = sum(digits[i * P.l + j].astype(object) * (1 << (P.w * j)) for j in range(P.l))
        assert (np.array(rec, dtype=object) == ct[1][i].astype(object)).all()
    for step, swap in [(2, False), (0, True), (-5, True)]:
        g = bfv.rotation_element(P, step)
        if swap:
            g = g * bfv.row_swap_element(P) % (2 * P.N)
        r = bfv.rotate_hoisted(P, ct, digits, bfv.galois_key(P, s, g, 9), g)
        a, b = np.roll(u[:half], -step), np.roll(u[half:], -step)
        ref = np.concatenate([b, a] if swap else [a, b])
        assert (bfv.decode(P, bfv.decrypt(P, s, r)) == ref).all()


def test_galois_key_structure(P, s):
    # b + a s = e + g_ij sigma(s) per limb: subtracting the gadget term leaves a small error
    g = bfv.rotation_element(P, 3)
    ksk = bfv.galois_key(P, s, g, 4)
    from oracle import _clib
    for i in range(P.L):
        for j in range(P.l):
            dd = i * P.l + j
            for k in range(P.L):
                q = P.q[k]
                sk = np.array([x % q for x in s.tolist()], dtype=np.uint64)
                asx = np.zeros(P.N, dtype=np.uint64)
                _clib.lib().orc_negacyclic_mul(ksk[dd, 1, k].copy(), sk, asx, P.N, q, P.psi[k])
                sg = np.zeros(P.N, dtype=np.uint64)
                _clib.lib().orc_automorphism(sk, sg, P.N, q, g)
                gij = pow(2, P.w * j, q) if k == i else 0
                e = [(int(b) + int(a) - gij * int(x)) % q for b, a, x in zip(ksk[dd, 0, k], asx, sg)]
                e = [prm.centred(v, q) for v in e]
                assert max(abs(v) for v in e) <= P.bound


def test_hadamard_identity_plain_and_encrypted(P, s):
    """Eq. 1: 2 PMult(m, [v0|v1]) = CMult(m, v0+v1) + PMult(CMult(m, v0-v1), [1|-1])."""
    half = P.N // 2
    u = _m(P, 8)
    for v0, v1 in [(3, -5), (8, 8), (-8, 7), (0, 1)]:
        target = np.concatenate([2 * v0 * u[:half], 2 * v1 * u[half:]]) % P.t
        w1 = [prm.centred(int(x), P.t) for x in bfv.encode(P, [1] * half + [-1] * half)]
        # plaintext level: polynomial arithmetic mod t
        ct = bfv.encrypt(P, s, bfv.encode(P, u), 2, 0)
        lhs = bfv.hadd(P, bfv.cmult(P, ct, v0 + v1), bfv.pmult(P, bfv.cmult(P, ct, v0 - v1), w1))
        assert (bfv.decode(P, bfv.decrypt(P, s, lhs)) == target).all()
        # the [k,-k] plaintext scales the result by k (Sec. 3.2.1 footnote)
        pk = bfv.hadamard_plaintext(P)
        lhs_k = bfv.hadd(P, bfv.cmult(P, ct, (v0 + v1) * P.k), bfv.pmult(P, bfv.cmult(P, ct, v0 - v1), pk))
        assert (bfv.decode(P, bfv.decrypt(P, s, lhs_k)) == (P.k * target) % P.t).all()


def test_hadamard_plaintext_is_sparse(P):
    pk = bfv.hadamard_plaintext(P)
    nz = np.nonzero(pk)[0].tolist()
    assert nz == [P.N // 4, 3 * P.N // 4]
    assert pk[P.N // 4] == pk[3 * P.N // 4] == P.kh
