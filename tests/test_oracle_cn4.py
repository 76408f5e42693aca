"""Pins for the oracle's c_n = 4 packing (Sec. 3.1's 4 x 4 Walsh-Hadamard basis over the slot
classes row x parity): the sparsity of the three pattern plaintexts by direct interpolation,
decrypt(HE layer) = 4 k4 conv mod t over the layout variants, and planted mistakes those
checks must catch."""
import numpy as np
import pytest

import synth
from oracle import bfv, conv
from oracle import params as prm


def _direct_patterns(N: int, bits: int = 20):
    """The three patterns interpolated by the O(N^2) formula of the parameter search (no NTT)."""
    t = prm.plain_modulus(N, bits)
    zeta = prm.min_primitive_root_2n(t, N)
    half = N // 2
    out = []
    for b in (1, 2, 3):
        vals = [conv.H4[b][2 * r + (i & 1)] for r in range(2) for i in range(half)]
        m = prm.encode_slots(vals, t, N, zeta)
        out.append([prm.centred(x, t) for x in m])
    return t, out


@pytest.mark.parametrize("N", [16, 32, 64, 128])
def test_pattern_sparsity(N):
    """Slot parity: two opposite coefficients at N/4 and 3N/4; row sign: two equal ones there;
    their product: one at N/2.  Every other coefficient is zero."""
    t, (par, row, prod) = _direct_patterns(N)
    nz = lambda m: [j for j, v in enumerate(m) if v]
    assert nz(par) == [N // 4, 3 * N // 4] and par[N // 4] == -par[3 * N // 4]
    assert nz(row) == [N // 4, 3 * N // 4] and row[N // 4] == row[3 * N // 4]
    assert nz(prod) == [N // 2]


def test_patterns_match_direct_interpolation():
    """hadamard4_patterns (batch encoding through the NTT) equals the direct interpolation."""
    P = prm.make_params(N=128, L=1, w=25)
    t, direct = _direct_patterns(128)
    assert t == P.t
    for got, ref in zip(conv.hadamard4_patterns(P), direct):
        assert got.tolist() == ref


def test_hadamard_basis_orthogonal():
    H = np.array(conv.H4)
    assert (H @ H.T == 4 * np.eye(4, dtype=int)).all() and (H == H.T).all()


def test_k4_is_the_minimiser():
    """k4 minimises k + sum |[k a]_t| over the patterns' coefficients (brute force over all k
    in range, plain integers)."""
    P = prm.make_params(N=64, L=1, w=25, t_bits=14)
    coeffs = [int(a) for pat in conv.hadamard4_patterns(P) for a in pat if a]
    G = lambda k: k + sum(abs(prm.centred(k * a, P.t)) for a in coeffs)
    best = min(range(1, min(P.t - 1, conv.K4_MAX) + 1), key=lambda k: (G(k), k))
    assert conv.k4_select(P) == best


@pytest.fixture(scope="module")
def P256():
    return prm.make_params(N=256, L=2, w=25)


def _run(P, lay, seed=0, wmax=8):
    act = synth.activations((lay.n_images, lay.C_in, lay.H, lay.W), P.t, label=seed)
    wt = synth.weights((lay.C_out, 1 if lay.depthwise else lay.C_in, lay.kh, lay.kh), label=seed, wmax=wmax)
    s = bfv.keygen(P, synth.SEED_KEYS)
    ksk = {g: bfv.galois_key(P, s, g, synth.SEED_KEYS) for g in conv.galois_elements(P, lay)}
    cts = conv.encrypt_image(P, lay, s, act, synth.SEED_ENC)
    out = conv.he_conv(P, lay, wt, cts, ksk)
    got = conv.decrypt_image(P, lay, s, out)
    ref = conv.conv_plain(act, wt, lay.stride, lay.P, lay.depthwise, P.t)
    return got, ref, out, s


CASES = [
    # C_in, C_out, H, W, k, stride, depthwise, images
    (5, 7, 6, 6, 3, 1, False, 1),     # ragged channel counts, one block fills a row
    (4, 4, 4, 4, 3, 1, False, 2),     # two images, one per ciphertext column
    (8, 8, 5, 5, 3, 1, True, 1),      # depthwise: class-preserving steps only
    (4, 6, 7, 6, 3, 2, False, 1),     # stride 2, two tiles
    (2, 4, 9, 10, 3, 1, False, 1),    # full-width strips with a ragged tail
    (6, 5, 5, 6, 1, 1, False, 2),     # pointwise: steps -1, 0, 1
    (4, 4, 4, 4, 5, 1, False, 1),     # 5x5 kernel
    (5, 5, 6, 6, 3, 2, True, 1),      # depthwise, stride 2, ragged channels
]


@pytest.mark.parametrize("case", CASES)
def test_he_conv_cn4_decrypts_to_conv(P256, case):
    C_in, C_out, H, W, k, S, dw, I = case
    lay = conv.Layout(N=P256.N, C_in=C_in, C_out=C_out, H=H, W=W, kh=k, stride=S, depthwise=dw, n_images=I, c_n=4)
    got, ref, out, s = _run(P256, lay)
    assert got.shape == ref.shape
    assert (got == ref).all()
    assert max(bfv.noise_of(P256, s, c) for c in out) < P256.delta // 2


def test_layout_geometry_cn4(P256):
    """A row holds N/4 block positions; 3x3 steps are 2o for the 9 offsets and 2o +- 1 (12 odd
    steps over the three kernel rows), each with and without the row swap."""
    lay = conv.Layout(N=256, C_in=8, C_out=8, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=1, c_n=4)
    assert lay.row_positions == 64 and (lay.T_h, lay.T_w) == (6, 6) and lay.blocks_per_row == 1
    assert lay.in_groups == 2 and lay.n_ct_in == 2
    assert len(conv.rotation_steps4(lay)) == 21 and len(conv.rotation_plan(P256, lay)) == 42
    dw = conv.Layout(N=256, C_in=8, C_out=8, H=6, W=6, kh=3, stride=1, depthwise=True, n_images=1, c_n=4)
    assert conv.rotation_steps4(dw) == sorted(2 * (dy * 8 + dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    # channel 4j + c: row c >> 1, parity c & 1 at position pos
    assert [lay.flat_slot(0, 5, r) for r in range(4)] == [10, 11, 128 + 10, 128 + 11]


# ---------------------------------------------------------------- planted mistakes
LAY4 = dict(C_in=8, C_out=8, H=5, W=6, kh=3, stride=1, depthwise=False, n_images=1, c_n=4)


def _fails(P, monkeypatch, target, replacement, **kw):
    monkeypatch.setattr(target[0], target[1], replacement)
    got, ref, _, _ = _run(P, conv.Layout(N=256, **dict(LAY4, **kw)))
    return not (got == ref).all()


def test_mistake_parity_offset(P256, monkeypatch):
    """Every step read at offset floor(step / 2), whatever the destination parity (right for
    parity 0, one position off for parity 1 on odd steps)."""
    def wrong(l, w, g, j, step, d):
        taps = {dy * l.W_b + dx: (dy, dx) for dy, dx in l.taps()}
        v = [0, 0, 0, 0]
        for c in range(4):
            e_src = ((c & 1) + step) & 1
            tap = taps.get(step // 2)
            o, i = 4 * g + c, 4 * j + 2 * ((c >> 1) ^ d) + e_src
            if tap is None or o >= l.C_out or i >= l.C_in:
                continue
            v[c] = int(w[o, i, tap[0] + l.P, tap[1] + l.P])
        return [sum(conv.H4[b][c] * v[c] for c in range(4)) for b in range(4)]
    assert _fails(P256, monkeypatch, (conv, "hadamard4_scalars"), wrong)


def test_mistake_h4_sign(P256, monkeypatch):
    orig = conv.hadamard4_scalars
    assert _fails(P256, monkeypatch, (conv, "hadamard4_scalars"),
                  lambda *a: (lambda s: [s[0], s[1], -s[2], s[3]])(orig(*a)))


def test_mistake_swapped_row_diagonal(P256, monkeypatch):
    orig = conv.hadamard4_scalars
    assert _fails(P256, monkeypatch, (conv, "hadamard4_scalars"), lambda l, w, g, j, st, d: orig(l, w, g, j, st, 1 - d))


@pytest.mark.parametrize("b", [0, 1, 2])
def test_mistake_dropped_pattern(P256, monkeypatch, b):
    orig = conv.hadamard4_plaintexts
    def wrong(P):
        k4, pks = orig(P)
        pks = list(pks)
        pks[b] = np.zeros_like(pks[b])
        return k4, pks
    assert _fails(P256, monkeypatch, (conv, "hadamard4_plaintexts"), wrong)


def test_mistake_no_odd_steps(P256, monkeypatch):
    orig = conv.rotation_steps4
    assert _fails(P256, monkeypatch, (conv, "rotation_steps4"), lambda l: [s for s in orig(l) if s % 2 == 0])
