"""Pins for the oracle's layer: the plain definition against torch's conv2d,
and decrypt(HE layer) = (2k) conv mod t for every layout variant, plus
planted mistakes that these checks must catch."""
import numpy as np
import pytest
import torch

import synth
from oracle import bfv, conv
from oracle import params as prm


def _torch_conv(act, w, stride, pad, depthwise, t):
    x = torch.tensor(act, dtype=torch.float64)
    k = torch.tensor(w, dtype=torch.float64)
    y = torch.nn.functional.conv2d(x, k, stride=stride, padding=pad, groups=act.shape[1] if depthwise else 1)
    return np.mod(np.round(y.numpy()).astype(np.int64), t)


@pytest.mark.parametrize("shape", [(2, 3, 7, 9, 5, 3, 1, False), (1, 4, 8, 8, 4, 3, 2, True), (1, 6, 5, 5, 2, 1, 1, False),
                                   (3, 5, 6, 4, 5, 3, 2, True)])
def test_conv_plain_matches_torch(shape):
    I, C, H, W, O, k, S, dw = shape
    t = 1032193
    act = synth.activations((I, C, H, W), t)
    wt = synth.weights((O, 1 if dw else C, k, k))
    # values small enough that float64 is exact
    small = act % 1000
    assert (conv.conv_plain(small, wt, S, (k - 1) // 2, dw, t) == _torch_conv(small, wt, S, (k - 1) // 2, dw, t)).all()


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
    # C_in, C_out, H, W, k, stride, depthwise, images, c_n
    (3, 5, 6, 6, 3, 1, False, 2, 2),      # odd channel counts, two images in one row
    (4, 4, 7, 9, 3, 1, False, 3, 1),      # padded convolution (no packing)
    (4, 4, 7, 9, 3, 1, True, 3, 2),       # depthwise, packed
    (3, 3, 7, 9, 3, 2, True, 1, 1),       # depthwise, stride 2, odd channels
    (4, 6, 9, 10, 3, 2, False, 1, 2),     # stride 2, several tiles
    (2, 2, 15, 13, 3, 1, False, 1, 2),    # image larger than a row: strips with a ragged tail
    (2, 4, 12, 40, 3, 1, False, 1, 2),    # one-row strips
    (2, 2, 12, 70, 3, 1, False, 1, 2),    # square tiles, ragged in both directions
    (6, 4, 5, 5, 1, 1, False, 2, 2),      # pointwise 1x1: row swap only
    (5, 3, 6, 6, 1, 1, False, 1, 1),      # pointwise, no packing
    (2, 2, 6, 6, 5, 1, False, 1, 2),      # 5x5 kernel
]


@pytest.mark.parametrize("case", CASES)
def test_he_conv_decrypts_to_conv(P256, case):
    C_in, C_out, H, W, k, S, dw, I, cn = case
    lay = conv.Layout(N=P256.N, C_in=C_in, C_out=C_out, H=H, W=W, kh=k, stride=S, depthwise=dw, n_images=I, c_n=cn)
    got, ref, out, s = _run(P256, lay)
    assert got.shape == ref.shape
    assert (got == ref).all()
    assert max(bfv.noise_of(P256, s, c) for c in out) < P256.delta // 2


def test_layout_geometry(P256):
    lay = conv.Layout(N=256, C_in=2, C_out=2, H=15, W=13, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    # strips of full width: (T_h + 2)(13 + 2) <= 128
    assert (lay.T_h, lay.T_w) == (6, 13) and lay.n_ty == 3 and lay.blocks_per_row == 1
    lay = conv.Layout(N=256, C_in=2, C_out=2, H=12, W=70, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    assert (lay.T_h, lay.T_w) == (9, 9) and lay.n_tx == 8 and lay.n_ty == 2
    lay = conv.Layout(N=4096, C_in=16, C_out=16, H=16, W=16, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    assert (lay.T_h, lay.T_w, lay.blocks_per_row, lay.n_ct_in) == (16, 16, 6, 8)
    # a 3x3 layer with packing needs 2*9 - 1 = 17 distinct non-trivial Galois elements
    P = prm.make_params(N=4096, L=2, w=25)
    assert len(conv.galois_elements(P, lay)) == 17


@pytest.mark.slow
def test_single_layer_16_full_size():
    """16 channels, 16x16, 3x3 -> 16 at N = 4096, L = 2 (about 10 s)."""
    P = prm.make_params(N=4096, L=2, w=25)
    lay = conv.Layout(N=4096, C_in=16, C_out=16, H=16, W=16, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    got, ref, out, s = _run(P, lay)
    assert (got == ref).all()
    assert max(bfv.noise_of(P, s, c) for c in out[:2]) < P.delta // 2


# ---------------------------------------------------------------- planted mistakes
def _fails(P, lay, monkeypatch, target, replacement):
    monkeypatch.setattr(target[0], target[1], replacement)
    got, ref, _, _ = _run(P, lay)
    return not (got == ref).all()


LAY = dict(C_in=4, C_out=4, H=5, W=6, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)


def test_mistake_swapped_diagonal(P256, monkeypatch):
    orig = conv.hadamard_scalars
    lay = conv.Layout(N=256, **LAY)
    assert _fails(P256, lay, monkeypatch, (conv, "hadamard_scalars"), lambda l, w, g, j, ti, d: orig(l, w, g, j, ti, 1 - d))


def test_mistake_hadamard_sign(P256, monkeypatch):
    orig = conv.hadamard_scalars
    lay = conv.Layout(N=256, **LAY)
    assert _fails(P256, lay, monkeypatch, (conv, "hadamard_scalars"),
                  lambda *a: (lambda s: (s[0], -s[1]))(orig(*a)))


def test_mistake_transposed_weights(P256, monkeypatch):
    orig = conv.hadamard_scalars
    lay = conv.Layout(N=256, **LAY)
    assert _fails(P256, lay, monkeypatch, (conv, "hadamard_scalars"),
                  lambda l, w, g, j, ti, d: orig(l, np.ascontiguousarray(w.transpose(1, 0, 2, 3)), g, j, ti, d))


def test_mistake_tap_flip(P256, monkeypatch):
    orig = conv.hadamard_scalars
    lay = conv.Layout(N=256, **LAY)
    assert _fails(P256, lay, monkeypatch, (conv, "hadamard_scalars"),
                  lambda l, w, g, j, ti, d: orig(l, w, g, j, l.kh * l.kh - 1 - ti, d))


def test_mistake_dropped_pmult_term(P256, monkeypatch):
    lay = conv.Layout(N=256, **LAY)
    assert _fails(P256, lay, monkeypatch, (bfv, "pmult"), lambda P, ct, pt: np.zeros_like(ct))


def test_mistake_wrong_rotation_sign(P256, monkeypatch):
    orig = bfv.rotation_element
    lay = conv.Layout(N=256, **LAY)
    assert _fails(P256, lay, monkeypatch, (bfv, "rotation_element"), lambda P, step: orig(P, -step))


@pytest.mark.parametrize("case,tile", [
    ((3, 4, 10, 9, 3, 1, False, 2, 2), (4, 5)),    # ragged tiles in both directions, two images
    ((4, 6, 12, 13, 3, 2, False, 2, 1), (6, 13)),  # stride-2 strips spanning an odd width, unpacked
    ((4, 4, 12, 12, 3, 2, True, 1, 2), (4, 6)),    # depthwise, stride 2, stride-aligned tiles
])
def test_he_conv_with_chosen_tiles_decrypts_to_conv(P256, case, tile):
    """Caller-chosen tiles (any size that fits a row, origins on the stride grid) give the same
    convolution as the default tiles, by the decryption invariant."""
    C_in, C_out, H, W, k, S, dw, I, cn = case
    lay = conv.Layout(N=P256.N, C_in=C_in, C_out=C_out, H=H, W=W, kh=k, stride=S, depthwise=dw, n_images=I, c_n=cn,
                      tile_h=tile[0], tile_w=tile[1])
    assert (lay.T_h, lay.T_w) == tile
    got, ref, out, s = _run(P256, lay)
    assert (got == ref).all()
    assert max(bfv.noise_of(P256, s, c) for c in out) < P256.delta // 2


# ---------------------------------------------------------------- polyphase stride 2
@pytest.mark.parametrize("shape", [(2, 3, 7, 9, 5, False, 2), (1, 4, 8, 8, 4, True, 2), (1, 3, 5, 5, 3, True, 1),
                                   (2, 2, 6, 7, 6, False, 1)])
def test_polyphase_planes_and_weights_give_the_stride2_conv(shape):
    """The derived stride-1 layer on the phase planes computes the stride-2 convolution (plaintext,
    brute-force definition of both)."""
    I, C, H, W, O, dw, c_n = shape
    t = 1032193
    act = synth.activations((I, C, H, W), t, label=H)
    wt = synth.weights((O, 1 if dw else C, 3, 3), label=W)
    planes = conv.polyphase_planes(act, c_n)
    w2 = conv.polyphase_weights(wt, C, c_n, dw)
    assert planes.shape == (I, 4 * (-(-C // c_n) * c_n), -(-H // 2), -(-W // 2))
    assert (w2[:, :, 2, :] == 0).all() and (w2[:, :, :, 2] == 0).all()  # no tap at offset +1
    assert (conv.conv_plain(planes, w2, 1, 1, False, t) == conv.conv_plain(act, wt, 2, 1, dw, t)).all()


@pytest.mark.parametrize("spec", [
    dict(C_in=3, C_out=5, H=7, W=9, kh=3, stride=2, depthwise=False, n_images=2, c_n=2),
    dict(C_in=4, C_out=4, H=8, W=6, kh=3, stride=2, depthwise=True, n_images=2, c_n=2),
    dict(C_in=3, C_out=3, H=5, W=7, kh=3, stride=2, depthwise=True, n_images=1, c_n=1),
])
def test_polyphase_he_conv_decrypts_to_stride2_conv(P256, spec):
    """Encrypted: the Hyena layer of the derived stride-1 layer, on the encrypted phase planes,
    decrypts to (2k) x the stride-2 convolution at every output position."""
    P = P256
    act = synth.activations((spec["n_images"], spec["C_in"], spec["H"], spec["W"]), P.t, label=spec["H"])
    wt = synth.weights((spec["C_out"], 1 if spec["depthwise"] else spec["C_in"], 3, 3), label=spec["W"])
    lay = conv.Layout(N=P.N, **conv.polyphase_spec(spec))
    planes = conv.polyphase_planes(act, spec["c_n"])
    w2 = conv.polyphase_weights(wt, spec["C_in"], spec["c_n"], spec["depthwise"])
    s = bfv.keygen(P, synth.SEED_KEYS)
    ksk = {g: bfv.galois_key(P, s, g, synth.SEED_KEYS) for g in conv.galois_elements(P, lay)}
    cts = conv.encrypt_image(P, lay, s, planes, synth.SEED_ENC)
    out = conv.he_conv(P, lay, w2, cts, ksk)
    dec = conv.decrypt_image(P, lay, s, out)
    assert (dec == conv.conv_plain(act, wt, 2, 1, spec["depthwise"], P.t)).all()
