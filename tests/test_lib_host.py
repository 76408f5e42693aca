"""Host-side checks of the C-ABI library (no GPU): every declared symbol is
exported, and the client-side code (parameters, keys, encryption, layout,
decryption) agrees bit for bit with the independent oracle."""
import re
import subprocess

import numpy as np
import pytest

import synth
from oracle import bfv, conv
from oracle import params as prm
from paper_2311_12519_gb300 import hyena as H


def _declared():
    inc = H._build.os.path.join(H._build.os.path.dirname(H._build.HERE), "include")
    src = "".join(open(H._build.os.path.join(inc, f)).read() for f in sorted(H._build.os.listdir(inc))
                  if f.endswith(".h"))
    return sorted(set(re.findall(r"\b(he_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    H.load()
    out = subprocess.run(["nm", "-D", "--defined-only", H.library_path()], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if " T " in line)
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    lib = H.load()
    for s in _declared():
        assert hasattr(lib, s)


@pytest.mark.parametrize("N,L,w", [(1024, 2, 25), (4096, 2, 25), (8192, 3, 50), (16384, 4, 50)])
def test_params_match_oracle(N, L, w):
    p = H.he_params_create(N, L, decomp_bits=w)
    info = H.he_params_info(p)
    P = prm.make_params(N=N, L=L, w=w)
    assert info.t == P.t and info.zeta == P.zeta and info.h == P.h % P.t and info.k == P.k
    assert info.kh == P.kh and info.l == P.l
    assert info.k4 == conv.k4_select(P)
    assert [info.q[i] for i in range(L)] == P.q
    assert abs(info.log2_delta - np.log2(float(P.delta))) < 1e-6
    H.he_params_destroy(p)


def test_param_selection_reproduces_worked_example():
    # n = 2048 with Gazelle's p = 307201 -> h = 84248 (centred, up to sign), k = 11 (Sec. 3.2.1)
    p = H.he_params_create(2048, 1, t=307201, decomp_bits=25)
    info = H.he_params_info(p)
    assert min(info.h, 307201 - info.h) == 84248 and info.k == 11
    assert abs(info.kh) == 5125
    H.he_params_destroy(p)


def test_auto_decomposition_base():
    # L = 2 (q ~ 2^100) cannot afford w = 50 for 16-channel 3x3 layers; L = 3 can
    p = H.he_params_create(4096, 2, est_mac_terms=16 * 9)
    assert H.he_params_info(p).w == 25
    p3 = H.he_params_create(8192, 3, est_mac_terms=64 * 9)
    assert H.he_params_info(p3).w == 50


def test_errors():
    with pytest.raises(H.HyenaError) as e:
        H.he_params_create(1000, 2, decomp_bits=25)
    assert e.value.code == H.HE_EINVAL
    with pytest.raises(H.HyenaError) as e:
        H.he_params_create(4096, 2, t=1032191, decomp_bits=25)
    assert e.value.code == H.HE_EINVAL
    p = H.he_params_create(1024, 2, decomp_bits=25)
    with pytest.raises(H.HyenaError) as e:
        H.he_layout_for_layer(p, H.conv_desc(4, 4, 8, 8, kh=2))
    assert e.value.code == H.HE_EINVAL
    with pytest.raises(H.HyenaError) as e:
        H.he_layout_for_layer(p, H.conv_desc(4, 4, 8, 8, n_images=0))
    assert e.value.code == H.HE_EINVAL
    # a plan without its Galois keys is refused before any device work
    sk = H.he_keygen(p, 1)
    d = H.conv_desc(4, 4, 8, 8)
    gk = H.he_galois_keys(p, sk, H.he_layer_galois(p, d)[:-1], 1)
    with pytest.raises(H.HyenaError) as e:
        H.he_conv_plan(p, gk, d, np.ones((4, 4, 3, 3)))
    assert e.value.code == H.HE_EMISSINGKEY
    gk2 = H.he_galois_keys(p, sk, H.he_layer_galois(p, d), 1)
    with pytest.raises(H.HyenaError) as e:
        H.he_conv_plan(p, gk2, d, np.full((4, 4, 3, 3), 20000))
    assert e.value.code == H.HE_EINVAL


def test_keys_and_ciphertexts_match_oracle():
    N, L, w = 1024, 2, 25
    p = H.he_params_create(N, L, decomp_bits=w)
    info = H.he_params_info(p)
    P = prm.make_params(N=N, L=L, w=w)
    sk = H.he_keygen(p, 7)
    s = bfv.keygen(P, 7)
    assert (H.he_seckey_export(sk, N) == s).all()
    for g in (3, 2 * N - 1, bfv.rotation_element(P, -5)):
        gk = H.he_galois_keys(p, sk, [g], 11)
        assert (H.he_galkeys_export(gk, g, info) == bfv.galois_key(P, s, g, 11)).all()
    slots = synth.activations((N,), P.t)
    for idx in (0, 9):
        ct = H.he_encrypt_slots(p, sk, slots, 3, idx, info)
        assert (ct == bfv.encrypt(P, s, bfv.encode(P, slots), 3, idx)).all()
        assert (H.he_decrypt_slots(p, sk, ct, N) == slots).all()


LAYERS = [
    dict(C_in=3, C_out=5, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=2, c_n=2),
    dict(C_in=4, C_out=4, H=7, W=9, kh=3, stride=1, depthwise=False, n_images=3, c_n=1),
    dict(C_in=4, C_out=4, H=7, W=9, kh=3, stride=2, depthwise=True, n_images=3, c_n=2),
    dict(C_in=2, C_out=2, H=30, W=40, kh=3, stride=1, depthwise=False, n_images=1, c_n=2),
    dict(C_in=2, C_out=2, H=12, W=200, kh=3, stride=2, depthwise=False, n_images=1, c_n=2),
    dict(C_in=6, C_out=4, H=5, W=5, kh=1, stride=1, depthwise=False, n_images=2, c_n=2),
    dict(C_in=2, C_out=2, H=6, W=6, kh=5, stride=1, depthwise=False, n_images=1, c_n=2),
    # caller-chosen tiles: ragged last tiles, strips, stride-aligned squares, a tile spanning an odd side
    dict(C_in=3, C_out=4, H=10, W=9, kh=3, stride=1, depthwise=False, n_images=2, c_n=2, tile_h=4, tile_w=5),
    dict(C_in=2, C_out=2, H=30, W=40, kh=3, stride=1, depthwise=False, n_images=1, c_n=1, tile_h=7, tile_w=40),
    dict(C_in=4, C_out=4, H=12, W=13, kh=3, stride=2, depthwise=True, n_images=2, c_n=2, tile_h=6, tile_w=13),
    # c_n = 4: N/4 positions per row, channel classes row x slot parity
    dict(C_in=5, C_out=7, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=2, c_n=4),
    dict(C_in=8, C_out=8, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=3, c_n=4),
    dict(C_in=8, C_out=8, H=7, W=9, kh=3, stride=2, depthwise=True, n_images=3, c_n=4),
    dict(C_in=6, C_out=4, H=5, W=5, kh=1, stride=1, depthwise=False, n_images=2, c_n=4),
    dict(C_in=2, C_out=4, H=30, W=40, kh=3, stride=1, depthwise=False, n_images=1, c_n=4),
    dict(C_in=4, C_out=4, H=6, W=6, kh=5, stride=1, depthwise=False, n_images=1, c_n=4),
    dict(C_in=3, C_out=4, H=10, W=9, kh=3, stride=1, depthwise=False, n_images=2, c_n=4, tile_h=4, tile_w=5),
]


@pytest.mark.parametrize("spec", LAYERS)
def test_layout_and_image_encryption_match_oracle(spec):
    N, L, w = 1024, 2, 25
    p = H.he_params_create(N, L, decomp_bits=w)
    info = H.he_params_info(p)
    P = prm.make_params(N=N, L=L, w=w)
    d = H.conv_desc(**spec)
    lay = H.he_layout_for_layer(p, d)
    ol = conv.Layout(N=N, **spec)
    assert (lay.T_h, lay.T_w, lay.blocks_per_row, lay.n_ct_in, lay.n_ct_out, lay.Ho, lay.Wo) == \
        (ol.T_h, ol.T_w, ol.blocks_per_row, ol.n_ct_in, ol.n_ct_out, ol.Ho, ol.Wo)
    assert list(H.he_layer_galois(p, d)) == conv.galois_elements(P, ol)
    assert lay.scale == conv.output_scale(P, ol)
    act = synth.activations((spec["n_images"], spec["C_in"], spec["H"], spec["W"]), P.t)
    sk = H.he_keygen(p, 1)
    s = bfv.keygen(P, 1)
    ct = H.he_encrypt_image(p, sk, d, act, 2, info)
    assert (ct == conv.encrypt_image(P, ol, s, act, 2)).all()
    # decrypting the (unrotated) input through the output path reads the input back
    if spec["kh"] == 3 and spec["stride"] == 1 and spec["C_in"] == spec["C_out"] and not spec.get("tile_h"):
        back = H.he_decrypt_image(p, sk, d, ct, unscale=False)
        assert (back == act).all()


@pytest.mark.parametrize("tile,why", [((4, 0), "one side only"), ((11, 4), "taller than the image"),
                                      ((3, 4), "not a multiple of the stride"), ((10, 60), "block beyond N/2")])
def test_tile_override_rejected_like_the_oracle(tile, why):
    N = 1024
    p = H.he_params_create(N, 2, decomp_bits=25)
    spec = dict(C_in=2, C_out=2, H=10, W=60, kh=3, stride=2, depthwise=False, n_images=1, c_n=2,
                tile_h=tile[0], tile_w=tile[1])
    with pytest.raises(H.HyenaError) as e:
        H.he_layout_for_layer(p, H.conv_desc(**spec))
    assert e.value.code == H.HE_EINVAL, why
    with pytest.raises(ValueError):
        conv.Layout(N=N, **spec)
    H.he_params_destroy(p)


@pytest.mark.parametrize("desc,why", [
    (dict(C_in=2048, C_out=4, H=8, W=8), "more than 16384 accumulation terms"),
    (dict(C_in=4, C_out=6, H=8, W=8, depthwise=True), "depthwise with C_in != C_out"),
    (dict(C_in=4, C_out=4, H=8, W=8, stride=3), "stride 3"),
    (dict(C_in=4, C_out=4, H=8, W=8, c_n=3), "c_n = 3"),
    (dict(C_in=4, C_out=4, H=8, W=8, stride=2, c_n=4, polyphase=1), "polyphase with c_n = 4"),
    (dict(C_in=4, C_out=4, H=8, W=8, kh=9), "kernel 9"),
    (dict(C_in=0, C_out=4, H=8, W=8), "no input channels"),
    (dict(C_in=4, C_out=4, H=0, W=8), "empty image"),
])
def test_plan_checks_refuse_invalid_layers(desc, why):
    """The plan's host checks (he_conv_check: no device needed) refuse malformed layers."""
    p = H.he_params_create(1024, 2, decomp_bits=25)
    d = H.conv_desc(**desc)
    cw = 1 if desc.get("depthwise") else max(1, desc["C_in"])
    kh = desc.get("kh", 3)
    w = np.ones((max(1, desc["C_out"]), cw, kh, kh), dtype=np.int32)
    assert H.he_conv_check(p, d, w) == H.HE_EINVAL, why
    H.he_params_destroy(p)


def test_cn4_runs_on_the_cuda_core_mac_only():
    """c_n = 4 plans take the CUDA-core MAC (auto or mac_impl 1); every other form is refused, and
    mac_groups must be a power of two up to 16."""
    p = H.he_params_create(1024, 2, decomp_bits=25)
    d = H.conv_desc(C_in=8, C_out=8, H=6, W=6, kh=3, stride=1, n_images=1, c_n=4)
    w = np.ones((8, 8, 3, 3), dtype=np.int32)
    assert H.he_conv_check(p, d, w) == H.HE_OK
    assert H.he_conv_check(p, d, w, mac_impl=1) == H.HE_OK
    assert H.he_conv_check(p, d, w, mac_impl=1, mac_groups=8) == H.HE_OK
    for impl in (2, 3, 4, 5, 6, 7, 8):
        assert H.he_conv_check(p, d, w, mac_impl=impl) == H.HE_EINVAL, impl
    for mg in (3, 6, 32):
        assert H.he_conv_check(p, d, w, mac_groups=mg) == H.HE_EINVAL, mg
    H.he_params_destroy(p)


def test_plan_checks_accept_the_network_stacks_and_refuse_oversized_launches():
    """Every layer of the three stacks passes the launch-size check; a layer whose stages would
    not fit one launch each is refused (host only)."""
    import synth as sy

    for shapes, N, L, images in ((sy.resnet20_convs(), 8192, 3, 1), (sy.vgg16_convs(), 16384, 4, 8),
                                 (sy.mobilenet_v1_convs(), 8192, 4, 32)):
        p = H.he_params_create(N, L, decomp_bits=50)
        for s in shapes:
            d = H.conv_desc(s.C_in, s.C_out, s.H, s.W, s.k, s.stride, s.depthwise, images, 2)
            w = np.ones((s.C_out, 1 if s.depthwise else s.C_in, s.k, s.k), dtype=np.int32)
            assert H.he_conv_check(p, d, w) == H.HE_OK, (s, H.load().he_last_error())
        H.he_params_destroy(p)
    # 1024 images of 224x224 with 1024 channels in one 1x1 layer at N = 1024: the MAC grid alone
    # would need 114688 row units x 2 x 4 limbs x 8 slot tiles x 512 output groups > 2^31 blocks
    p = H.he_params_create(1024, 4, decomp_bits=50)
    d = H.conv_desc(1024, 1024, 224, 224, 1, 1, False, 1024, 2)
    assert H.he_conv_check(p, d, np.ones((1024, 1024, 1, 1), dtype=np.int32)) == H.HE_EINVAL
    assert "too large" in H.load().he_last_error().decode()
    H.he_params_destroy(p)


def test_noalloc_scratch_size_matches_the_header():
    """The binding's copy of the static scratch size is the header's #define."""
    inc = H._build.os.path.join(H._build.os.path.dirname(H._build.HERE), "include", "hyena.h")
    m = re.search(r"#define\s+HE_NOALLOC_MAX_SCRATCH_BYTES\s+(\d+)u?", open(inc).read())
    assert m and int(m.group(1)) == H.HE_NOALLOC_MAX_SCRATCH_BYTES


def test_cluster_and_form_choices_are_checked_without_a_device():
    """he_conv_check applies the tensor-core form and cluster rules on the host: clusters need a
    layer wider than one row tile, the fused form a layer that fits one, the CTA-pair form takes
    neither clusters nor a row tile."""
    p = H.he_params_create(1024, 2, decomp_bits=25)
    narrow = H.conv_desc(C_in=6, C_out=16, H=3, W=3, kh=3, stride=1, n_images=1, c_n=2)
    wide = H.conv_desc(C_in=6, C_out=512, H=3, W=3, kh=3, stride=1, n_images=1, c_n=2)
    wn, ww = synth.weights((16, 6, 3, 3)), synth.weights((512, 6, 3, 3))
    assert H.he_conv_check(p, narrow, wn, tc_cluster=2) == H.HE_EINVAL
    assert H.he_conv_check(p, wide, ww, tc_cluster=2) == H.HE_OK
    assert H.he_conv_check(p, wide, ww, tc_cluster=8) == H.HE_OK
    assert H.he_conv_check(p, wide, ww, tc_cluster=3) == H.HE_EINVAL
    assert H.he_conv_check(p, narrow, wn, mac_impl=6) == H.HE_OK
    assert H.he_conv_check(p, wide, ww, mac_impl=6) == H.HE_EINVAL
    assert H.he_conv_check(p, wide, ww, mac_impl=7) == H.HE_OK
    assert H.he_conv_check(p, narrow, wn, mac_impl=7) == H.HE_OK
    assert H.he_conv_check(p, wide, ww, mac_impl=7, tc_cluster=2) == H.HE_EINVAL
    assert H.he_conv_check(p, wide, ww, mac_impl=7, tc_rows=64) == H.HE_EINVAL
    assert H.he_conv_check(p, wide, ww, mac_impl=8) == H.HE_OK
    assert H.he_conv_check(p, wide, ww, mac_impl=8, tc_rows=64) == H.HE_EINVAL
    assert H.he_conv_check(p, wide, ww, mac_impl=9) == H.HE_EINVAL
    H.he_params_destroy(p)


POLY = [
    dict(C_in=3, C_out=5, H=7, W=9, kh=3, stride=2, depthwise=False, n_images=2, c_n=2, polyphase=1),
    dict(C_in=4, C_out=4, H=8, W=6, kh=3, stride=2, depthwise=True, n_images=3, c_n=2, polyphase=1),
    dict(C_in=3, C_out=3, H=9, W=7, kh=3, stride=2, depthwise=True, n_images=2, c_n=1, polyphase=1),
    dict(C_in=2, C_out=4, H=12, W=60, kh=3, stride=2, depthwise=False, n_images=1, c_n=2, polyphase=1,
         tile_h=3, tile_w=30),
]


@pytest.mark.parametrize("spec", POLY)
def test_polyphase_layout_and_encryption_match_the_oracle_derived_layer(spec):
    """Polyphase packing: the library's layout is the oracle's derived stride-1 layer on the phase
    planes, and its client encryption equals the oracle's encryption of the planes; its rotations
    are the derived layer's taps at offsets -1 and 0 only (a subset of the oracle's)."""
    N, L, w = 1024, 2, 25
    p = H.he_params_create(N, L, decomp_bits=w)
    info = H.he_params_info(p)
    P = prm.make_params(N=N, L=L, w=w)
    d = H.conv_desc(**spec)
    lay = H.he_layout_for_layer(p, d)
    ol = conv.Layout(N=N, **conv.polyphase_spec(spec))
    assert (lay.T_h, lay.T_w, lay.blocks_per_row, lay.n_ct_in, lay.n_ct_out, lay.Ho, lay.Wo) == \
        (ol.T_h, ol.T_w, ol.blocks_per_row, ol.n_ct_in, ol.n_ct_out, ol.Ho, ol.Wo)
    gal = set(int(g) for g in H.he_layer_galois(p, d))
    assert gal < set(conv.galois_elements(P, ol))
    packed_dense = spec["c_n"] == 2 and not spec["depthwise"]
    assert len(gal) == (7 if packed_dense else 3)
    act = synth.activations((spec["n_images"], spec["C_in"], spec["H"], spec["W"]), P.t, label=spec["W"])
    sk = H.he_keygen(p, 1)
    s = bfv.keygen(P, 1)
    ct = H.he_encrypt_image(p, sk, d, act, 2, info)
    assert (ct == conv.encrypt_image(P, ol, s, conv.polyphase_planes(act, spec["c_n"]), 2)).all()
    with pytest.raises(H.HyenaError):
        H.he_layout_for_layer(p, H.conv_desc(**dict(spec, stride=1)))
    H.he_params_destroy(p)


def test_fill_packing_agrees_between_library_and_oracle_layouts():
    """bench.py's per-layer packing rule (c_n = 1 where the tiles fill the slot rows) gives the
    same choice on the library's layouts as the stored-sample generator's copy on the oracle's."""
    import importlib.util
    import os

    import bench
    import synth
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("mns", os.path.join(here, "golden", "make_network_samples.py"))
    mns = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mns)
    for wl in ("vgg16", "mobilenet", "resnet20"):
        specs, N, L, _ = bench.layer_specs(wl)
        p = H.he_params_create(N, L, limb_bits=bench.LIMB_BITS, decomp_bits=50)
        lib = bench.fill_packing(specs, lambda x: (lambda o: (o.n_ct_in, o.n_ct_out))(
            H.he_layout_for_layer(p, H.conv_desc(**x))))
        ora = [1 if mns.fills_rows(N, s) else 2 for s in specs]
        assert [s["c_n"] for s in lib] == ora, wl
        H.he_params_destroy(p)


def test_stored_samples_cover_the_per_layer_packing():
    """Every layer the default packing runs unpacked has a stored oracle sample ('<stack>-cn1')
    whose output ciphertext count is the library's for that layout, and every packed layer has
    one in the stack's own entry: the bench can check each layer of its default line."""
    import json
    import os

    import bench
    golden = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                         "network_samples.json")))
    for wl in ("vgg16", "mobilenet"):
        specs, N, L, _ = bench.layer_specs(wl)
        p = H.he_params_create(N, L, limb_bits=bench.LIMB_BITS, decomp_bits=50)
        filled = bench.fill_packing(specs, lambda x: (lambda o: (o.n_ct_in, o.n_ct_out))(
            H.he_layout_for_layer(p, H.conv_desc(**x))))
        cn1 = {r["layer"]: r for r in golden[wl + "-cn1"]["samples"]}
        packed = {r["layer"]: r for r in golden[wl]["samples"]}
        for i, s in enumerate(filled):
            row = cn1[i] if s["c_n"] == 1 else packed[i]
            assert row["n_ct_out"] == H.he_layout_for_layer(p, H.conv_desc(**s)).n_ct_out, (wl, i)
        H.he_params_destroy(p)
