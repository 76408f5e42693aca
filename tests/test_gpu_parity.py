"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Ciphertexts are compared word for word (exact modular arithmetic, so the bar
is bit-exactness), and outputs are decrypted against the plain convolution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import bfv, conv  # noqa: E402
from oracle import params as prm  # noqa: E402
from paper_2311_12519_gb300 import hyena as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).view(np.int64)).cuda()


def from_dev(t, shape):
    return t.cpu().numpy().view(np.uint64).reshape(shape)


def gpu_layer(p, gk, d, w, cts, L, N, stream=None, mac_groups=0, mac_impl=0, tc_rows=0, tc_cluster=0):
    plan = H.he_conv_plan(p, gk, d, w, mac_groups=mac_groups, mac_impl=mac_impl, tc_rows=tc_rows,
                          tc_cluster=tc_cluster)
    n_in, n_out, ws = H.he_conv_sizes(plan)
    assert n_in == cts.size
    d_in = to_dev(cts)
    d_out = torch.full((n_out,), -1, dtype=torch.int64, device="cuda")
    d_ws = torch.empty(ws // 8 + 1, dtype=torch.int64, device="cuda")
    s = stream or torch.cuda.current_stream()
    H.he_conv_forward(plan, d_in.data_ptr(), d_out.data_ptr(), d_ws.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    assert (from_dev(d_in, cts.shape) == cts).all(), "input modified"
    out = from_dev(d_out, (n_out // (2 * L * N), 2, L, N))
    H.he_conv_status(plan)
    H.he_plan_destroy(plan)
    return out


class Setup:
    def __init__(self, N, L, w, limb_bits=50):
        self.N, self.L, self.w = N, L, w
        self.p = H.he_params_create(N, L, limb_bits=limb_bits, decomp_bits=w)
        self.info = H.he_params_info(self.p)
        self.P = prm.make_params(N=N, L=L, w=w, limb_bits=limb_bits)
        self.sk = H.he_keygen(self.p, synth.SEED_KEYS)
        self.s = bfv.keygen(self.P, synth.SEED_KEYS)
        self._ksk = {}

    def oracle_keys(self, gs):
        for g in gs:
            if g not in self._ksk:
                self._ksk[g] = bfv.galois_key(self.P, self.s, g, synth.SEED_KEYS)
        return self._ksk

    def layer(self, spec, label=0, sample=None, mac_groups=0, mac_impl=0, wmax=8, tc_rows=0, tc_cluster=0):
        N, L = self.N, self.L
        d = H.conv_desc(**spec)
        ol = conv.Layout(N=N, **spec)
        act = synth.activations((spec["n_images"], spec["C_in"], spec["H"], spec["W"]), self.P.t, label=label)
        wt = synth.weights((spec["C_out"], 1 if spec["depthwise"] else spec["C_in"], spec["kh"], spec["kh"]),
                           label=label, wmax=wmax)
        gs = H.he_layer_galois(self.p, d)
        gk = H.he_galois_keys(self.p, self.sk, gs, synth.SEED_KEYS)
        cts = H.he_encrypt_image(self.p, self.sk, d, act, synth.SEED_ENC, self.info)
        ref_in = conv.encrypt_image(self.P, ol, self.s, act, synth.SEED_ENC)
        assert (cts == ref_in).all()
        out = gpu_layer(self.p, gk, d, wt, cts, L, N, mac_groups=mac_groups, mac_impl=mac_impl, tc_rows=tc_rows,
                        tc_cluster=tc_cluster)
        ref = conv.he_conv(self.P, ol, wt, ref_in, self.oracle_keys(gs), out_cts=sample)
        idx = range(len(out)) if sample is None else sample
        for c in idx:
            assert (out[c] == ref[c]).all(), f"ciphertext {c} differs from the oracle"
        dec = H.he_decrypt_image(self.p, self.sk, d, out)
        plain = conv.conv_plain(act, wt, spec["stride"], (spec["kh"] - 1) // 2, spec["depthwise"], self.P.t)
        assert (dec == plain).all(), "decryption differs from the plain convolution"
        H.he_galkeys_destroy(gk)
        return out


@pytest.fixture(scope="module")
def small():
    return Setup(1024, 2, 25)


# ---------------------------------------------------------------- NTT
@pytest.mark.parametrize("N,L,w", [(1024, 2, 25), (4096, 2, 25), (8192, 3, 50), (16384, 6, 50)])
def test_ntt_round_trip_and_negacyclic_product(N, L, w):
    p = H.he_params_create(N, L, decomp_bits=w)
    P = prm.make_params(N=N, L=L, w=w)
    rng = np.random.default_rng(N + L)
    a = np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in P.q])
    b = np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in P.q])
    da, db = to_dev(a), to_dev(b)
    H.he_ntt_forward(p, da.data_ptr(), L)
    H.he_ntt_forward(p, db.data_ptr(), L)
    torch.cuda.synchronize()
    A, B = from_dev(da, (L, N)), from_dev(db, (L, N))
    # pointwise product in the NTT domain, then back: the negacyclic product
    C = np.stack([(A[k].astype(object) * B[k].astype(object) % P.q[k]).astype(np.uint64) for k in range(L)])
    dc = to_dev(C)
    H.he_ntt_inverse(p, dc.data_ptr(), L)
    H.he_ntt_inverse(p, da.data_ptr(), L)
    torch.cuda.synchronize()
    assert (from_dev(da, (L, N)) == a).all()
    from oracle import _clib
    for k in range(min(L, 2)):
        ref = np.zeros(N, dtype=np.uint64)
        _clib.lib().orc_negacyclic_mul(a[k].copy(), b[k].copy(), ref, N, P.q[k], P.psi[k])
        assert (from_dev(dc, (L, N))[k] == ref).all()
    H.he_params_destroy(p)


# ---------------------------------------------------------------- rotation
@pytest.mark.parametrize("N,L,w,step,swap", [(1024, 2, 25, 1, False), (1024, 2, 25, -7, True), (4096, 2, 25, 35, False),
                                             (8192, 3, 50, -1, True)])
def test_rotation_matches_oracle(N, L, w, step, swap):
    S = Setup(N, L, w)
    g = bfv.rotation_element(S.P, step)
    if swap:
        g = g * bfv.row_swap_element(S.P) % (2 * N)
    gk = H.he_galois_keys(S.p, S.sk, [g], synth.SEED_KEYS)
    n_ct = 3
    slots = [synth.activations((N,), S.P.t, label=i) for i in range(n_ct)]
    cts = np.stack([H.he_encrypt_slots(S.p, S.sk, slots[i], synth.SEED_ENC, i, S.info) for i in range(n_ct)])
    d_in, d_out = to_dev(cts), torch.empty(cts.size, dtype=torch.int64, device="cuda")
    d_ws = torch.empty(H.he_rotate_workspace_bytes(S.p, n_ct) // 8 + 1, dtype=torch.int64, device="cuda")
    H.he_rotate(S.p, gk, g, d_in.data_ptr(), d_out.data_ptr(), n_ct, d_ws.data_ptr())
    out = from_dev(d_out, cts.shape)
    ksk = S.oracle_keys([g])[g]
    half = N // 2
    for i in range(n_ct):
        assert (out[i] == bfv.hrot(S.P, cts[i], ksk, g)).all()
        a, b = np.roll(slots[i][:half], -step), np.roll(slots[i][half:], -step)
        assert (H.he_decrypt_slots(S.p, S.sk, out[i], N) == np.concatenate([b, a] if swap else [a, b])).all()


# ---------------------------------------------------------------- layers, small ring
SMALL = [
    dict(C_in=3, C_out=5, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=2, c_n=2),
    dict(C_in=4, C_out=4, H=7, W=9, kh=3, stride=1, depthwise=False, n_images=3, c_n=1),
    dict(C_in=4, C_out=4, H=7, W=9, kh=3, stride=1, depthwise=True, n_images=3, c_n=2),
    dict(C_in=3, C_out=3, H=7, W=9, kh=3, stride=2, depthwise=True, n_images=2, c_n=1),
    dict(C_in=4, C_out=6, H=9, W=10, kh=3, stride=2, depthwise=False, n_images=1, c_n=2),
    dict(C_in=2, C_out=2, H=30, W=40, kh=3, stride=1, depthwise=False, n_images=1, c_n=2),
    dict(C_in=2, C_out=3, H=12, W=200, kh=3, stride=1, depthwise=False, n_images=1, c_n=2),
    dict(C_in=6, C_out=4, H=5, W=5, kh=1, stride=1, depthwise=False, n_images=2, c_n=2),
    dict(C_in=5, C_out=3, H=6, W=6, kh=1, stride=1, depthwise=False, n_images=1, c_n=1),
    dict(C_in=2, C_out=2, H=6, W=6, kh=5, stride=1, depthwise=False, n_images=1, c_n=2),
    dict(C_in=1, C_out=1, H=1, W=1, kh=3, stride=1, depthwise=False, n_images=1, c_n=2),
    dict(C_in=20, C_out=18, H=5, W=5, kh=3, stride=1, depthwise=False, n_images=5, c_n=2),
    # caller-chosen tiles (ragged last tiles; stride-2 strips)
    dict(C_in=3, C_out=4, H=10, W=9, kh=3, stride=1, depthwise=False, n_images=2, c_n=2, tile_h=4, tile_w=5),
    dict(C_in=4, C_out=6, H=12, W=13, kh=3, stride=2, depthwise=False, n_images=2, c_n=1, tile_h=6, tile_w=13),
]


@pytest.mark.parametrize("spec", SMALL)
def test_layer_small_ring(small, spec):
    small.layer(spec)


@pytest.mark.parametrize("groups", [1, 2, 4, 8])
def test_mac_group_tiling_is_invisible(small, groups):
    spec = dict(C_in=6, C_out=22, H=5, W=5, kh=3, stride=1, depthwise=False, n_images=2, c_n=2)
    small.layer(spec, mac_groups=groups)


# ---------------------------------------------------------------- c_n = 4 (4 x 4 Walsh-Hadamard basis)
CN4 = [
    dict(C_in=5, C_out=7, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=2, c_n=4),    # ragged channels
    dict(C_in=8, C_out=8, H=7, W=9, kh=3, stride=1, depthwise=True, n_images=3, c_n=4),     # depthwise
    dict(C_in=8, C_out=12, H=9, W=10, kh=3, stride=2, depthwise=False, n_images=1, c_n=4),  # stride 2
    dict(C_in=2, C_out=4, H=30, W=40, kh=3, stride=1, depthwise=False, n_images=1, c_n=4),  # strips, ragged tail
    dict(C_in=6, C_out=4, H=5, W=5, kh=1, stride=1, depthwise=False, n_images=2, c_n=4),    # pointwise
    dict(C_in=4, C_out=4, H=6, W=6, kh=5, stride=1, depthwise=False, n_images=1, c_n=4),    # 5x5
    dict(C_in=20, C_out=18, H=5, W=5, kh=3, stride=1, depthwise=False, n_images=5, c_n=4),  # groups x images
    dict(C_in=3, C_out=4, H=10, W=9, kh=3, stride=1, depthwise=False, n_images=2, c_n=4, tile_h=4, tile_w=5),
]


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("spec", CN4)
def test_cn4_layer_matches_oracle(small, spec, impl):
    """c_n = 4 layers (the CUDA-core MAC with four rows per output group and the three pattern
    PMults in its epilogue) word for word against the oracle, and decrypted against the convolution."""
    small.layer(spec, mac_impl=impl)


@pytest.mark.parametrize("groups", [1, 2, 4, 8])
def test_cn4_mac_group_tiling_is_invisible(small, groups):
    small.layer(dict(C_in=6, C_out=22, H=5, W=5, kh=3, stride=1, depthwise=False, n_images=2, c_n=4),
                mac_groups=groups)


# ---------------------------------------------------------------- the 16-channel layer, N = 4096
def test_single_layer_16_channels():
    S = Setup(4096, 2, 25)
    S.layer(dict(C_in=16, C_out=16, H=16, W=16, kh=3, stride=1, depthwise=False, n_images=1, c_n=2))


# ---------------------------------------------------------------- ResNet-20 shapes at N = 8192, L = 3
@pytest.fixture(scope="module")
def resnet():
    return Setup(8192, 3, 50)


@pytest.fixture(scope="module")
def resnet_stack(resnet):
    """The 19 layers of the ResNet-20 stack with the stack's seeds: the library's input ciphertexts
    (equal to the oracle's encryption) and the oracle's outputs for every output ciphertext."""
    S = resnet
    rows = []
    for i in range(len(synth.resnet20_convs())):
        sp = synth.stack_layer("resnet20", i)
        d = H.conv_desc(**sp)
        ol = conv.Layout(N=S.N, **sp)
        act, wt, seed = synth.stack_inputs("resnet20", i, S.P.t)
        gs = H.he_layer_galois(S.p, d)
        gk = H.he_galois_keys(S.p, S.sk, gs, synth.SEED_KEYS)
        cts = H.he_encrypt_image(S.p, S.sk, d, act, seed, S.info)
        ref_in = conv.encrypt_image(S.P, ol, S.s, act, seed)
        assert (cts == ref_in).all(), f"layer {i}: library encryption differs from the oracle's"
        ref = conv.he_conv(S.P, ol, wt, ref_in, S.oracle_keys(gs))
        rows.append(dict(spec=sp, d=d, act=act, wt=wt, gk=gk, cts=cts, ref=ref))
    yield rows
    for r in rows:
        H.he_galkeys_destroy(r["gk"])


@pytest.mark.parametrize("li", range(19))
def test_resnet20_layer_matches_oracle(resnet, resnet_stack, li):
    """Every output ciphertext of every ResNet-20 layer, per-layer form, word for word."""
    r = resnet_stack[li]
    out = gpu_layer(resnet.p, r["gk"], r["d"], r["wt"], r["cts"], resnet.L, resnet.N)
    assert out.shape == r["ref"].shape
    bad = [c for c in range(len(out)) if not (out[c] == r["ref"][c]).all()]
    assert not bad, f"layer {li}: ciphertexts {bad[:8]} differ from the oracle"
    dec = H.he_decrypt_image(resnet.p, resnet.sk, r["d"], out)
    sp = r["spec"]
    assert (dec == conv.conv_plain(r["act"], r["wt"], sp["stride"], 1, False, resnet.P.t)).all()


@pytest.mark.parametrize("spec", [
    dict(C_in=16, C_out=16, H=32, W=32, kh=3, stride=1, depthwise=False, n_images=1, c_n=4),
    dict(C_in=32, C_out=64, H=16, W=16, kh=3, stride=2, depthwise=False, n_images=1, c_n=4),
])
def test_cn4_resnet20_shapes_match_oracle(resnet, spec):
    """ResNet-20 layer shapes with c_n = 4 at N = 8192, L = 3: every output ciphertext."""
    resnet.layer(spec)


# ---------------------------------------------------------------- largest ring
def test_largest_ring_depthwise_and_pointwise():
    S = Setup(16384, 4, 50)
    S.layer(dict(C_in=4, C_out=4, H=40, W=40, kh=3, stride=2, depthwise=True, n_images=2, c_n=2), sample=[1])
    S.layer(dict(C_in=6, C_out=4, H=20, W=20, kh=1, stride=1, depthwise=False, n_images=3, c_n=2), sample=[1])


# ---------------------------------------------------------------- streams and repeats
def test_repeat_on_side_stream_and_host_path(small):
    spec = dict(C_in=4, C_out=6, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=2, c_n=2)
    d = H.conv_desc(**spec)
    act = synth.activations((2, 4, 6, 6), small.P.t)
    wt = synth.weights((6, 4, 3, 3))
    gk = H.he_galois_keys(small.p, small.sk, H.he_layer_galois(small.p, d), synth.SEED_KEYS)
    cts = H.he_encrypt_image(small.p, small.sk, d, act, synth.SEED_ENC, small.info)
    s = torch.cuda.Stream()
    a = gpu_layer(small.p, gk, d, wt, cts, 2, 1024, stream=s)
    b = gpu_layer(small.p, gk, d, wt, cts, 2, 1024)
    assert (a == b).all()
    plan = H.he_conv_plan(small.p, gk, d, wt)
    n_in, n_out, ws = H.he_conv_sizes(plan)
    h_out = np.zeros(n_out, dtype=np.uint64)
    d_in = torch.empty(n_in, dtype=torch.int64, device="cuda")
    d_out = torch.empty(n_out, dtype=torch.int64, device="cuda")
    d_ws = torch.empty(ws // 8 + 1, dtype=torch.int64, device="cuda")
    H.he_conv_forward_host(plan, np.ascontiguousarray(cts.reshape(-1)), h_out, d_in.data_ptr(), d_out.data_ptr(),
                           d_ws.data_ptr())
    assert (h_out.reshape(a.shape) == a).all()
    H.he_plan_destroy(plan)


# ---------------------------------------------------------------- both MAC implementations
@pytest.mark.parametrize("impl", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("spec", [SMALL[0], SMALL[1], SMALL[4], SMALL[7], SMALL[11]])
def test_mac_implementations(small, spec, impl):
    """1 lazy CUDA-core, 2 tensor-core in the automatic form, 3 eager (reduced after every CMult
    and HAdd, Sec. 3.2.2's conventional form), 4 tensor-core with in-kernel fp16 conversion, 5
    tensor-core fed with operand images written by the key switch, 6 key switch fused into the
    tensor-core MAC, 7 operand images on CTA pairs (rows as the MMA's M), 8 operand images in chunk
    passes (up to 256 rows per CTA): all give the oracle's words."""
    small.layer(spec, mac_impl=impl)


def test_eager_mac_rejects_depthwise(small):
    d = H.conv_desc(**SMALL[2])
    gk = H.he_galois_keys(small.p, small.sk, H.he_layer_galois(small.p, d), synth.SEED_KEYS)
    with pytest.raises(H.HyenaError) as e:
        H.he_conv_plan(small.p, gk, d, synth.weights((4, 1, 3, 3)), mac_impl=3)
    assert e.value.code == H.HE_EINVAL
    H.he_galkeys_destroy(gk)


def test_tensor_core_mac_is_chosen_when_exact(small):
    spec = dict(C_in=4, C_out=4, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    d = H.conv_desc(**spec)
    gk = H.he_galois_keys(small.p, small.sk, H.he_layer_galois(small.p, d), synth.SEED_KEYS)
    for wmax, expect in ((8, 4), (9, 1)):  # |s| = |v0 +- v1| <= 16 is the exactness bound (4: one row tile)
        w = np.full((4, 4, 3, 3), wmax)
        plan = H.he_conv_plan(small.p, gk, d, w)
        assert H.he_conv_info(plan) == expect
        H.he_plan_destroy(plan)
    with pytest.raises(H.HyenaError):
        H.he_conv_plan(small.p, gk, d, np.full((4, 4, 3, 3), 9), mac_impl=2)


@pytest.mark.parametrize("pairs", [2048 // 18, 228])
def test_tensor_core_mac_at_the_exactness_bound(pairs):
    """Every scalar 16 and every chunk at -512 drive each fp32 sum to its largest magnitude.
    A zero ciphertext makes every rotated residue 0 (all chunks 0 -> -512 after the offset).
    113 pairs: K = 2034 terms in one accumulation of the in-kernel conversion form (mac_impl 4);
    the image form pads each rotation's 113 terms to 120, 2160 terms in two segments.  228 pairs:
    K = 4104 terms, three segments (2048 + 2048 + 8; the image form 4176 terms) whose results add
    mod q in the output."""
    S = Setup(1024, 2, 25)
    C_in = 2 * pairs
    spec = dict(C_in=C_in, C_out=4, H=2, W=2, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    d = H.conv_desc(**spec)
    gk = H.he_galois_keys(S.p, S.sk, H.he_layer_galois(S.p, d), synth.SEED_KEYS)
    lay = H.he_layout_for_layer(S.p, d)
    zero = np.zeros((lay.n_ct_in, 2, 2, 1024), dtype=np.uint64)
    w = np.full((4, C_in, 3, 3), 8)
    for impl in (2, 4, 5, 6, 7, 8):
        out_tc = gpu_layer(S.p, gk, d, w, zero, 2, 1024, mac_impl=impl)
        assert (out_tc == 0).all()
    # and on a real encryption, the tensor-core path equals the CUDA-core path word for word
    act = synth.activations((1, C_in, 2, 2), S.P.t)
    cts = H.he_encrypt_image(S.p, S.sk, d, act, synth.SEED_ENC, S.info)
    w = np.where(synth.weights((4, C_in, 3, 3)) >= 0, 8, -8)
    a = gpu_layer(S.p, gk, d, w, cts, 2, 1024, mac_impl=1)
    b = gpu_layer(S.p, gk, d, w, cts, 2, 1024, mac_impl=2)
    c = gpu_layer(S.p, gk, d, w, cts, 2, 1024, mac_impl=4)
    e = gpu_layer(S.p, gk, d, w, cts, 2, 1024, mac_impl=5)
    f = gpu_layer(S.p, gk, d, w, cts, 2, 1024, mac_impl=6)
    h = gpu_layer(S.p, gk, d, w, cts, 2, 1024, mac_impl=7)
    i = gpu_layer(S.p, gk, d, w, cts, 2, 1024, mac_impl=8)
    assert (a == b).all() and (a == c).all() and (a == e).all() and (a == f).all() and (a == h).all()
    assert (a == i).all()
    dec = H.he_decrypt_image(S.p, S.sk, d, b)
    assert (dec == conv.conv_plain(act, w, 1, 1, False, S.P.t)).all()


@pytest.mark.parametrize("impl", [4, 5, 6, 7, 8])
@pytest.mark.parametrize("C_in", [240, 512])
def test_tensor_core_multi_segment_matches_oracle(small, C_in, impl):
    """Contractions longer than one exact fp32 accumulation: K = 2160 terms (two segments of at
    most 2048) and K = 4608 (three segments, the 512-channel layers of VGG-16), whose segment
    results add mod q in the output, in each tensor-core form (in-kernel conversion 4, operand
    images 5, fused key switch 6, operand images on CTA pairs 7, chunk passes 8); every output
    ciphertext word for word against the oracle."""
    spec = dict(C_in=C_in, C_out=6, H=4, W=4, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    small.layer(spec, label=C_in, mac_impl=impl)


@pytest.mark.parametrize("C_out,cluster", [(128, 0), (128, 2), (256, 4), (512, 8), (1024, 8), (200, 2)])
def test_tensor_core_clusters_match_oracle(small, C_out, cluster):
    """Layers wider than one 96-row tile, with the tensor-core MAC in clusters of 2, 4 or 8 CTAs
    that share each operand image by TMA multicast (tc_cluster), or without (0): every output
    ciphertext word for word against the oracle."""
    spec = dict(C_in=6, C_out=C_out, H=3, W=3, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    small.layer(spec, label=C_out, mac_impl=2, tc_cluster=cluster)


@pytest.mark.parametrize("C_out,c_n", [(256, 2), (512, 2), (300, 2), (128, 1), (520, 1), (40, 2)])
def test_cta_pair_mac_matches_oracle(small, C_out, c_n):
    """The operand-image MAC on CTA pairs (mac_impl 7: tcgen05 cta_group::2, 256 scalar rows per
    pair as the MMA's M, 64 slots as its N): full, several and ragged pair tiles, packed and
    unpacked; every output ciphertext word for word against the oracle."""
    spec = dict(C_in=6, C_out=C_out, H=3, W=3, kh=3, stride=1, depthwise=False, n_images=1, c_n=c_n)
    small.layer(spec, label=C_out, mac_impl=7)


@pytest.mark.parametrize("C_out,c_n", [(256, 2), (512, 2), (300, 2), (128, 1), (520, 1), (96, 2), (40, 2)])
def test_chunk_pass_mac_matches_oracle(small, C_out, c_n):
    """The operand-image MAC in chunk passes (mac_impl 8: up to 256 rows per CTA, floor(512 / rows)
    chunks per pass): items of 256, ragged and fewer rows, two to five chunks per pass, packed and
    unpacked; every output ciphertext word for word against the oracle."""
    spec = dict(C_in=6, C_out=C_out, H=3, W=3, kh=3, stride=1, depthwise=False, n_images=1, c_n=c_n)
    small.layer(spec, label=C_out + 1, mac_impl=8)


@pytest.mark.parametrize("c_n", [1, 2])
def test_image_key_switch_rotation_groups(small, c_n):
    """A small image-form layer whose key switch splits its rotations into groups to fill the GPU:
    136 input channels at N = 1024 ask for 4 groups of 9 rotations (unpacked) or 8 of 18 (packed),
    which as groups of ceil(9 / 4) = 3 and ceil(18 / 8) = 3 rotations need only 3 and 6; every
    rotation is keyed once and every output ciphertext equals the oracle's."""
    spec = dict(C_in=136, C_out=8, H=3, W=3, kh=3, stride=1, depthwise=False, n_images=1, c_n=c_n)
    small.layer(spec, label=136 + c_n, mac_impl=5)


def test_cta_pair_mac_takes_no_cluster_or_rows(small):
    spec = dict(C_in=6, C_out=16, H=3, W=3, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    d = H.conv_desc(**spec)
    gk = H.he_galois_keys(small.p, small.sk, H.he_layer_galois(small.p, d), synth.SEED_KEYS)
    for impl in (7, 8):
        for kw in ({"tc_cluster": 2}, {"tc_rows": 32}):
            with pytest.raises(H.HyenaError) as e:
                H.he_conv_plan(small.p, gk, d, synth.weights((16, 6, 3, 3)), mac_impl=impl, **kw)
            assert e.value.code == H.HE_EINVAL
    H.he_galkeys_destroy(gk)


def test_tensor_core_cluster_needs_enough_rows(small):
    spec = dict(C_in=6, C_out=16, H=3, W=3, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    d = H.conv_desc(**spec)
    gk = H.he_galois_keys(small.p, small.sk, H.he_layer_galois(small.p, d), synth.SEED_KEYS)
    for cl in (8, 3):
        with pytest.raises(H.HyenaError) as e:
            H.he_conv_plan(small.p, gk, d, synth.weights((16, 6, 3, 3)), tc_cluster=cl)
        assert e.value.code == H.HE_EINVAL
    H.he_galkeys_destroy(gk)


# ---------------------------------------------------------------- batched execution
def _plan_and_inputs(S, spec, label, mac_impl=0):
    d = H.conv_desc(**spec)
    act = synth.activations((spec["n_images"], spec["C_in"], spec["H"], spec["W"]), S.P.t, label=label)
    wt = synth.weights((spec["C_out"], 1 if spec["depthwise"] else spec["C_in"], spec["kh"], spec["kh"]), label=label)
    gk = H.he_galois_keys(S.p, S.sk, H.he_layer_galois(S.p, d), synth.SEED_KEYS)
    plan = H.he_conv_plan(S.p, gk, d, wt, mac_impl=mac_impl)
    cts = H.he_encrypt_image(S.p, S.sk, d, act, synth.SEED_ENC + label, S.info)
    return plan, gk, cts


def test_batch_equals_single_layers(small):
    """One launch per stage over mixed layers (c_n 1, 2 and 4, depthwise, 1x1, all three MAC kinds)."""
    specs = [SMALL[0], SMALL[1], SMALL[2], SMALL[3], SMALL[7], SMALL[11], SMALL[5], SMALL[4], SMALL[8], CN4[0], CN4[1],
             CN4[6]]
    impls = [0, 1, 0, 0, 2, 1, 0, 3, 3, 0, 1, 1]
    items = [_plan_and_inputs(small, sp, i, impl) for i, (sp, impl) in enumerate(zip(specs, impls))]
    plans = [it[0] for it in items]
    refs, d_ins, d_outs = [], [], []
    for plan, gk, cts in items:
        n_in, n_out, ws = H.he_conv_sizes(plan)
        d_in = to_dev(cts)
        ref = torch.empty(n_out, dtype=torch.int64, device="cuda")
        d_ws = torch.empty(ws // 8 + 1, dtype=torch.int64, device="cuda")
        H.he_conv_forward(plan, d_in.data_ptr(), ref.data_ptr(), d_ws.data_ptr())
        refs.append(ref)
        d_ins.append(d_in)
        d_outs.append(torch.full((n_out,), -1, dtype=torch.int64, device="cuda"))
    b = H.he_batch_create(plans)
    ws = torch.empty(H.he_batch_workspace_bytes(b) // 8 + 1, dtype=torch.int64, device="cuda")
    H.he_batch_forward(b, [t.data_ptr() for t in d_ins], [t.data_ptr() for t in d_outs], ws.data_ptr())
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(d_outs[i], refs[i]), f"layer {i} differs in the batch"
        d_outs[i].fill_(-1)
    s = torch.cuda.Stream()
    for _ in range(2):  # capture, then replay
        H.he_batch_graph_launch(b, [t.data_ptr() for t in d_ins], [t.data_ptr() for t in d_outs], ws.data_ptr(),
                                s.cuda_stream)
        s.synchronize()
        for i in range(len(plans)):
            assert torch.equal(d_outs[i], refs[i]), f"layer {i} differs in the graph replay"
            d_outs[i].fill_(-1)
    # end to end from pinned host buffers
    h_ins = [t.cpu().pin_memory() for t in d_ins]
    h_outs = [torch.full((t.numel(),), -1, dtype=torch.int64).pin_memory() for t in d_outs]
    for t in d_ins:
        t.fill_(0)
    H.he_batch_forward_host(b, [t.data_ptr() for t in h_ins], [t.data_ptr() for t in h_outs],
                            [t.data_ptr() for t in d_ins], [t.data_ptr() for t in d_outs], ws.data_ptr(), s.cuda_stream)
    for i in range(len(plans)):
        assert torch.equal(h_outs[i], refs[i].cpu()), f"layer {i} differs through the host path"
    # the same through a batch of one layer per wave (the in-order host path)
    b1 = H.he_batch_create_limited(plans, 1)
    assert H.he_batch_waves(b1) == len(plans)
    ws1 = torch.empty(H.he_batch_workspace_bytes(b1) // 8 + 1, dtype=torch.int64, device="cuda")
    for t in h_outs:
        t.fill_(-1)
    H.he_batch_forward_host(b1, [t.data_ptr() for t in h_ins], [t.data_ptr() for t in h_outs],
                            [t.data_ptr() for t in d_ins], [t.data_ptr() for t in d_outs], ws1.data_ptr(),
                            s.cuda_stream)
    for i in range(len(plans)):
        assert torch.equal(h_outs[i], refs[i].cpu()), f"layer {i} differs through the host path in waves"
    # waves of several layers (the first wave's input NTTs run layer by layer behind its copies)
    sizes = sorted((H.he_conv_sizes(pl)[2] + 255) // 256 * 256 for pl in plans)
    b2 = H.he_batch_create_limited(plans, sizes[-1] + sizes[-2])  # the two largest share the first wave
    assert 2 <= H.he_batch_waves(b2) < len(plans)
    ws2 = torch.empty(H.he_batch_workspace_bytes(b2) // 8 + 1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        for t in h_outs:
            t.fill_(-1)
        H.he_batch_forward_host(b2, [t.data_ptr() for t in h_ins], [t.data_ptr() for t in h_outs],
                                [t.data_ptr() for t in d_ins], [t.data_ptr() for t in d_outs], ws2.data_ptr(),
                                s.cuda_stream)
        for i in range(len(plans)):
            assert torch.equal(h_outs[i], refs[i].cpu()), f"layer {i} differs through the host path in multi-layer waves"
    H.he_batch_destroy(b2)
    H.he_batch_destroy(b1)
    H.he_batch_destroy(b)
    for plan, gk, _ in items:
        H.he_conv_status(plan)
        H.he_plan_destroy(plan)
        H.he_galkeys_destroy(gk)


def test_batch_of_resnet20_stack_matches_oracle(resnet, resnet_stack):
    """The whole 19-layer stack in one batch, captured and replayed as a CUDA graph: every output
    ciphertext of every layer equals the oracle's, word for word, on the capture and on a replay."""
    plans, d_ins, d_outs = [], [], []
    for r in resnet_stack:
        plan = H.he_conv_plan(resnet.p, r["gk"], r["d"], r["wt"])
        n_in, n_out, _ = H.he_conv_sizes(plan)
        plans.append(plan)
        d_ins.append(to_dev(r["cts"]))
        d_outs.append(torch.full((n_out,), -1, dtype=torch.int64, device="cuda"))
    b = H.he_batch_create(plans)
    ws = torch.empty(H.he_batch_workspace_bytes(b) // 8 + 1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    for rep in range(2):
        for t in d_outs:
            t.fill_(-1)
        torch.cuda.synchronize()
        H.he_batch_graph_launch(b, [t.data_ptr() for t in d_ins], [t.data_ptr() for t in d_outs], ws.data_ptr(),
                                s.cuda_stream)
        s.synchronize()
        for i, r in enumerate(resnet_stack):
            out = from_dev(d_outs[i], r["ref"].shape)
            bad = [c for c in range(len(out)) if not (out[c] == r["ref"][c]).all()]
            assert not bad, f"replay {rep}, layer {i}: ciphertexts {bad[:8]} differ from the oracle"
    H.he_batch_destroy(b)
    for plan in plans:
        H.he_conv_status(plan)
        H.he_plan_destroy(plan)


# ---------------------------------------------------------------- failure detection
def test_bounded_wait_gives_up_and_the_context_stays_usable(small):
    """A wait on an mbarrier that nothing arrives at gives up after its poll limit and reports
    HE_ETIMEOUT through the device status word (no fault, no hang); afterwards the same context
    still runs a tensor-core layer to the oracle's words."""
    import time

    t0 = time.time()
    assert H.he_selftest_bounded_wait() == H.HE_ETIMEOUT
    assert time.time() - t0 < 30
    small.layer(SMALL[0], mac_impl=2)


# ---------------------------------------------------------------- limb widths and digit counts
@pytest.mark.parametrize("limb_bits,L,w", [(54, 2, 27), (30, 3, 15), (40, 4, 13)])
def test_other_limb_widths_and_digit_counts(limb_bits, L, w):
    """Limbs of 54 bits (the widest the key switch's 25-bit split allows; the tensor core needs
    limbs below 2^50, so the CUDA-core MAC runs), 30 bits (two digits per limb) and 40 bits with
    4 digits per limb (L l = 16, the largest key-switch template)."""
    S = Setup(1024, L, w, limb_bits)
    assert S.info.l * L <= 16 and max(S.info.q[:L]).bit_length() == limb_bits
    spec = dict(C_in=4, C_out=6, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=2, c_n=2)
    S.layer(spec)
    S.layer(dict(spec, c_n=1))


# ---------------------------------------------------------------- polyphase stride 2
POLY = [
    dict(C_in=3, C_out=5, H=7, W=9, kh=3, stride=2, depthwise=False, n_images=2, c_n=2, polyphase=1),
    dict(C_in=4, C_out=6, H=10, W=10, kh=3, stride=2, depthwise=False, n_images=1, c_n=1, polyphase=1),
    dict(C_in=4, C_out=4, H=8, W=6, kh=3, stride=2, depthwise=True, n_images=3, c_n=2, polyphase=1),
    dict(C_in=3, C_out=3, H=9, W=7, kh=3, stride=2, depthwise=True, n_images=2, c_n=1, polyphase=1),
    dict(C_in=6, C_out=200, H=6, W=6, kh=3, stride=2, depthwise=False, n_images=1, c_n=2, polyphase=1),
]


@pytest.mark.parametrize("impl", [0, 1, 4, 5])
@pytest.mark.parametrize("spec", POLY)
def test_polyphase_layer_matches_oracle(small, spec, impl):
    """Polyphase packing of 3x3 stride-2 layers: every output ciphertext equals the oracle's layer
    on the derived stride-1 layer of the phase planes, word for word (each MAC form the layer
    admits), and decrypts to the stride-2 convolution."""
    if impl in (4, 5) and spec["depthwise"]:
        pytest.skip("depthwise layers run on CUDA cores")
    S, N, L = small, small.N, small.L
    d = H.conv_desc(**spec)
    act = synth.activations((spec["n_images"], spec["C_in"], spec["H"], spec["W"]), S.P.t, label=spec["H"])
    wt = synth.weights((spec["C_out"], 1 if spec["depthwise"] else spec["C_in"], 3, 3), label=spec["W"])
    gk = H.he_galois_keys(S.p, S.sk, H.he_layer_galois(S.p, d), synth.SEED_KEYS)
    cts = H.he_encrypt_image(S.p, S.sk, d, act, synth.SEED_ENC, S.info)
    out = gpu_layer(S.p, gk, d, wt, cts, L, N, mac_impl=impl)
    ol = conv.Layout(N=N, **conv.polyphase_spec(spec))
    planes = conv.polyphase_planes(act, spec["c_n"])
    ref_in = conv.encrypt_image(S.P, ol, S.s, planes, synth.SEED_ENC)
    assert (ref_in == cts).all()
    w2 = conv.polyphase_weights(wt, spec["C_in"], spec["c_n"], spec["depthwise"])
    ref = conv.he_conv(S.P, ol, w2, ref_in, S.oracle_keys(conv.galois_elements(S.P, ol)))
    bad = [c for c in range(len(out)) if not (out[c] == ref[c]).all()]
    assert not bad, f"ciphertexts {bad[:8]} differ from the oracle"
    dec = H.he_decrypt_image(S.p, S.sk, d, out)
    assert (dec == conv.conv_plain(act, wt, 2, 1, spec["depthwise"], S.P.t)).all()
    H.he_galkeys_destroy(gk)
