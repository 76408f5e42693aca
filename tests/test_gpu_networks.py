"""Full-size network stacks on the GPU, batched in waves under a workspace limit.

  * VGG-16: the 13 3x3 convolutions on 8 images of 224x224, N = 16384, L = 4
    (6128 input and 8704 output ciphertexts, over 100 GB of rotated copies in
    all, so the batch runs in waves that share one workspace region).
  * MobileNetV1: the 27 convolutions (3x3 depthwise and 1x1 pointwise) on 32
    images of 224x224, N = 8192, L = 4, mixed layer sizes in one batch.

For every layer:
  * the batched output equals he_conv_forward of that layer word for word;
  * one seeded output ciphertext equals the oracle's, word for word.  A deep
    layer's output ciphertext depends on all (up to 256) input ciphertexts of
    its row-unit, each rotated 17 times, which takes the plain oracle minutes
    per layer even on all cores, so the oracle's words for these samples are
    stored as SHA-256 digests by tests/golden/make_network_samples.py (which
    calls only the oracle; it also checks each sample's decryption against the
    plain convolution).  The first layer is also recomputed by the oracle here.
Every output of the first and the last layer is decrypted and compared with the
plain convolution (torch.nn.functional.conv2d in float64, exact here: every
partial sum is an integer below 2^20 * 8 * 4608 < 2^53).
"""
import hashlib
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import bfv, conv  # noqa: E402
from oracle import params as prm  # noqa: E402
from paper_2311_12519_gb300 import hyena as H  # noqa: E402

pytestmark = pytest.mark.gpu

WAVE_LIMIT = 40 << 30  # bytes of workspace per wave
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "network_samples.json")


def plain_conv(act, wt, stride, depthwise, t):
    x = torch.from_numpy(act.astype(np.float64))
    w = torch.from_numpy(wt.astype(np.float64))
    y = torch.nn.functional.conv2d(x, w, stride=stride, padding=(wt.shape[-1] - 1) // 2,
                                   groups=act.shape[1] if depthwise else 1)
    return np.mod(y.numpy().astype(np.int64), t)


def digest(ct):
    return hashlib.sha256(np.ascontiguousarray(ct, dtype="<u8").tobytes()).hexdigest()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _run_stack(stack, oracle_samples, decrypt_layers):
    golden = json.load(open(GOLDEN))[stack]
    shapes, N, L, n_images = synth.STACKS[stack]
    assert (golden["N"], golden["L"], golden["images"]) == (N, L, n_images)
    p = H.he_params_create(N, L, decomp_bits=golden["w"])
    info = H.he_params_info(p)
    sk = H.he_keygen(p, synth.SEED_KEYS)
    n_layers = len(shapes())
    specs = [synth.stack_layer(stack, i) for i in range(n_layers)]
    descs = [H.conv_desc(**sp) for sp in specs]
    gal = sorted(set(int(g) for d in descs for g in H.he_layer_galois(p, d)))
    gk = H.he_galois_keys(p, sk, gal, synth.SEED_KEYS)
    plans, d_ins, d_outs, host_in, acts, wts = [], [], [], [], [], []
    for i, (sp, d) in enumerate(zip(specs, descs)):
        act, wt, enc_seed = synth.stack_inputs(stack, i, info.t)
        cts = H.he_encrypt_image(p, sk, d, act, enc_seed, info)
        plans.append(H.he_conv_plan(p, gk, d, wt))
        n_in, n_out, _ = H.he_conv_sizes(plans[-1])
        assert n_in == cts.size
        assert n_out // (2 * L * N) == golden["samples"][i]["n_ct_out"]
        d_ins.append(torch.from_numpy(cts.reshape(-1).view(np.int64)).cuda())
        d_outs.append(torch.full((n_out,), -1, dtype=torch.int64, device="cuda"))
        keep = i in oracle_samples or i in decrypt_layers
        host_in.append(cts if i in oracle_samples else None)
        acts.append(act if keep else None)
        wts.append(wt if keep else None)
    b = H.he_batch_create_limited(plans, WAVE_LIMIT)
    assert H.he_batch_waves(b) >= 2, "the stack should need more than one wave at this limit"
    ws_bytes = H.he_batch_workspace_bytes(b)
    assert ws_bytes <= WAVE_LIMIT or ws_bytes == max(H.he_conv_sizes(pl)[2] for pl in plans)
    ws = torch.empty(ws_bytes // 8 + 1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    H.he_batch_graph_launch(b, [t.data_ptr() for t in d_ins], [t.data_ptr() for t in d_outs], ws.data_ptr(),
                            s.cuda_stream)
    s.synchronize()
    for plan in plans:
        H.he_conv_status(plan)
    # one seeded output ciphertext of every layer against the oracle's stored words
    bad = []
    for i, row in enumerate(golden["samples"]):
        out = d_outs[i].cpu().numpy().view(np.uint64).reshape(-1, 2, L, N)
        if digest(out[row["ct"]]) != row["sha256"]:
            bad.append((i, row["ct"]))
    assert not bad, f"(layer, ciphertext) samples that differ from the oracle: {bad}"
    # batched = plain per-layer, every layer, word for word (the workspace is free again)
    tmp = torch.empty(max(t.numel() for t in d_outs), dtype=torch.int64, device="cuda")
    for i, plan in enumerate(plans):
        n_out = d_outs[i].numel()
        tmp[:n_out].fill_(-1)
        H.he_conv_forward(plan, d_ins[i].data_ptr(), tmp.data_ptr(), ws.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(tmp[:n_out], d_outs[i]), f"layer {i}: batched output differs from he_conv_forward"
    del tmp, ws
    # the first layer's samples recomputed by the oracle here, from the same input ciphertexts
    P = prm.make_params(N=N, L=L, w=golden["w"])
    s_or = bfv.keygen(P, synth.SEED_KEYS)
    ksk = {}
    for i, cts in sorted(oracle_samples.items()):
        ol = conv.Layout(N=N, **specs[i])
        for g in H.he_layer_galois(p, descs[i]):
            if g not in ksk:
                ksk[g] = bfv.galois_key(P, s_or, g, synth.SEED_KEYS)
        out = d_outs[i].cpu().numpy().view(np.uint64).reshape(-1, 2, L, N)
        ref = conv.he_conv(P, ol, wts[i], host_in[i], ksk, out_cts=cts)
        for c in cts:
            assert (out[c] == ref[c]).all(), f"layer {i}, ciphertext {c} differs from the oracle"
    for i in decrypt_layers:
        sp = specs[i]
        out = d_outs[i].cpu().numpy().view(np.uint64).reshape(-1, 2, L, N)
        dec = H.he_decrypt_image(p, sk, descs[i], out)
        plain = plain_conv(acts[i], wts[i], sp["stride"], sp["depthwise"], info.t)
        assert (dec == plain).all(), f"layer {i}: decryption differs from the plain convolution"
    H.he_batch_destroy(b)
    for plan in plans:
        H.he_plan_destroy(plan)
    H.he_galkeys_destroy(gk)
    H.he_seckey_destroy(sk)
    H.he_params_destroy(p)


def test_vgg16_stack_8_images_batched_in_waves():
    _run_stack("vgg16", oracle_samples={0: [0, 1791]}, decrypt_layers=[0, 12])


def test_mobilenet_v1_stack_32_images_batched_in_waves():
    _run_stack("mobilenet", oracle_samples={0: [3], 2: [5], 3: [0, 77]}, decrypt_layers=[0, 3, 26])
