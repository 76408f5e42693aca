"""Writes network_samples.json: the oracle's words for one seeded output ciphertext of every
layer of the VGG-16 (8 images, N = 16384, L = 4) and MobileNetV1 (32 images, N = 8192, L = 4)
stacks, as a SHA-256 digest of the ciphertext's little-endian uint64 words [2][L][N] plus a few
words for diagnosis.

Calls only the oracle (oracle/) and the seeded workload generators (synth/): the input
ciphertexts of the sampled row-unit are encrypted by the oracle with the stack's seeds, the
layer's hoisted rotations and sums are computed by oracle.conv.he_conv (Sec. 2.3 hoisting,
Sec. 3.1 Walsh-Hadamard packing, eager reduction), and the result's decryption is checked against
the plain convolution at every valid position of that ciphertext before it is stored.

A deep layer's output ciphertext depends on all input ciphertexts of its row-unit (up to 256
here, each rotated 17 times), which takes the oracle minutes per layer even on all cores; the
stored digests let the GPU tests compare every layer's sample word for word in seconds.

Usage: python tests/golden/make_network_samples.py [--stacks vgg16,mobilenet] [--polyphase | --dw-cn4 | --cn1]
(--polyphase: the 3x3 stride-2 layers only, with polyphase packing, as entries '<stack>-polyphase';
--dw-cn4: the depthwise layers only, packed four channels per ciphertext, as '<stack>-dwcn4';
--cn1: the layers whose tiles fill the slot rows, unpacked (c_n = 1: no more input or output
ciphertexts than with c_n = 2), as '<stack>-cn1').
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import bfv, conv  # noqa: E402
from oracle import params as prm  # noqa: E402

OUT = os.path.join(HERE, "network_samples.json")
STACK_LABEL = {"resnet20": 1, "vgg16": 2, "mobilenet": 3}


def digest(ct: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(ct, dtype="<u8").tobytes()).hexdigest()


def fills_rows(N, sp):
    """True if the layer packed one channel per ciphertext (c_n = 1) needs no more input and output
    ciphertexts than with c_n = 2: its tiles already fill the slot rows, so packing would only add
    Hadamard rows and row-swap rotations (the paper packs only when an image leaves slots empty)."""
    a = conv.Layout(N=N, **dict(sp, c_n=1))
    b = conv.Layout(N=N, **dict(sp, c_n=2))
    return a.n_ct_in <= b.n_ct_in and a.n_ct_out <= b.n_ct_out


def sample_layer(P, s, ksk, stack, i, polyphase=False, dw_cn4=False, c_n=None):
    sp = synth.stack_layer(stack, i, polyphase, dw_cn4)
    if c_n is not None:
        sp["c_n"] = c_n
    act, wt, enc_seed = synth.stack_inputs(stack, i, P.t)
    poly = sp.get("polyphase", 0)
    if poly:
        # polyphase packing: the oracle's layer on the derived stride-1 layer of the phase planes
        act_in = conv.polyphase_planes(act, sp["c_n"])
        wt_in = conv.polyphase_weights(wt, sp["C_in"], sp["c_n"], sp["depthwise"])
        lay = conv.Layout(N=P.N, **conv.polyphase_spec(sp))
    else:
        act_in, wt_in = act, wt
        lay = conv.Layout(N=P.N, **sp)
    c = synth.sample_index(100 * STACK_LABEL[stack] + i, lay.n_ct_out)
    ru, g = divmod(c, lay.out_groups)
    dw = lay.depthwise
    need = [ru * lay.in_groups + (g if dw else j) for j in ([0] if dw else range(lay.in_groups))]
    cts = conv.encrypt_image(P, lay, s, act_in, enc_seed, only=need)
    for gal in conv.galois_elements(P, lay):
        if gal not in ksk:
            ksk[gal] = bfv.galois_key(P, s, gal, synth.SEED_KEYS)
    out = conv.he_conv(P, lay, wt_in, cts, ksk, out_cts=[c])[c]
    # the sampled ciphertext must decrypt to the plain convolution at its valid positions
    slots = bfv.decode(P, bfv.decrypt(P, s, out))
    inv = pow(conv.output_scale(P, lay), -1, P.t)
    pos = conv.ct_positions(lay, c)
    imgs = sorted({q[0] for q in pos})
    plain = conv.conv_plain(act[imgs], wt, sp["stride"], 1 if poly else lay.P, sp["depthwise"], P.t)
    ok = all(int(slots[x]) * inv % P.t == plain[imgs.index(im), ch, y, xx] for im, ch, y, xx, x in pos)
    assert pos and ok, f"{stack} layer {i}: oracle sample fails decryption"
    return {"layer": i, "n_ct_out": lay.n_ct_out, "ct": c, "sha256": digest(out),
            "words": [int(out[p, k, x]) for p in (0, 1) for k in (0, P.L - 1) for x in (0, P.N - 1)]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--stacks", default="vgg16,mobilenet")
    ap.add_argument("--polyphase", action="store_true",
                    help="sample the 3x3 stride-2 layers with polyphase packing (entries '<stack>-polyphase')")
    ap.add_argument("--dw-cn4", action="store_true",
                    help="sample the depthwise layers packed with c_n = 4 (entries '<stack>-dwcn4')")
    ap.add_argument("--cn1", action="store_true",
                    help="sample the layers whose tiles fill the rows, with c_n = 1 (entries '<stack>-cn1')")
    args = ap.parse_args()
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for stack in args.stacks.split(","):
        shapes, N, L, images = synth.STACKS[stack]
        P = prm.make_params(N=N, L=L, w=50)
        s = bfv.keygen(P, synth.SEED_KEYS)
        ksk = {}
        rows = []
        for i, sh in enumerate(shapes()):
            if args.polyphase and not (sh.stride == 2 and sh.k == 3):
                continue
            if args.dw_cn4 and not sh.depthwise:
                continue
            if args.cn1 and not fills_rows(N, synth.stack_layer(stack, i)):
                continue
            t0 = time.time()
            rows.append(sample_layer(P, s, ksk, stack, i, args.polyphase, args.dw_cn4, 1 if args.cn1 else None))
            print(f"{stack} layer {i}: ct {rows[-1]['ct']} in {time.time() - t0:.0f} s", flush=True)
        key = stack + ("-polyphase" if args.polyphase else "-dwcn4" if args.dw_cn4 else "-cn1" if args.cn1 else "")
        data[key] = {"N": N, "L": L, "w": 50, "images": images, "seeds": "keys 1, encryption 2 + layer, "
                     "activations label = layer, weights label = layer", "samples": rows}
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
