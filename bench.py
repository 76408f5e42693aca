"""Throughput of encrypted convolution on the GB300 (one JSON line on stdout).

Default workload: the 13 3x3 convolutions of VGG-16 on 8 images of 224x224
per GPU, N = 16384, L = 4 RNS limbs of 50 bits, t = 786433, Hyena packing
where it saves ciphertexts (c_n = 2 for the 28x28 and 14x14 layers; the 224 to
56 layers, whose tiles fill the slot rows, unpacked with c_n = 1; --packing 2
packs all): 6100 input and 8704 output ciphertexts per step.  A step runs all
13 layers once on synthetic ciphertexts resident in HBM.  value = layers/s
over all ranks of the batched form (one launch per stage for all layers of a
workspace wave, replayed as a CUDA graph); the plain per-layer form
(he_conv_forward per layer) is reported beside it, with modMAC/s.  e2e
repeats the step from pinned host buffers through he_batch_forward_host
(copies inside the timed region).  After the timed region, one seeded output
ciphertext of every layer is compared with the oracle's words (digests stored
by tests/golden/make_network_samples.py) and the last layer is decrypted and
compared with the plain convolution.  --workload resnet20|mobilenet measures
the ResNet-20 (1 image, N = 8192, L = 3) or MobileNetV1 (32 images) stack the
same way; --mode ablation prints one line per variant of the latency study;
--mode learned runs every layer in the learned cost model's configuration;
--impl reference times the CPU oracle instead.

Launch: python bench.py [--gpus N --steps K --warmup W]; N > 1 under
torch.distributed.run (one process per GPU, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

LIMB_BITS = 50
METRIC = "HE-conv layers/s and modMAC/s, batched vs plain per-layer, bit-exact; % HBM roof"
# workload -> (batch workspace limit in bytes or None, description)
WORKLOADS = {
    "vgg16": (64 << 30, "vgg16-3x3-stack (13 convs), 224x224, 8 images/GPU, N=16384, L=4x50-bit, t=786433, c_n=2"),
    "resnet20": (None, "resnet20-3x3-stack (19 convs), 32x32, 1 image/GPU, N=8192, L=3x50-bit, t=1032193, c_n=2"),
    "mobilenet": (64 << 30, "mobilenetv1-dw+pw-stack (27 convs), 224x224, 32 images/GPU, N=8192, L=4x50-bit, "
                            "t=1032193, c_n=2"),
}
DEFAULT_WORKLOAD = "vgg16"
L2_BYTES = 129 * 2**20
GOLDEN = os.path.join(ROOT, "tests", "golden", "network_samples.json")
# DRAM bytes (read + write) of one launch of each kernel of the batched step, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel source with this digest prefix
# (kernel_source_digest), per workload; reported as roofline traffic only while the kernels are unchanged
# keyed by the line's full workload description (packing and layer choices included)
PROFILED_TRAFFIC = {
    # profiles/vgg16_stack_batched_launches.md (every layer packed, --packing 2): the key-switch
    # stage's 4 launches of one forward
    ("vgg16-3x3-stack (13 convs), 224x224, 8 images/GPU, N=16384, L=4x50-bit, t=786433, c_n=2",
     "k_keyswitch + k_keyswitch_img"): ("326c3143f1cbf5c2", 41486645856),
}


def kernel_source_digest():
    """sha256 of device.cu up to its device-table section, without comments and blank space: the
    kernels and their launch code, which fix what a profiled launch does (the host API below them
    does not)."""
    import re

    text = open(os.path.join(ROOT, "paper_2311_12519_gb300", "csrc", "device.cu"), "rb").read()
    cut = text.find(b"// ================================================================== device tables")
    code = re.sub(rb"//[^\n]*", b"", text[:cut] if cut > 0 else text)
    return hashlib.sha256(re.sub(rb"\s+", b" ", code))


def host_cores():
    """Host threads this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def layer_specs(workload, layers=None, polyphase=False, dw_cn4=False):
    """The stack's layer descriptions (all, or the listed layer indices), ring and images; with
    `polyphase`, its 3x3 stride-2 layers use polyphase packing; with `dw_cn4`, its other depthwise
    layers pack four channels per ciphertext."""
    shapes, N, L, images = synth.STACKS[workload]
    idx = range(len(shapes())) if layers is None else layers
    return [synth.stack_layer(workload, i, polyphase, dw_cn4) for i in idx], N, L, images


# c_n of the stack layers: "2" packs every layer (the pair of Eq. 1); "fill" packs a layer only
# where packing saves ciphertexts (fill_packing)
PACKING_DESC = {"2": "c_n=2", "fill": "c_n per layer (1 where its tiles fill the slot rows, else 2)"}


def workload_name(wl, packing):
    return WORKLOADS[wl][1].replace("c_n=2", PACKING_DESC[packing])


def fill_packing(specs, counts):
    """c_n per layer.  The paper packs c_n = n / n_i channels only while an image leaves slots
    empty (Sec. 3.1) and runs its large inputs unpacked (Sec. 4); with many tiles per ciphertext
    the same holds per layer: a layer whose tiles fill the slot rows gets c_n = 1 (no more input
    and output ciphertexts than the pair, half its Hadamard rows and no row-swap rotations), the
    others keep c_n = 2.  `counts(spec)` gives (n_ct_in, n_ct_out) of a layer description."""
    out = []
    for s in specs:
        if s["c_n"] == 2:
            a, b = counts(dict(s, c_n=1)), counts(s)
            if a[0] <= b[0] and a[1] <= b[1]:
                s = dict(s, c_n=1)
        out.append(s)
    return out


def layer_counts(spec, lay, L, l, N):
    """Algorithmic counts of one layer (one image batch): conv and key-switch modMACs, and the
    bytes of Sec. 8(d)'s rooflines for each stage."""
    rows = spec["c_n"]  # MAC rows per output group: 1, 2 or 4
    n_rot = lay.n_galois + 1  # the rotated copies of an input ciphertext, identity included
    # a depthwise output reads one ciphertext per phase plane (four with polyphase packing)
    K = (lay.in_groups // lay.out_groups) * n_rot if spec["depthwise"] else lay.in_groups * n_rot
    conv = lay.row_units * lay.out_groups * rows * K * 2 * L * N
    ks = lay.n_ct_in * lay.n_galois * 2 * L * l * L * N
    w8 = N * 8
    return {
        "conv_modmac": conv, "ks_modmac": ks, "ks_modmac_stage": ks,
        # forward transforms of c0 and of the digits of c1 (the single digit of c1 in its own limb is c1)
        "ntt_in_transforms": lay.n_ct_in * (L + L * l * L),
        # the key stream of every Galois element once, plus the digit and c0 transforms the switch reads
        "ks_bytes": lay.n_galois * L * l * 2 * L * w8 + lay.n_ct_in * (L * l * L + L) * w8,
        "ntt_out_transforms": lay.n_ct_out * 2 * L,
        "in_bytes": lay.n_ct_in * 2 * L * w8, "out_bytes": lay.n_ct_out * 2 * L * w8,
        # rotated copies the MAC streams (this design's own traffic, not the method's minimum)
        "mac_r_bytes": lay.n_ct_in * n_rot * 2 * L * w8,
    }


def rank_inputs(workload, i, rank, t):
    """Layer i's inputs on a rank: rank 0 runs the stack's own seeds (those of the tests and the
    stored oracle samples); rank r > 0 its own activations and encryption randomness."""
    act, wt, seed = synth.stack_inputs(workload, i, t)
    if rank:
        sp = synth.stack_layer(workload, i)
        act = synth.activations(act.shape, t, label=i + 1000 * rank)
        seed = seed + 7919 * rank
        del sp
    return act, wt, seed


def reduce_max(values, device, world):
    """Max over ranks of the timed values (barrier + max timing; no data-path collective)."""
    if world <= 1:
        return list(values)
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def layers_per_second(world, n_layers, steps, seconds):
    """Whole-job throughput: every rank runs n_layers layers per step on its own images."""
    return world * n_layers * steps / seconds


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index, self.rows, self.proc, self.start = index, [], None, 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # sampling is live before the timed region starts; samples taken before it are not counted
            t0 = time.time()
            while not self.rows and time.time() - t0 < 3.0:
                time.sleep(0.01)
            self.start = len(self.rows)
        except OSError:
            self.proc = None
        return self

    def keep_busy(self, step, min_samples=3, max_seconds=2.0):
        """After the timed steps, repeats the same step (untimed, synchronised) until min_samples
        samples have been taken since the timed region began: the timed region alone is often
        shorter than the sampling interval."""
        t0 = time.time()
        while self.proc and len(self.rows) - self.start < min_samples and time.time() - t0 < max_seconds:
            step()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = self.rows[self.start:]
        sm = [float(r[0]) for r in rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 2 + i and r[2 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm),
                "window": "the timed steps, then the same step repeated untimed until 3 samples"}


# ------------------------------------------------------------------ oracle (CPU) sample
def oracle_layer_estimate(workload, i, threads, keys_cache, packing="2"):
    """Seconds the CPU oracle (oracle/conv.he_conv on `threads` host threads) needs for layer i of
    the stack, from a bounded sample: the layer with its input channels cut to `threads` channel
    groups (same ring, kernel, images and output channels), of which `threads` output ciphertexts
    of the first row-unit are computed.  The timed rotation phase gives the cost per input
    ciphertext (decomposition + hoisted rotations, one ciphertext per thread), the timed sum phase
    the cost per accumulated term of an output ciphertext (CMult + HAdd, one ciphertext per
    thread, with its reduction and PMult); the layer's estimate scales them by its own counts
    (input ciphertexts; output ciphertexts x terms)."""
    from oracle import bfv, conv
    from oracle import params as prm

    shapes, N, L, images = synth.STACKS[workload]
    if (N, L) not in keys_cache:
        P = prm.make_params(N=N, L=L, w=50)
        keys_cache[(N, L)] = (P, bfv.keygen(P, synth.SEED_KEYS), {})
    P, s, ksk = keys_cache[(N, L)]
    sp = synth.stack_layer(workload, i)
    if packing == "fill":
        sp = fill_packing([sp], lambda x: (lambda o: (o.n_ct_in, o.n_ct_out))(conv.Layout(N=N, **x)))[0]
    lay = conv.Layout(N=N, **sp)
    groups = min(threads, lay.in_groups)
    sub = dict(sp, C_in=min(sp["C_in"], sp["c_n"] * groups))
    if sp["depthwise"]:
        sub["C_out"] = sub["C_in"]
    lay_s = conv.Layout(N=N, **sub)
    act, wt, seed = synth.stack_inputs(workload, i, P.t)
    act_s = np.ascontiguousarray(act[:, :sub["C_in"]])
    wt_s = np.ascontiguousarray(wt[:sub["C_out"], :(1 if sp["depthwise"] else sub["C_in"])])
    cts = conv.encrypt_image(P, lay_s, s, act_s, seed, only=range(lay_s.in_groups), threads=threads)
    for g in conv.galois_elements(P, lay_s):
        if g not in ksk:
            ksk[g] = bfv.galois_key(P, s, g, synth.SEED_KEYS)
    n_out = min(threads, lay_s.out_groups)
    tm = {}
    conv.he_conv(P, lay_s, wt_s, cts, ksk, out_cts=list(range(n_out)), threads=threads, timings=tm)
    n_rot = len(conv.rotation_plan(P, lay_s))
    k_s = n_rot if sp["depthwise"] else lay_s.in_groups * n_rot
    k = n_rot if sp["depthwise"] else lay.in_groups * n_rot
    rot_in = lay_s.in_groups if not sp["depthwise"] else n_out
    per_ct = tm["rotations"] / rot_in
    per_term = tm["sums"] / (n_out * k_s)
    est = per_ct * lay.n_ct_in + per_term * lay.n_ct_out * k
    return est, tm["rotations"] + tm["sums"], {"layer": i, "input_cts": rot_in, "output_cts": n_out, "terms": k_s}


def oracle_sample(workload, layers, threads, packing="2"):
    """Estimated oracle seconds for each sampled layer, wall seconds spent, and a description."""
    cache, est, spent, parts = {}, [], 0.0, []
    for i in layers:
        e, w, info = oracle_layer_estimate(workload, i, threads, cache, packing)
        est.append(e)
        spent += w
        parts.append(info)
    n_layers = len(synth.STACKS[workload][0]())
    desc = (f"CPU oracle (oracle/conv.he_conv) on {threads} host threads; layers {list(layers)} of the "
            f"{n_layers}-layer stack, each cut to {threads} input channel groups with {threads} output ciphertexts "
            "computed; rotation and sum phases timed and scaled by each layer's input ciphertexts and "
            "output ciphertexts x terms; layers/s = sampled layers / estimated seconds")
    return est, spent, desc, parts


def run_reference(args, rank):
    """The oracle as the reference arm: each step estimates one layer of the stack (cycling)."""
    if rank != 0:
        return
    wl = args.workload
    n_layers = len(synth.STACKS[wl][0]())
    threads = host_cores()
    steps, warm = max(1, args.steps), max(0, args.warmup)
    cache, est = {}, []
    t0 = time.perf_counter()
    for st in range(warm + steps):
        e, _, _ = oracle_layer_estimate(wl, st % n_layers, threads, cache, args.packing)
        if st >= warm:
            est.append(e)
    wall = time.perf_counter() - t0
    value = len(est) / sum(est)
    desc = (f"CPU oracle (oracle/conv.he_conv) on {threads} host threads; step s estimates layer s mod {n_layers} "
            f"of the stack from a sample cut to {threads} input channel groups and {threads} output ciphertexts "
            "(rotation and sum phases timed, scaled by the layer's counts); layers/s = steps / estimated seconds")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "layers/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1000 * sum(est) / len(est), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload_name(wl, args.packing)},
            "wall_seconds": round(wall, 1),
            "cpu_baseline": {"value": value, "unit": "layers/s", "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def verify_outputs(H, p, sk, info, workload, specs, descs, d_outs, rank, index):
    """After the timed region, on rank 0 (whose inputs are the stack's own seeds): one seeded output
    ciphertext of every layer against the oracle's stored words, and every output ciphertext of
    the last layer decrypted and compared with the plain convolution (float64 torch conv2d)."""
    import torch

    if rank != 0:
        return {"checked": False, "why": "rank > 0 runs its own inputs; rank 0 checks the stack's seeds"}
    res = {"checked": True}
    L, N = info.L, info.N
    ctw = 2 * L * N
    try:
        golden = json.load(open(GOLDEN)).get(workload)
    except OSError:
        golden = None
    try:
        poly = {r["layer"]: r for r in json.load(open(GOLDEN)).get(workload + "-polyphase", {}).get("samples", [])}
        dwcn4 = {r["layer"]: r for r in json.load(open(GOLDEN)).get(workload + "-dwcn4", {}).get("samples", [])}
        cn1 = {r["layer"]: r for r in json.load(open(GOLDEN)).get(workload + "-cn1", {}).get("samples", [])}
    except OSError:
        poly, dwcn4, cn1 = {}, {}, {}
    if golden and (golden["N"], golden["L"]) == (N, L):
        ok, bad, skipped = 0, [], []
        for i, li in enumerate(index):
            row = golden["samples"][li]
            alt = poly if specs[i].get("polyphase") else {4: dwcn4, 1: cn1}.get(specs[i]["c_n"])
            if specs[i].get("polyphase") and specs[i]["c_n"] != 2:
                alt = {}  # phase planes without the pair: no stored sample
            if alt is not None:
                if li not in alt:
                    skipped.append(li)
                    continue
                row = alt[li]
            c = row["ct"]
            words = d_outs[i][c * ctw:(c + 1) * ctw].cpu().numpy().view(np.uint64)
            if hashlib.sha256(np.ascontiguousarray(words, dtype="<u8").tobytes()).hexdigest() == row["sha256"]:
                ok += 1
            else:
                bad.append(li)
        res["oracle_samples"] = {"layers": len(index) - len(skipped), "equal": ok, "differ": bad,
                                 "not_sampled": skipped,
                                 "what": "one seeded output ciphertext per layer vs the oracle's words (SHA-256)"}
    else:
        res["oracle_samples"] = None
    i = len(specs) - 1
    sp = specs[i]
    act, wt, _ = synth.stack_inputs(workload, index[i], info.t)
    out = d_outs[i].cpu().numpy().view(np.uint64).reshape(-1, 2, L, N)
    dec = H.he_decrypt_image(p, sk, descs[i], out)
    x = torch.from_numpy(act.astype(np.float64))
    w = torch.from_numpy(wt.astype(np.float64))
    y = torch.nn.functional.conv2d(x, w, stride=sp["stride"], padding=(sp["kh"] - 1) // 2,
                                   groups=sp["C_in"] if sp["depthwise"] else 1)
    plain = np.mod(y.numpy().astype(np.int64), info.t)
    res["decrypt_last_layer"] = {"layer": index[i], "ciphertexts": int(out.shape[0]),
                                 "equal": bool((dec == plain).all())}
    res["bit_exact"] = bool(res["decrypt_last_layer"]["equal"] and
                            (res["oracle_samples"] is None or not res["oracle_samples"]["differ"]))
    return res


# 32x32 -> 64-bit multiply-adds (mad.wide.u32) per clock per SM on this GPU, measured by a
# throughput probe (eight independent dependent chains per thread, 2048 threads per SM, each
# multiply reading the previous result: 45.9 per SM per ns at 2070 MHz)
MAD_WIDE_PER_CLK_SM = 22.2
# mad.lo.u32 per clock per SM from the same probe (130.97 per SM per ns)
MAD_LO_PER_CLK_SM = 63.3
# wide-product equivalents per Shoup butterfly: a*w mod 2^64 and Q*q mod 2^64 (one wide product and
# two 32-bit products each, a 32-bit product costing MAD_WIDE / MAD_LO of a wide one) and the high
# half of a*w' (four wide products)
WIDE_PER_BUTTERFLY = 2 * (1 + 2 * MAD_WIDE_PER_CLK_SM / MAD_LO_PER_CLK_SM) + 4


def stage_rooflines(stages, counts, steps, peaks, N, sm_mhz=None):
    """The roofline of each stage kernel of the batched step, from its event-timed duration, in
    two views: Sec. 8(d)'s memory view (NTTs 16 N bytes per transform, the key switch its key
    stream plus the digit and c0 transforms it reads, against the measured HBM copy bandwidth)
    and the arithmetic view (the tensor-core MAC at 10 fp16 flops per modMAC -- five 10-bit chunks,
    one multiply-add each -- against the measured dense bf16 = fp16 tensor peak; the key switch at
    3 mad.wide per modMAC (Karatsuba products) and the NTTs at WIDE_PER_BUTTERFLY per butterfly,
    against the probed mad.wide rate x 152 SMs x the SM clock).  The view with the larger
    fraction is the binding one and is reported first."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    tc = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
    mhz = float(sm_mhz or peaks.get("sm_max_mhz", 2070.0))
    wide = MAD_WIDE_PER_CLK_SM * 152 * mhz * 1e6  # mad.wide per second
    out = {}
    for st, (ms, launches) in stages.items():
        if not launches:  # e.g. no key-switch launch when every layer's key switch is fused
            out[st] = None
            continue
        sec = ms / 1000 / max(1, steps)
        views = []
        if st in ("ntt_in", "ntt_out"):
            tr = counts[st + "_transforms"]
            views.append({"bound": "hbm", "algorithmic": tr * 16 * N, "unit": "GB/s", "peak": hbm, "scale": 1e9})
            views.append({"bound": "alu", "algorithmic": tr * (N // 2) * (N.bit_length() - 1), "unit": "Tbutterfly/s",
                          "peak": wide / WIDE_PER_BUTTERFLY / 1e12, "scale": 1e12})
        elif st == "keyswitch":
            views.append({"bound": "hbm", "algorithmic": counts["ks_bytes"], "unit": "GB/s", "peak": hbm, "scale": 1e9})
            views.append({"bound": "alu", "algorithmic": counts["ks_modmac_stage"], "unit": "TmodMAC/s",
                          "peak": wide / 3 / 1e12, "scale": 1e12})
        else:
            views.append({"bound": "tensor", "algorithmic": 10 * counts["conv_modmac"], "unit": "TFLOP/s", "peak": tc,
                          "scale": 1e12,
                          "fused_key_switch": {"key_and_digit_bytes": counts["mac_ks_bytes"],
                                               "modmac": counts["mac_ks_modmac"]}})
        for v in views:
            v["achieved"] = v["algorithmic"] / sec / v.pop("scale")
            v["frac"] = v["achieved"] / v["peak"]
        views.sort(key=lambda v: -v["frac"])
        r = dict(views[0])
        if len(views) > 1:
            r["other_view"] = views[1]
        r["ms_per_step"] = ms / max(1, steps)
        r["launches_per_step"] = launches / max(1, steps)
        out[st] = r
    return out


def run_gpu(args, rank, world):
    import torch

    from paper_2311_12519_gb300 import hyena as H

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    wl = args.workload
    ws_limit, workload = WORKLOADS[wl][0], workload_name(wl, args.packing)
    specs, n_ring, n_limbs, images = layer_specs(wl, args.layers, args.polyphase, args.dw_cn4)
    index = list(range(len(specs))) if args.layers is None else list(args.layers)
    if args.layers is not None:
        workload += f", layers {index} only"
    if args.polyphase:
        workload += ", 3x3 stride-2 layers with polyphase packing"
    if args.dw_cn4:
        workload += ", depthwise layers" + (" not so packed" if args.polyphase else "") + " with c_n=4"
    t_setup = time.perf_counter()
    p = H.he_params_create(n_ring, n_limbs, limb_bits=LIMB_BITS, decomp_bits=50)
    info = H.he_params_info(p)
    N, L, l = info.N, info.L, info.l
    sk = H.he_keygen(p, synth.SEED_KEYS)
    if args.packing == "fill":
        specs = fill_packing(specs, lambda x: (lambda o: (o.n_ct_in, o.n_ct_out))(H.he_layout_for_layer(p, H.conv_desc(**x))))
    tunes = [{} for _ in specs]
    if args.mac_impl or args.tc_cluster:
        # a forced MAC form or cluster size where the layer admits it (depthwise layers take no
        # tensor-core form; clusters need more than one row tile per CTA); the automatic form elsewhere
        p0 = H.he_params_create(n_ring, n_limbs, limb_bits=LIMB_BITS, decomp_bits=50)
        for i, s in enumerate(specs):
            d0, w0 = H.conv_desc(**s), synth.stack_inputs(wl, index[i], H.he_params_info(p0).t)[1]
            if args.mac_impl and H.he_conv_check(p0, d0, w0, mac_impl=args.mac_impl) == H.HE_OK:
                tunes[i]["mac_impl"] = args.mac_impl
            if args.tc_cluster and H.he_conv_check(p0, d0, w0, tc_cluster=args.tc_cluster, **tunes[i]) == H.HE_OK:
                tunes[i]["tc_cluster"] = args.tc_cluster
        H.he_params_destroy(p0)
    tuned = None
    if args.tuned:
        # per layer, the fastest packing, tile and MAC schedule on this ring, timed exhaustively
        from paper_2311_12519_gb300 import costmodel as CM

        rings = CM.Rings()
        rings.p[(N, L)] = p
        t_tune = time.perf_counter()
        tuned = []
        for i, s in enumerate(specs):
            shape = CM.Shape(s["C_in"], s["C_out"], s["H"], s["W"], s["kh"], s["stride"], s["depthwise"], images)
            best, best_ms, times = CM.autotune(rings, shape, CM.candidates(rings, shape, [(N, L)]))
            specs[i] = dict(s, c_n=best.c_n, tile_h=best.tile[0], tile_w=best.tile[1])
            tunes[i] = dict(mac_groups=best.mac_groups, mac_impl=best.mac_impl, tc_rows=best.tc_rows)
            default = times.get(CM.Config(N, L, 2, (0, 0), 1, 0, 0) if s["depthwise"] else
                                CM.Config(N, L, 2, (0, 0), 2, 96, 0))
            tuned.append({"layer": i, "c_n": best.c_n, "tile": list(best.tile), **tunes[i], "ms": round(best_ms, 4),
                          "default_ms": None if default is None else round(default, 4), "candidates": len(times)})
        rings.p = {}
        tune_s = time.perf_counter() - t_tune
    descs = [H.conv_desc(**s) for s in specs]
    gal = sorted(set(int(g) for d in descs for g in H.he_layer_galois(p, d)))
    gk = H.he_galois_keys(p, sk, gal, synth.SEED_KEYS)
    plans, d_ins, d_outs, h_ins, h_outs = [], [], [], [], []
    ws_max = 0
    counts = {"ks_bytes": 0, "ks_modmac_stage": 0, "mac_ks_bytes": 0, "mac_ks_modmac": 0}
    impls = []
    for i, (s, d) in enumerate(zip(specs, descs)):
        act, wt, enc_seed = rank_inputs(wl, index[i], rank, info.t)
        cts = H.he_encrypt_image(p, sk, d, act, enc_seed, info)
        plan = H.he_conv_plan(p, gk, d, wt, **tunes[i])
        n_in, n_out, ws = H.he_conv_sizes(plan)
        lay = H.he_layout_for_layer(p, d)
        lc = layer_counts(s, lay, L, l, N)
        impl = H.he_conv_info(plan)
        impls.append(impl)
        if impl == 6:  # the key switch runs inside the fused MAC kernel: its work is that stage's
            lc["mac_ks_bytes"], lc["mac_ks_modmac"] = lc.pop("ks_bytes"), lc.pop("ks_modmac_stage")
        for k, v in lc.items():
            counts[k] = counts.get(k, 0) + v
        plans.append(plan)
        h_ins.append(torch.from_numpy(cts.reshape(-1).view(np.int64)))
        h_outs.append(n_out)
        d_outs.append(torch.empty(n_out, dtype=torch.int64, device=dev))
        ws_max = max(ws_max, ws)
        del cts
    # the host buffers of all layers as views of one pinned allocation: with dozens of separately
    # pinned multi-GB tensors live at once, host-to-device copies from them ran at a quarter of the
    # link's rate on the GB300 machine (48 against 211 GB/s), from one allocation at the full rate
    n_words = sum(a.numel() for a in h_ins) + sum(h_outs)
    arena = torch.empty(n_words, dtype=torch.int64, pin_memory=True)
    off, views = 0, []
    for a in h_ins:
        arena[off:off + a.numel()].copy_(a)
        views.append(arena[off:off + a.numel()])
        off += a.numel()
    h_ins = views
    views = []
    for n in h_outs:
        views.append(arena[off:off + n])
        off += n
    h_outs = views
    d_ins = [a.to(dev) for a in h_ins]
    # the batch runs in waves under the workspace limit; the plain per-layer form shares its workspace
    batch = H.he_batch_create(plans) if ws_limit is None else H.he_batch_create_limited(plans, ws_limit)
    d_ws = torch.empty(max(ws_max, H.he_batch_workspace_bytes(batch)) // 8 + 1, dtype=torch.int64, device=dev)
    setup_s = time.perf_counter() - t_setup
    ins_p, outs_p = [a.data_ptr() for a in d_ins], [b.data_ptr() for b in d_outs]
    if args.mode == "batch":
        # profiler mode: per step one launch per stage and wave, nothing else on the GPU
        torch.cuda.synchronize()
        for _ in range(args.warmup + args.steps):
            H.he_batch_forward(batch, ins_p, outs_p, d_ws.data_ptr(), 0)
        torch.cuda.synchronize()
        for plan in plans:
            H.he_conv_status(plan)
        print(json.dumps({"mode": "batch", "workload": wl, "steps": args.steps, "warmup": args.warmup,
                          "layers": len(plans)}))
        return
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    n_layers = len(plans)
    sp = stream.cuda_stream
    warm = max(3, args.warmup)

    def step_plain():
        for plan, a, b in zip(plans, d_ins, d_outs):
            H.he_conv_forward(plan, a.data_ptr(), b.data_ptr(), d_ws.data_ptr(), sp)

    def step_batch():
        H.he_batch_graph_launch(batch, ins_p, outs_p, d_ws.data_ptr(), sp)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(fn):
        """W warm-up steps, then K steps with the L2 flushed before each (outside the events)."""
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for e0, e1 in ev:
                flush.zero_()
                e0.record(stream)
                fn()
                e1.record(stream)
            torch.cuda.synchronize()
            clk.keep_busy(lambda: (flush.zero_(), fn(), torch.cuda.synchronize()))
        barrier()
        return sum(e0.elapsed_time(e1) for e0, e1 in ev), clk.summary()

    with torch.cuda.stream(stream):
        # batched form (the headline): one launch per stage and wave, replayed as a CUDA graph
        ms, clocks_b = timed(step_batch)
        verified = verify_outputs(H, p, sk, info, wl, specs, descs, d_outs, rank, index)
        # plain per-layer form, with the per-stage event times of its launches
        H.he_profile_enable(True)
        H.he_profile_collect()
        ms_plain, clocks_p = timed(step_plain)
        H.he_profile_enable(False)
        H.he_profile_collect()
        # per-stage times of the batched form (events around each stage launch, same kernels)
        H.he_profile_enable(True)
        H.he_profile_collect()
        for _ in range(args.steps):
            flush.zero_()
            H.he_batch_forward(batch, ins_p, outs_p, d_ws.data_ptr(), sp)
        torch.cuda.synchronize()
        H.he_profile_enable(False)
        stages_b = H.he_profile_collect()
        # end to end through host buffers: the batch (he_batch_forward_host)
        for _ in range(2):
            H.he_batch_forward_host(batch, h_ins, h_outs, d_ins, d_outs, d_ws.data_ptr(), sp)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            H.he_batch_forward_host(batch, h_ins, h_outs, d_ins, d_outs, d_ws.data_ptr(), sp)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        barrier()
    for plan in plans:
        H.he_conv_status(plan)
    ms, ms_plain, e2e_s = reduce_max([ms, ms_plain, e2e_s], dev, world)
    if rank != 0:
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    roofs = stage_rooflines(stages_b, counts, args.steps, peaks, N, clocks_b.get("sm_mhz"))
    top = max(stages_b, key=lambda k: stages_b[k][0])
    # the kernels of each stage: he_conv_info 1 CUDA-core MAC, 3 eager, 4 tensor-core with in-kernel
    # conversion, 5 tensor-core on operand images, 6 fused key switch + tensor-core MAC, 7 operand
    # images on CTA pairs, 8 operand images in chunk passes
    mac_k = {1: "k_mac", 3: "k_mac_eager", 4: "k_mac_tc", 5: "k_mac_img", 6: "k_ksmac", 7: "k_mac_pair", 8: "k_mac_cp"}
    ks_k = {1: "k_keyswitch", 3: "k_keyswitch", 4: "k_keyswitch", 5: "k_keyswitch_img", 7: "k_keyswitch_img",
            8: "k_keyswitch_img"}
    kname = {"mac": " + ".join(sorted({mac_k[i] for i in impls})),
             "keyswitch": " + ".join(sorted({ks_k[i] for i in impls if i != 6})) or "none (fused)",
             "ntt_in": "k_ntt_inputs", "ntt_out": "k_intt"}
    top = max((k for k in stages_b if roofs[k]), key=lambda k: stages_b[k][0])
    roof = {k: v for k, v in roofs[top].items() if k in ("bound", "achieved", "peak", "unit", "frac")}
    src = kernel_source_digest().hexdigest()
    prof = PROFILED_TRAFFIC.get((workload, kname[top]))
    roof["traffic"] = prof[1] if prof and src.startswith(prof[0]) else None
    roof.update(kernel=kname[top], per_launch="one launch per stage and wave; achieved = algorithmic units of the "
                "step / the kernel's event-timed time in the step",
                peak_source={"GB/s": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                             "TFLOP/s": "MEASURED_PEAKS.json bf16_tflops_sustained, fp16 dense = bf16 dense (of measured)"}
                .get(roof["unit"], "derived: probed mad.wide rate %.1f/clk/SM x 152 SMs x SM clock %s MHz" % (
                    MAD_WIDE_PER_CLK_SM, clocks_b.get("sm_mhz"))))
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        layers = sorted({index[min(1, len(index) - 1)], index[-1]})
        threads = host_cores()
        est, spent, desc, parts = oracle_sample(wl, layers, threads, args.packing)
        # every layer of these stacks costs the oracle per input ciphertext and per term alike
        # (one ring, one rotation set per kernel size), so the sampled layers' unit costs give the
        # stack's layers/s over its own layer mix
        cpu = {"value": len(layers) / sum(est), "unit": "layers/s", "cores": threads, "kind": "oracle",
               "sample": desc, "sampled_layers": parts, "wall_seconds": round(spent, 1),
               "estimated_seconds_per_sampled_layer": [round(e, 1) for e in est]}
    line = {
        "metric": METRIC, "value": layers_per_second(world, n_layers, args.steps, ms / 1000), "unit": "layers/s",
        "n_gpus": world, "steps": args.steps, "warmup": warm, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload, "layers_per_step": n_layers, "images_per_gpu": images,
                   "batch_waves": H.he_batch_waves(batch),
                   "l2": "flushed before each timed step (256 MiB write)", "decomp_bits": info.w,
                   "parallelism": f"replicas x{world} (independent images, no collective)"},
        "modmac_per_s": (counts["conv_modmac"] + counts["ks_modmac"]) * world * args.steps / (ms / 1000),
        "modmac_per_step": {"conv": counts["conv_modmac"], "keyswitch": counts["ks_modmac"]},
        "e2e": {"value": layers_per_second(world, n_layers, args.steps, e2e_s), "unit": "layers/s",
                "h2d_bytes_per_step": counts["in_bytes"], "d2h_bytes_per_step": counts["out_bytes"],
                "call": "he_batch_forward_host (host buffers: views of one pinned allocation; copies and kernels in the timed region)"},
        "gpu_launches": int(sum(v[1] for v in stages_b.values()) // max(1, args.steps) * args.steps),
        "roofline": roof,
        "roofline_per_kernel": {kname[k]: v for k, v in roofs.items() if v},
        "cpu_baseline": cpu,
        "clocks": clocks_b,
        "verified": verified,
        "form": f"batched: one launch per stage for all {n_layers} layers of each of {H.he_batch_waves(batch)} "
                "workspace wave(s), replayed as a CUDA graph",
        "plain_per_layer": {"value": layers_per_second(world, n_layers, args.steps, ms_plain / 1000),
                            "unit": "layers/s", "ms_per_step": ms_plain / args.steps, "clocks": clocks_p},
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages_b.items()},
        "setup_seconds": round(setup_s, 1),
        "tuning": None if tuned is None else {"per_layer": tuned, "seconds": round(tune_s, 1),
                                              "method": "exhaustive timing of every packing x tile x schedule"},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ learned configuration
def run_learned(args):
    """The stack with every layer in the configuration the learned cost model picks (ring,
    packing, tile, MAC schedule; no timing of candidates), layers of one ring batched and
    replayed as CUDA graphs; a step runs every ring's batch once."""
    import torch

    from paper_2311_12519_gb300 import costmodel as CM
    from paper_2311_12519_gb300 import hyena as H

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    if not os.path.exists(CM.WEIGHTS):
        print(json.dumps({"mode": "learned", "unavailable": "no trained cost model weights in the package"}))
        return
    ws_limit, workload = WORKLOADS[args.workload]
    specs, _, _, images = layer_specs(args.workload)
    model = CM.CostModel.load(CM.WEIGHTS)
    rings = CM.Rings()
    t0 = time.perf_counter()
    shapes = [CM.Shape(s["C_in"], s["C_out"], s["H"], s["W"], s["kh"], s["stride"], s["depthwise"], images)
              for s in specs]
    picks = [CM.pick(rings, model, sh) for sh in shapes]
    pick_s = time.perf_counter() - t0
    groups = {}
    for i, c in enumerate(picks):
        groups.setdefault((c.N, c.L), []).append(i)
    batches, keep, checks = [], [], []
    for (N, L), idx in sorted(groups.items()):
        p = rings.get(N, L)
        info = H.he_params_info(p)
        sk = H.he_keygen(p, synth.SEED_KEYS)
        descs = {i: picks[i].desc(shapes[i]) for i in idx}
        gal = sorted(set(int(g) for d in descs.values() for g in H.he_layer_galois(p, d)))
        gk = H.he_galois_keys(p, sk, gal, synth.SEED_KEYS)
        plans, ins, outs = [], [], []
        for i in idx:
            s, c = specs[i], picks[i]
            act, wt, enc_seed = synth.stack_inputs(args.workload, i, info.t)
            cts = H.he_encrypt_image(p, sk, descs[i], act, enc_seed, info)
            plans.append(H.he_conv_plan(p, gk, descs[i], wt, mac_groups=c.mac_groups, mac_impl=c.mac_impl,
                                        tc_rows=c.tc_rows))
            ins.append(torch.from_numpy(cts.reshape(-1).view(np.int64)).to(dev))
            outs.append(torch.empty(H.he_conv_sizes(plans[-1])[1], dtype=torch.int64, device=dev))
        b = H.he_batch_create(plans) if ws_limit is None else H.he_batch_create_limited(plans, ws_limit)
        ws = torch.empty(H.he_batch_workspace_bytes(b) // 8 + 1, dtype=torch.int64, device=dev)
        batches.append((b, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], ws.data_ptr()))
        keep += [ins, outs, ws, plans, gk, sk]
        checks.append((p, sk, idx, descs, outs))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    def step():
        for b, i_p, o_p, w in batches:
            H.he_batch_graph_launch(b, i_p, o_p, w, sp)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with ClockSampler(0) as clk:
            for e0, e1 in ev:
                flush.zero_()
                e0.record(stream)
                step()
                e1.record(stream)
            torch.cuda.synchronize()
            clk.keep_busy(lambda: (flush.zero_(), step(), torch.cuda.synchronize()))
    for plan in [pl for k in keep[3::6] for pl in k]:
        H.he_conv_status(plan)
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / args.steps
    # every output of every layer, as the last timed step left it, decrypted and compared with the
    # plain convolution (float64 torch conv2d, exact at these sizes)
    decrypt_ok = []
    for p, sk, idx, descs, outs in checks:
        info = H.he_params_info(p)
        for i, o in zip(idx, outs):
            s = specs[i]
            act, wt, _ = synth.stack_inputs(args.workload, i, info.t)
            dec = H.he_decrypt_image(p, sk, descs[i], o.cpu().numpy().view(np.uint64).reshape(-1, 2, info.L, info.N))
            y = torch.nn.functional.conv2d(torch.from_numpy(act.astype(np.float64)),
                                           torch.from_numpy(wt.astype(np.float64)), stride=s["stride"],
                                           padding=(s["kh"] - 1) // 2, groups=s["C_in"] if s["depthwise"] else 1)
            decrypt_ok.append((i, bool((dec == np.mod(y.numpy().astype(np.int64), info.t)).all())))
    decrypt_ok.sort()
    print(json.dumps({
        "mode": "learned", "metric": METRIC,
        "decrypts_to_plain_conv": {"layers": len(decrypt_ok), "equal": sum(ok for _, ok in decrypt_ok),
                                   "differ": [i for i, ok in decrypt_ok if not ok]},
        "value": len(specs) * 1000.0 / ms, "unit": "layers/s", "ms_per_step": ms, "steps": args.steps,
        "workload": workload.split(", N=")[0] + ", ring, packing, tile and MAC schedule per layer by the cost model",
        "rings": {f"{N},{L}": len(idx) for (N, L), idx in sorted(groups.items())}, "pick_seconds": round(pick_s, 2),
        "picks": [dict(layer=i, N=c.N, L=c.L, c_n=c.c_n, tile=list(c.tile), mac_impl=c.mac_impl, tc_rows=c.tc_rows,
                       mac_groups=c.mac_groups) for i, c in enumerate(picks)],
        "clocks": clk.summary(), "l2": "flushed before each timed step (256 MiB write)"}), flush=True)


# ------------------------------------------------------------------ ablation
ABLATION = [
    # (name, counterpart in the paper's latency study, decomp_bits, c_n, mac_impl)
    ("eager, w=25", "Fig. latency (c): no latency optimisation", 25, 2, 3),
    ("eager, w=50", "Fig. latency (d): parameter selection only", 50, 2, 3),
    ("lazy CUDA-core, w=50", "Fig. latency (e): all optimisations", 50, 2, 1),
    ("lazy tensor-core, in-kernel fp16 conversion, w=50", "(e) on tcgen05, residues split into chunks by the MAC",
     50, 2, 4),
    ("lazy tensor-core, operand images, w=50", "(e) on tcgen05, operand images written by the key switch",
     50, 2, 5),
    ("lazy tensor-core, fused key switch, w=50", "(e) on tcgen05, key switch inside the MAC kernel", 50, 2, 6),
    ("lazy tensor-core, w=50", "(e) on tcgen05, the automatic form (in-kernel conversion for layers of one "
     "row tile, operand images for wider ones)", 50, 2, 2),
    ("lazy tensor-core, w=50, c_n=1", "padded convolution without output-channel packing (Sec. 2.4)", 50, 1, 2),
    ("lazy CUDA-core, w=50, c_n=4", "Sec. 3.1's 4 x 4 Walsh-Hadamard basis over row x slot-parity classes "
     "(compare with the c_n=2 CUDA-core row)", 50, 4, 1),
]


def conv_mod_t(act, wt, stride, t):
    """Plain 2-D convolution (zero padding 1, 3x3 taps) reduced mod t, for checking decryptions."""
    n, ci, h, w = act.shape
    x = np.pad(act.astype(np.int64), ((0, 0), (0, 0), (1, 1), (1, 1)))
    ho, wo = (h - 1) // stride + 1, (w - 1) // stride + 1
    out = np.zeros((n, wt.shape[0], ho, wo), dtype=np.int64)
    for dy in range(3):
        for dx in range(3):
            win = x[:, :, dy:dy + h:stride, dx:dx + w:stride][:, :, :ho, :wo]
            out += np.einsum("nchw,oc->nohw", win, wt[:, :, dy, dx].astype(np.int64))
    return out % t


def run_ablation(args):
    """Each row of ABLATION on the whole 19-layer stack in the batched graph form: ms per step,
    per-stage times, and the decryptions of every layer checked against the plain convolution;
    the MAC variants at the same w must also agree word for word."""
    import torch

    from paper_2311_12519_gb300 import hyena as H

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    specs, n_ring, n_limbs, _ = layer_specs("resnet20")
    words = {}
    for name, paper, w, c_n, impl in ABLATION:
        p = H.he_params_create(n_ring, n_limbs, limb_bits=LIMB_BITS, decomp_bits=w, est_mac_terms=64 * 9)
        info = H.he_params_info(p)
        sk = H.he_keygen(p, synth.SEED_KEYS)
        descs = [H.conv_desc(**dict(s, c_n=c_n)) for s in specs]
        gal = sorted(set(int(g) for d in descs for g in H.he_layer_galois(p, d)))
        gk = H.he_galois_keys(p, sk, gal, synth.SEED_KEYS)
        plans, d_ins, d_outs, acts, wts = [], [], [], [], []
        for i, (s, d) in enumerate(zip(specs, descs)):
            act = synth.activations((1, s["C_in"], s["H"], s["W"]), info.t, label=i)
            wt = synth.weights((s["C_out"], s["C_in"], s["kh"], s["kh"]), label=i)
            cts = H.he_encrypt_image(p, sk, d, act, synth.SEED_ENC, info)
            plan = H.he_conv_plan(p, gk, d, wt, mac_impl=impl)
            plans.append(plan)
            acts.append(act)
            wts.append(wt)
            d_ins.append(torch.from_numpy(cts.reshape(-1).view(np.int64)).to(dev))
            d_outs.append(torch.empty(H.he_conv_sizes(plan)[1], dtype=torch.int64, device=dev))
        batch = H.he_batch_create(plans)
        d_ws = torch.empty(H.he_batch_workspace_bytes(batch) // 8 + 1, dtype=torch.int64, device=dev)
        ins_p, outs_p = [a.data_ptr() for a in d_ins], [b.data_ptr() for b in d_outs]
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                H.he_batch_graph_launch(batch, ins_p, outs_p, d_ws.data_ptr(), sp)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            with ClockSampler(0) as clk:
                for e0, e1 in ev:
                    flush.zero_()
                    e0.record(stream)
                    H.he_batch_graph_launch(batch, ins_p, outs_p, d_ws.data_ptr(), sp)
                    e1.record(stream)
                torch.cuda.synchronize()
                clk.keep_busy(lambda: (flush.zero_(), H.he_batch_graph_launch(batch, ins_p, outs_p, d_ws.data_ptr(), sp),
                                       torch.cuda.synchronize()))
            ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / args.steps
            H.he_profile_enable(True)
            H.he_profile_collect()
            for _ in range(args.steps):
                flush.zero_()
                H.he_batch_forward(batch, ins_p, outs_p, d_ws.data_ptr(), sp)
            torch.cuda.synchronize()
            H.he_profile_enable(False)
            stages = H.he_profile_collect()
        decrypt_ok = True
        outs = []
        for d, s, act, wt, o in zip(descs, specs, acts, wts, d_outs):
            out = o.cpu().numpy().view(np.uint64)
            outs.append(out)
            dec = H.he_decrypt_image(p, sk, d, out.reshape(-1, 2, info.L, info.N))
            decrypt_ok &= bool(((dec - conv_mod_t(act, wt, s["stride"], info.t)) % info.t == 0).all())
        key = (w, c_n)
        same_words = None
        if key in words:
            same_words = all(np.array_equal(a, b) for a, b in zip(words[key], outs))
        else:
            words[key] = outs
        print(json.dumps({
            "ablation": name, "paper": paper, "decomp_bits": info.w, "c_n": c_n,
            "mac_impl": H.he_conv_info(plans[0]), "ms_per_step": ms, "layers_per_s": len(plans) * 1000 / ms,
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "est_noise_log2": info.est_noise_log2, "log2_delta": info.log2_delta,
            "decrypts_to_plain_conv": decrypt_ok, "words_equal_to_first_mac_form": same_words,
            "clocks": clk.summary(), "workload": WORKLOADS["resnet20"][1].replace("c_n=2", f"c_n={c_n}")}), flush=True)
        H.he_batch_destroy(batch)
        for plan in plans:
            H.he_plan_destroy(plan)
        H.he_galkeys_destroy(gk)
        H.he_seckey_destroy(sk)
        H.he_params_destroy(p)
        del d_ins, d_outs, d_ws
        torch.cuda.empty_cache()


# ------------------------------------------------------------------ tensor-core forms per layer
def run_forms(args):
    """Every layer of the stack timed alone (he_conv_time: uniform residues, median of `steps`
    forwards) in each tensor-core form it admits (4 in-kernel conversion, 5 operand images, 6 fused
    key switch) and with the automatic choice: one JSON line per layer with per-stage ms."""
    import torch

    from paper_2311_12519_gb300 import hyena as H

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    specs, N, L, images = layer_specs(args.workload, args.layers, args.polyphase, args.dw_cn4)
    index = list(range(len(specs))) if args.layers is None else list(args.layers)
    p = H.he_params_create(N, L, limb_bits=LIMB_BITS, decomp_bits=50)
    for i, s in zip(index, specs):
        d = H.conv_desc(**s)
        _, wt, _ = synth.stack_inputs(args.workload, i, H.he_params_info(p).t)
        row = {"mode": "forms", "workload": args.workload, "layer": i}
        for impl in (0, 4, 5, 6, 7, 8):
            try:
                total, stages = H.he_conv_time(p, d, wt, mac_impl=impl, reps=max(3, args.steps),
                                               stream=stream.cuda_stream)
                row[str(impl)] = {"ms": round(total, 4), "stages": [round(x, 4) for x in stages]}
            except H.HyenaError as e:
                row[str(impl)] = {"unavailable": str(e).split(": ", 1)[-1][:80]}
        print(json.dumps(row), flush=True)
    H.he_params_destroy(p)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hyena", choices=["hyena", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS),
                    help="the headline VGG-16 stack (8 images), or the ResNet-20 (1 image) or MobileNetV1 "
                         "(32 images) stack")
    ap.add_argument("--polyphase", action="store_true",
                    help="pack the 3x3 stride-2 layers' inputs as phase planes (stride-1 layers on them)")
    ap.add_argument("--packing", default="fill", choices=["fill", "2"],
                    help="c_n of the stack layers: 'fill' packs a layer (c_n = 2) only where its tiles leave "
                         "slot rows empty and runs the others unpacked (c_n = 1); '2' packs every layer")
    ap.add_argument("--dw-cn4", action="store_true",
                    help="pack the depthwise layers (those not packed as phase planes) four channels per "
                         "ciphertext (c_n = 4)")
    ap.add_argument("--tc-cluster", type=int, default=0,
                    help="run the image-form MAC of layers wider than one row tile in clusters of this many CTAs")
    ap.add_argument("--mac-impl", type=int, default=0,
                    help="force the MAC form of every layer that admits it (he_tune.mac_impl; 0 = automatic per layer)")
    ap.add_argument("--layers", type=lambda v: [int(x) for x in v.split(",")], default=None,
                    help="run only these layer indices of the stack (comma list), e.g. for profiler captures")
    ap.add_argument("--tuned", action="store_true",
                    help="pick each layer's packing, tile and MAC schedule by timing every candidate first")
    ap.add_argument("--mode", default="full", choices=["full", "batch", "ablation", "learned", "forms"],
                    help="batch: only the batched forward, W + K times, no JSON (for profiler captures); "
                         "ablation: one JSON line per variant of the latency study (reduction, w, c_n, MAC unit); "
                         "learned: every layer in the configuration the trained cost model picks")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.mode == "ablation":
        if rank == 0:
            run_ablation(args)
        return
    if args.mode == "learned":
        if rank == 0:
            run_learned(args)
        return
    if args.mode == "forms":
        if rank == 0:
            run_forms(args)
        return
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl")
    try:
        run_gpu(args, rank, world)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
