"""Throughput of encrypted convolution on the GB300 (one JSON line on stdout).

Workload: the 19 3x3 convolutions of a ResNet-20 on 32x32 inputs, one image
per GPU, N = 8192, L = 3 RNS limbs of 50 bits, t = 1032193, Hyena packing
(c_n = 2).  A step runs all 19 layers once on fresh synthetic ciphertexts
resident in HBM.  value = layers/s over all ranks of the batched form (one
launch per stage for all layers, replayed as a CUDA graph); the plain
per-layer form (he_conv_forward per layer) is reported beside it, with
modMAC/s.  e2e repeats the step from pinned host buffers through
he_batch_forward_host (copies inside the timed region; layer by layer through
he_conv_forward_host beside it).  --workload vgg16|mobilenet
measures the VGG-16 (8 images, N = 16384) or MobileNetV1 (32 images) stack
the same way; --mode ablation prints one line per variant of the latency
study; --impl reference times the CPU oracle instead.

Launch: python bench.py [--gpus N --steps K --warmup W]; N > 1 under
torch.distributed.run (one process per GPU, no collective on the data path).
"""
from __future__ import annotations

import argparse
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

N_RING, L_LIMBS, LIMB_BITS = 8192, 3, 50
WORKLOAD = "resnet20-3x3-stack, 32x32, 1 image/GPU, N=8192, L=3x50-bit, t=1032193, c_n=2"
# other stacks (not the headline): name -> (shapes, N, L, images per GPU, batch workspace limit, description)
WORKLOADS = {
    "resnet20": (synth.resnet20_convs, N_RING, L_LIMBS, 1, None, WORKLOAD),
    "vgg16": (synth.vgg16_convs, 16384, 4, 8, 64 << 30,
              "vgg16-3x3-stack, 224x224, 8 images/GPU, N=16384, L=4x50-bit, t=786433, c_n=2"),
    "mobilenet": (synth.mobilenet_v1_convs, 8192, 4, 32, 64 << 30,
                  "mobilenetv1-dw+pw-stack, 224x224, 32 images/GPU, N=8192, L=4x50-bit, t=1032193, c_n=2"),
}
METRIC = "HE-conv layers/s (ResNet-20 stack, bit-exact)"
L2_BYTES = 129 * 2**20
# DRAM bytes (read + write) of one launch of each kernel of the batched step, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel source with this digest prefix
# (kernel_source_digest); reported as roofline traffic only while the kernels are unchanged
PROFILED_TRAFFIC = {"source": "6a8f6476f848e201", "k_keyswitch": 2.715e9, "k_mac_tc": 2.358e9, "k_ntt_inputs": 0.381e9,
                    "k_intt": 0.223e9}


def kernel_source_digest():
    """sha256 of device.cu up to its device-table section, without comments and blank space: the
    kernels and their launch code, which fix what a profiled launch does (the host API below them
    does not)."""
    import hashlib
    import re

    text = open(os.path.join(ROOT, "paper_2311_12519_gb300", "csrc", "device.cu"), "rb").read()
    cut = text.find(b"// ================================================================== device tables")
    code = re.sub(rb"//[^\n]*", b"", text[:cut] if cut > 0 else text)
    return hashlib.sha256(re.sub(rb"\s+", b" ", code))


def layer_descs(workload="resnet20"):
    shapes, _, _, images, _, _ = WORKLOADS[workload]
    return [dict(C_in=s.C_in, C_out=s.C_out, H=s.H, W=s.W, kh=s.k, stride=s.stride, depthwise=s.depthwise,
                 n_images=images, c_n=2) for s in shapes()]


def modmacs(spec, lay, n_rot, L, l, N):
    """Algorithmic modular multiply-accumulates of one layer (conv MAC + key switch)."""
    K = n_rot if spec["depthwise"] else lay.in_groups * n_rot
    conv = lay.row_units * lay.out_groups * (2 if spec["c_n"] == 2 else 1) * K * 2 * L * N
    ks = lay.n_ct_in * lay.n_galois * 2 * L * l * L * N
    return conv, ks


# ------------------------------------------------------------------ ranks
def rank_inputs(rank):
    """Per-rank workload: rank r encrypts its own image (activation labels and
    encryption seed depend on r); weights and keys are shared by all ranks."""
    return {"act_label": 1000 * rank, "enc_seed": synth.SEED_ENC + 7919 * rank}


def reduce_max(values, device, world):
    """Max over ranks of the timed values (barrier + max timing; no data-path collective)."""
    if world <= 1:
        return list(values)
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def layers_per_second(world, n_layers, steps, seconds):
    """Whole-job throughput: every rank runs n_layers layers per step on its own image."""
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
def oracle_sample(reps=1):
    """The CPU oracle on one whole layer of the stack (16 -> 16 channels, 32x32):
    returns (seconds per layer, description).  Single-threaded."""
    from oracle import bfv, conv
    from oracle import params as prm

    P = prm.make_params(N=N_RING, L=L_LIMBS, w=50)
    spec = layer_descs()[1]
    lay = conv.Layout(N=N_RING, **spec)
    s = bfv.keygen(P, synth.SEED_KEYS)
    ksk = {g: bfv.galois_key(P, s, g, synth.SEED_KEYS) for g in conv.galois_elements(P, lay)}
    act = synth.activations((1, spec["C_in"], spec["H"], spec["W"]), P.t, label=1)
    wt = synth.weights((spec["C_out"], spec["C_in"], 3, 3), label=1)
    cts = conv.encrypt_image(P, lay, s, act, synth.SEED_ENC)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        conv.he_conv(P, lay, wt, cts, ksk)
        times.append(time.perf_counter() - t0)
    return times, "one whole ResNet-20 layer (16->16 channels, 32x32, N=8192, L=3) per step, 1 thread"


def run_reference(args, rank):
    if rank != 0:
        return
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    times, desc = oracle_sample(reps=steps + warm)
    t = sum(times[warm:])
    value = steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "layers/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1000 * t / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "layers/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world):
    import torch

    from paper_2311_12519_gb300 import hyena as H

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    _, n_ring, n_limbs, images, ws_limit, workload = WORKLOADS[args.workload]
    specs = layer_descs(args.workload)
    k_max = max(s["kh"] ** 2 * (1 if s["depthwise"] else s["C_in"]) for s in specs)
    p = H.he_params_create(n_ring, n_limbs, limb_bits=LIMB_BITS, decomp_bits=0, est_mac_terms=k_max)
    info = H.he_params_info(p)
    N, L, l = info.N, info.L, info.l
    sk = H.he_keygen(p, synth.SEED_KEYS)
    tunes = [{} for _ in specs]
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
            # the untuned plan: packing 2, default tile, tensor core with 96 rows (CUDA cores if depthwise)
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
    ws_max, conv_mm, ks_mm, in_bytes, out_bytes = 0, 0, 0, 0, 0
    stage_bytes = {"ntt_in": 0, "keyswitch": 0, "mac": 0, "ntt_out": 0}
    for i, (s, d) in enumerate(zip(specs, descs)):
        ri = rank_inputs(rank)
        act = synth.activations((images, s["C_in"], s["H"], s["W"]), info.t, label=i + ri["act_label"])
        wt = synth.weights((s["C_out"], 1 if s["depthwise"] else s["C_in"], s["kh"], s["kh"]), label=i)
        cts = H.he_encrypt_image(p, sk, d, act, ri["enc_seed"], info)
        plan = H.he_conv_plan(p, gk, d, wt, **tunes[i])
        n_in, n_out, ws = H.he_conv_sizes(plan)
        lay = H.he_layout_for_layer(p, d)
        n_rot = s["kh"] ** 2 * (2 if s["c_n"] == 2 and not s["depthwise"] else 1)
        cm, km = modmacs(s, lay, n_rot, L, l, N)
        conv_mm += cm
        ks_mm += km
        ctb = 2 * L * N * 8
        # algorithmic bytes of each stage (one read of every input, one write of every output)
        stage_bytes["ntt_in"] += lay.n_ct_in * ctb + lay.n_ct_in * (2 * L + L * l * L) * N * 8
        # minimum: rotated copies written once, digit NTTs, NTT(c0) and keys read once
        stage_bytes["keyswitch"] += (lay.n_ct_in * lay.n_galois * ctb + lay.n_ct_in * (L * l * L + L) * N * 8
                                     + lay.n_galois * L * l * 2 * L * N * 8)
        stage_bytes["mac"] += lay.n_ct_in * n_rot * ctb + lay.n_ct_out * ctb
        stage_bytes["ntt_out"] += 2 * lay.n_ct_out * ctb
        plans.append(plan)
        h_in = torch.from_numpy(cts.reshape(-1).view(np.int64)).pin_memory()
        h_ins.append(h_in)
        h_outs.append(torch.empty(n_out, dtype=torch.int64).pin_memory())
        d_ins.append(h_in.to(dev))
        d_outs.append(torch.empty(n_out, dtype=torch.int64, device=dev))
        ws_max = max(ws_max, ws)
        in_bytes += n_in * 8
        out_bytes += n_out * 8
    # the batch runs in waves under the workspace limit; the plain per-layer form shares its workspace
    batch = H.he_batch_create(plans) if ws_limit is None else H.he_batch_create_limited(plans, ws_limit)
    d_ws = torch.empty(max(ws_max, H.he_batch_workspace_bytes(batch)) // 8 + 1, dtype=torch.int64, device=dev)
    d_wsb = d_ws
    if args.mode == "batch":
        # profiler mode: per step one launch per stage and wave, nothing else on the GPU
        ins_p, outs_p = [a.data_ptr() for a in d_ins], [b.data_ptr() for b in d_outs]
        torch.cuda.synchronize()
        for _ in range(args.warmup + args.steps):
            H.he_batch_forward(batch, ins_p, outs_p, d_wsb.data_ptr(), 0)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "batch", "steps": args.steps, "warmup": args.warmup, "layers": len(plans)}))
        return
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    n_layers = len(plans)
    sp = stream.cuda_stream

    def step():
        for plan, a, b in zip(plans, d_ins, d_outs):
            H.he_conv_forward(plan, a.data_ptr(), b.data_ptr(), d_ws.data_ptr(), sp)

    def step_host():
        for plan, a, b, ha, hb in zip(plans, d_ins, d_outs, h_ins, h_outs):
            H.he_conv_forward_host(plan, ha.data_ptr(), hb.data_ptr(), a.data_ptr(), b.data_ptr(), d_ws.data_ptr(),
                                   sp)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        # timed region: K steps, L2 flushed before each (outside the events)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        H.he_profile_enable(True)
        H.he_profile_collect()
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for e0, e1 in ev:
                flush.zero_()
                e0.record(stream)
                step()
                e1.record(stream)
            torch.cuda.synchronize()
            clk.keep_busy(lambda: (flush.zero_(), step(), torch.cuda.synchronize()))
        barrier()
        H.he_profile_enable(False)
        stages = H.he_profile_collect()
        ms_plain = sum(e0.elapsed_time(e1) for e0, e1 in ev)
        # batched form: one launch per stage for all layers, replayed as a CUDA graph
        ins_p, outs_p = [a.data_ptr() for a in d_ins], [b.data_ptr() for b in d_outs]

        def step_batch():
            H.he_batch_graph_launch(batch, ins_p, outs_p, d_wsb.data_ptr(), sp)

        for _ in range(max(3, args.warmup)):
            step_batch()
        torch.cuda.synchronize()
        evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk_b:
            for e0, e1 in evb:
                flush.zero_()
                e0.record(stream)
                step_batch()
                e1.record(stream)
            torch.cuda.synchronize()
            clk_b.keep_busy(lambda: (flush.zero_(), step_batch(), torch.cuda.synchronize()))
        barrier()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evb)
        # per-stage times of the batched form (events around each stage launch)
        H.he_profile_enable(True)
        H.he_profile_collect()
        for _ in range(args.steps):
            flush.zero_()
            H.he_batch_forward(batch, ins_p, outs_p, d_wsb.data_ptr(), sp)
        torch.cuda.synchronize()
        H.he_profile_enable(False)
        stages_b = H.he_profile_collect()
        # end to end through host buffers: the batch (he_batch_forward_host), and layer by layer
        def step_host_batch():
            H.he_batch_forward_host(batch, h_ins, h_outs, d_ins, d_outs, d_wsb.data_ptr(), sp)

        e2e = {}
        for name, fn in (("batch", step_host_batch), ("plain", step_host)):
            for _ in range(2):
                fn()
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                fn()
            torch.cuda.synchronize()
            e2e[name] = time.perf_counter() - t0
            barrier()
        e2e_s, e2e_plain_s = e2e["batch"], e2e["plain"]
    ms, ms_plain, e2e_s, e2e_plain_s = reduce_max([ms, ms_plain, e2e_s, e2e_plain_s], dev, world)
    if rank != 0:
        return
    ms_step = ms / args.steps
    layers_per_s = layers_per_second(world, n_layers, args.steps, ms / 1000)
    # dominant stage and its roofline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    top = max(stages_b, key=lambda k: stages_b[k][0])
    top_ms, top_launches = stages_b[top]
    per_launch_s = top_ms / 1000 / max(1, top_launches)
    mac_tc = all(H.he_conv_info(pl) == 2 for pl in plans)
    if top == "mac" and mac_tc:
        # tensor-core contraction: 10 fp16 flops per modMAC would put it at a few % of the tensor roof;
        # the binding roof is HBM (every rotated residue read once, every output written once)
        achieved = stage_bytes["mac"] * args.steps / (top_ms / 1000) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": "k_mac_tc", "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "tensor_tflops_equiv": 10 * conv_mm * args.steps / (top_ms / 1000) / 1e12}
    elif top == "mac":
        # CUDA-core integer roof: 2 IMAD.WIDE per modMAC, 64 IMAD lanes per SM per clock issue
        # at half rate for the 64-bit wide form -> 32 wide products per SM per clock
        alu_peak = 152 * 2.07e9 * 32 / 2 / 1e12  # TmodMAC/s
        achieved = conv_mm * args.steps / (top_ms / 1000) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TmodMAC/s",
                "frac": achieved / alu_peak, "traffic": None, "kernel": "k_mac",
                "peak_source": "derived: 152 SMs x 2070 MHz x 32 IMAD.WIDE/clk/SM / 2 per modMAC"}
    else:
        achieved = stage_bytes[top] * args.steps / (top_ms / 1000) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": top, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    roof["ms_per_launch"] = per_launch_s * 1000
    src = kernel_source_digest()
    kname = {"mac": "k_mac_tc" if mac_tc else "k_mac", "keyswitch": "k_keyswitch", "ntt_in": "k_ntt_inputs",
             "ntt_out": "k_intt"}[top]
    if (src.hexdigest().startswith(PROFILED_TRAFFIC["source"]) and kname in PROFILED_TRAFFIC
            and args.workload == "resnet20"):
        roof["traffic"] = PROFILED_TRAFFIC[kname]
    roof["kernel"] = kname
    roof["stage_share"] = {k: round(v[0] / max(1e-9, sum(x[0] for x in stages_b.values())), 4)
                           for k, v in stages_b.items()}
    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.workload == "resnet20":
        times, desc = oracle_sample(reps=1)
        cpu = {"value": 1.0 / times[0], "unit": "layers/s", "cores": 1, "kind": "oracle", "sample": desc}
    line = {
        "metric": METRIC if args.workload == "resnet20" else METRIC.replace("ResNet-20", args.workload),
        "value": layers_per_s, "unit": "layers/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload, "layers_per_step": n_layers, "images_per_gpu": images,
                   "batch_waves": H.he_batch_waves(batch),
                   "l2": "flushed before each timed step (256 MiB write)", "decomp_bits": info.w,
                   "parallelism": f"replicas x{world} (independent images, no collective)"},
        "modmac_per_s": (conv_mm + ks_mm) * world * args.steps / (ms / 1000),
        "modmac_per_step": {"conv": conv_mm, "keyswitch": ks_mm},
        "e2e": {"value": layers_per_second(world, n_layers, args.steps, e2e_s), "unit": "layers/s",
                "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": out_bytes,
                "call": "he_batch_forward_host (pinned host buffers, copies and graph replay in the timed region)",
                "plain_per_layer": layers_per_second(world, n_layers, args.steps, e2e_plain_s)},
        "gpu_launches": sum(v[1] for v in stages_b.values()),
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk_b.summary(),
        "form": f"batched: one launch per stage for all {n_layers} layers of each of {H.he_batch_waves(batch)} "
                "workspace wave(s), replayed as a CUDA graph",
        "plain_per_layer": {"value": layers_per_second(world, n_layers, args.steps, ms_plain / 1000),
                            "unit": "layers/s", "ms_per_step": ms_plain / args.steps,
                            "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
                            "clocks": clk.summary()},
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages_b.items()},
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
    _, n_ring, n_limbs, images, ws_limit, workload = WORKLOADS[args.workload]
    specs = layer_descs(args.workload)
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
    batches, keep = [], []
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
            act = synth.activations((images, s["C_in"], s["H"], s["W"]), info.t, label=i)
            wt = synth.weights((s["C_out"], 1 if s["depthwise"] else s["C_in"], s["kh"], s["kh"]), label=i)
            cts = H.he_encrypt_image(p, sk, descs[i], act, synth.SEED_ENC, info)
            plans.append(H.he_conv_plan(p, gk, descs[i], wt, mac_groups=c.mac_groups, mac_impl=c.mac_impl,
                                        tc_rows=c.tc_rows))
            ins.append(torch.from_numpy(cts.reshape(-1).view(np.int64)).to(dev))
            outs.append(torch.empty(H.he_conv_sizes(plans[-1])[1], dtype=torch.int64, device=dev))
        b = H.he_batch_create(plans) if ws_limit is None else H.he_batch_create_limited(plans, ws_limit)
        ws = torch.empty(H.he_batch_workspace_bytes(b) // 8 + 1, dtype=torch.int64, device=dev)
        batches.append((b, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], ws.data_ptr()))
        keep += [ins, outs, ws, plans, gk, sk]
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
    print(json.dumps({
        "mode": "learned", "metric": METRIC if args.workload == "resnet20" else METRIC.replace("ResNet-20", args.workload),
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
    ("lazy tensor-core, w=50", "(e) with the contraction on tcgen05 (the default form)", 50, 2, 2),
    ("lazy tensor-core, w=50, c_n=1", "padded convolution without output-channel packing (Sec. 2.4)", 50, 1, 2),
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
    specs = layer_descs()
    words = {}
    for name, paper, w, c_n, impl in ABLATION:
        p = H.he_params_create(N_RING, L_LIMBS, limb_bits=LIMB_BITS, decomp_bits=w, est_mac_terms=64 * 9)
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
            "clocks": clk.summary(), "workload": WORKLOAD.replace("c_n=2", f"c_n={c_n}")}), flush=True)
        H.he_batch_destroy(batch)
        for plan in plans:
            H.he_plan_destroy(plan)
        H.he_galkeys_destroy(gk)
        H.he_seckey_destroy(sk)
        H.he_params_destroy(p)
        del d_ins, d_outs, d_ws
        torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hyena", choices=["hyena", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="resnet20", choices=sorted(WORKLOADS),
                    help="the headline ResNet-20 stack, or the VGG-16 (8 images) or MobileNetV1 (32 images) stack")
    ap.add_argument("--tuned", action="store_true",
                    help="pick each layer's packing, tile and MAC schedule by timing every candidate first")
    ap.add_argument("--mode", default="full", choices=["full", "batch", "ablation", "learned"],
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
