"""Autotuner and learned cost model for encrypted convolution layers.

A layer configuration is a ring (N, L limbs of 50 bits), a packing c_n, an
interior tile shape and a MAC schedule (tensor-core rows per CTA, or the
CUDA-core MAC's group tile).  Every configuration computes exact results; they
differ only in time.  The paper fixes its parameters by the noise analysis of
Sec. 3.2.1 (N by input size, Sec. 4.1); here the noise estimate only decides
which configurations are admissible, and time decides between them:

  * autotune(): the exhaustive search, timing every admissible configuration
    of a layer on the GPU through he_conv_time (the fallback, and the yardstick the model is scored against);
  * CostModel: the perceptron of hyena_costmodel.h, trained on kernel
    latencies (four stages per timed layer) of random layers, which ranks the
    same configurations without running them.

Command line (GPU):
  python -m paper_2311_12519_gb300.costmodel --samples 5000 --out DIR
collects the training latencies, trains the model, and evaluates it on the
ResNet-20, VGG-16 and MobileNetV1 stacks: per layer the model's pick against
the exhaustive optimum (regret) and against the default configuration, with a
JSON report in DIR.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import hyena as H

STAGES = ("ntt_in", "keyswitch", "mac", "ntt_out")
# (N, L) rings with q = L 50-bit primes inside the 128-bit-security bound on log q
# (109, 218 and 438 bits for N = 4096, 8192, 16384)
TRAIN_RINGS = [(4096, 2), (8192, 2), (8192, 3), (8192, 4), (16384, 2), (16384, 3), (16384, 4), (16384, 5),
               (16384, 6)]
SELECT_RINGS = [(4096, 2), (8192, 3), (16384, 4)]
TC_ROWS = (32, 64, 96)
MAC_GROUPS = (4, 8)


@dataclass(frozen=True)
class Shape:
    C_in: int
    C_out: int
    H: int
    W: int
    k: int = 3
    stride: int = 1
    depthwise: bool = False
    n_images: int = 1


@dataclass(frozen=True)
class Config:
    N: int
    L: int
    c_n: int
    tile: tuple      # (tile_h, tile_w); (0, 0) = the library's default
    mac_impl: int    # 1 CUDA-core, 2 tensor-core
    tc_rows: int = 0
    mac_groups: int = 0

    def desc(self, s: Shape):
        return H.conv_desc(s.C_in, s.C_out, s.H, s.W, s.k, s.stride, s.depthwise, s.n_images, self.c_n,
                           self.tile[0], self.tile[1])


def timing_weights(s: Shape, seed: int = 4) -> np.ndarray:
    """Integer weights in [-8, 8] (the value range decides only the tensor-core exactness test)."""
    rng = np.random.default_rng(seed)
    return rng.integers(-8, 9, (s.C_out, 1 if s.depthwise else s.C_in, s.k, s.k)).astype(np.int32)


class Rings:
    """he_params per (N, L), made once (automatic decomposition base for the largest layer)."""

    def __init__(self):
        self.p = {}

    def get(self, N, L):
        if (N, L) not in self.p:
            self.p[(N, L)] = H.he_params_create(N, L, decomp_bits=0, est_mac_terms=1024 * 9)
        return self.p[(N, L)]

    def close(self):
        for p in self.p.values():
            H.he_params_destroy(p)
        self.p = {}


def tile_candidates(N: int, s: Shape) -> list:
    """The default tile and up to two alternatives: full-width strips half as tall as fit, and
    square tiles half as wide as the default, each kept only if valid and different."""
    half, P, S = N // 2, (s.k - 1) // 2, s.stride
    out = [(0, 0)]

    def ok(th, tw):
        return (0 < th <= s.H and 0 < tw <= s.W and (th % S == 0 or th == s.H) and (tw % S == 0 or tw == s.W)
                and (th + 2 * P) * (tw + 2 * P) <= half)

    th = ((half // 2) // (s.W + 2 * P) - 2 * P) // S * S
    if ok(th, s.W) and th < s.H:
        out.append((th, s.W))
    side = int(math.isqrt(half)) - 2 * P
    side = max(S, (side // 2) // S * S)
    if ok(min(side, s.H), min(side, s.W)) and (min(side, s.H), min(side, s.W)) not in out:
        out.append((min(side, s.H), min(side, s.W)))
    return out


def schedules(s: Shape) -> list:
    if s.depthwise:
        return [(1, 0, 0)]
    return [(2, r, 0) for r in TC_ROWS] + [(1, 0, g) for g in MAC_GROUPS]


def candidates(rings: "Rings", s: Shape, ring_list=SELECT_RINGS) -> list:
    """Admissible layouts x schedules; tiles that come out as the same layout are kept once."""
    out = []
    for N, L in ring_list:
        for c_n in (2, 1):
            seen = set()
            for tile in tile_candidates(N, s):
                c0 = Config(N, L, c_n, tile, 1)
                try:
                    lay = H.he_layout_for_layer(rings.get(N, L), c0.desc(s))
                except H.HyenaError:
                    continue
                if (lay.T_h, lay.T_w) in seen:
                    continue
                seen.add((lay.T_h, lay.T_w))
                for impl, rows, groups in schedules(s):
                    out.append(Config(N, L, c_n, tile, impl, rows, groups))
    return out


def default_config(s: Shape, N: int, L: int) -> Config:
    """What the library picks without tuning: Hyena packing, default tile, automatic MAC."""
    return Config(N, L, 2, (0, 0), 0)


# ------------------------------------------------------------------ features
N_FEATURES = 28


def _lg(x):
    return math.log2(max(1.0, float(x)))


def features(rings: Rings, s: Shape, c: Config) -> np.ndarray | None:
    """Per-stage feature rows [4][N_FEATURES], or None if the layout is invalid."""
    p = rings.get(c.N, c.L)
    info = H.he_params_info(p)
    try:
        lay = H.he_layout_for_layer(p, c.desc(s))
    except H.HyenaError:
        return None
    N, L, l = c.N, c.L, info.l
    n_rot = s.k * s.k * (2 if (c.c_n == 2 and not s.depthwise) else 1)
    K = n_rot if s.depthwise else lay.in_groups * n_rot
    logN = math.log2(N)
    work = [lay.n_ct_in * (L + L * l * L) * N * logN,                      # input NTT butterflies
            lay.n_ct_in * lay.n_galois * 2 * L * l * L * N,                 # key-switch products
            lay.row_units * lay.out_groups * c.c_n * K * 2 * L * N,         # MAC terms
            lay.n_ct_out * 2 * L * N * logN]                                # output NTT butterflies
    byts = [lay.n_ct_in * (2 + L * l) * L * N * 8,
            lay.n_ct_in * lay.n_galois * 2 * L * N * 8 + lay.n_galois * L * l * 2 * L * N * 8,
            lay.n_ct_in * n_rot * 2 * L * N * 8,
            lay.n_ct_out * 4 * L * N * 8]
    base = [logN, L, l, c.c_n, float(s.depthwise), s.k, s.stride, _lg(s.C_in), _lg(s.C_out), _lg(s.H), _lg(s.W),
            _lg(s.n_images), _lg(lay.T_h), _lg(lay.T_w), _lg(lay.n_ct_in), _lg(lay.n_ct_out), _lg(lay.row_units),
            n_rot, lay.n_galois, _lg(K), float(c.mac_impl == 2), _lg(c.tc_rows or 96) if c.mac_impl != 1 else 0.0,
            _lg(c.mac_groups or 8) if c.mac_impl == 1 else 0.0]
    rows = []
    for i in range(4):
        onehot = [1.0 if j == i else 0.0 for j in range(4)]
        rows.append(base + [_lg(work[i]), _lg(byts[i])] + onehot[:3])
    X = np.array(rows, dtype=np.float32)
    assert X.shape[1] == N_FEATURES
    return X


# ------------------------------------------------------------------ measurement
def measure(rings: Rings, s: Shape, c: Config, reps: int = 2):
    """(total ms, per-stage ms) of one forward, or None if the configuration is not admissible
    (invalid layout, noise budget exceeded, tensor core not exact, or out of device memory)."""
    p = rings.get(c.N, c.L)
    try:
        return H.he_conv_time(p, c.desc(s), timing_weights(s), mac_groups=c.mac_groups, mac_impl=c.mac_impl,
                              tc_rows=c.tc_rows, reps=reps)
    except H.HyenaError as e:
        if e.code in (H.HE_EINVAL, H.HE_ENOISE, H.HE_ENOMEM):
            return None
        raise


def workspace_gb(rings: Rings, s: Shape, c: Config) -> float:
    p = rings.get(c.N, c.L)
    lay = H.he_layout_for_layer(p, c.desc(s))
    n_rot = s.k * s.k * (2 if (c.c_n == 2 and not s.depthwise) else 1)
    return (lay.n_ct_in * (n_rot + 1) + lay.n_ct_out * 2) * 2 * c.L * c.N * 8 / 1e9


def random_shape(rng) -> Shape:
    dw = rng.random() < 0.2
    k = 3 if dw else int(rng.choice([1, 3], p=[0.3, 0.7]))
    c_in = int(round(2 ** rng.uniform(math.log2(3), 10)))
    c_out = c_in if dw else int(round(2 ** rng.uniform(math.log2(3), 10)))
    hw = int(round(2 ** rng.uniform(math.log2(7), math.log2(224))))
    return Shape(c_in, c_out, hw, hw, k, int(rng.choice([1, 2], p=[0.75, 0.25])), dw,
                 int(rng.choice([1, 2, 4, 8])))


def collect(rings: Rings, n_samples: int, seed: int = 1, max_ws_gb: float = 6.0, log=None,
            max_seconds: float = float("inf")):
    """Times n_samples random (shape, configuration) pairs (fewer if max_seconds runs out);
    returns X [4n][F], y [4n] (log2 ms) and the raw records."""
    rng = np.random.default_rng(seed)
    X, y, recs = [], [], []
    t0 = time.time()
    while len(recs) < n_samples and time.time() - t0 < max_seconds:
        s = random_shape(rng)
        N, L = TRAIN_RINGS[rng.integers(len(TRAIN_RINGS))]
        c_n = int(rng.choice([1, 2]))
        tiles = tile_candidates(N, s)
        impl, rows, groups = schedules(s)[rng.integers(len(schedules(s)))]
        c = Config(N, L, c_n, tiles[rng.integers(len(tiles))], impl, rows, groups)
        f = features(rings, s, c)
        if f is None or workspace_gb(rings, s, c) > max_ws_gb:
            continue
        if H.he_conv_check(rings.get(N, L), c.desc(s), timing_weights(s), c.mac_groups, c.mac_impl,
                           c.tc_rows) != H.HE_OK:
            continue
        r = measure(rings, s, c)
        if r is None:
            continue
        total, st = r
        X.append(f)
        y.append(np.log2(np.maximum(np.array(st, dtype=np.float64), 1e-4)))
        recs.append({"shape": s.__dict__, "config": c.__dict__, "ms": total, "stage_ms": st})
        if log and len(recs) % 500 == 0:
            log(f"collected {len(recs)} layers ({time.time() - t0:.0f} s)")
    return np.concatenate(X), np.concatenate(y).astype(np.float32), recs


class CostModel:
    """he_mlp trained on per-stage log2 latencies; a layer's prediction is the sum over stages."""

    def __init__(self, seed: int = 3):
        import torch

        self.torch = torch
        self.m = H.he_mlp_create(N_FEATURES, seed)

    def train(self, X, y, steps=6000, batch=512, lr=2e-3, seed=5):
        t = self.torch
        dX, dy = t.from_numpy(np.ascontiguousarray(X)).cuda(), t.from_numpy(np.ascontiguousarray(y)).cuda()
        return H.he_mlp_train(self.m, dX.data_ptr(), dy.data_ptr(), len(y), steps, batch, lr, seed)

    def predict_rows(self, X) -> np.ndarray:
        t = self.torch
        dX = t.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        out = t.empty(len(X), dtype=t.float32, device="cuda")
        H.he_mlp_predict(self.m, dX.data_ptr(), len(X), out.data_ptr())
        t.cuda.synchronize()
        return out.cpu().numpy()

    def predict_layers(self, feats: list) -> np.ndarray:
        """Predicted ms of each configuration (feature blocks of 4 rows)."""
        rows = self.predict_rows(np.concatenate(feats))
        return (2.0 ** rows.reshape(-1, 4)).sum(axis=1)

    def save(self, path):
        json.dump({"n_features": N_FEATURES, "params": [float(x) for x in H.he_mlp_params(self.m)]},
                  open(path, "w"))

    @classmethod
    def load(cls, path):
        d = json.load(open(path))
        if d["n_features"] != N_FEATURES:
            raise ValueError("cost model weights were trained on another feature set")
        m = cls()
        H.he_mlp_set_params(m.m, np.array(d["params"], dtype=np.float32))
        return m

    def close(self):
        H.he_mlp_destroy(self.m)


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_weights.json")


def pick(rings: Rings, model: CostModel, s: Shape, ring_list=SELECT_RINGS, max_ws_gb: float = 60.0) -> Config:
    """The model's choice among the candidate configurations of a layer (no timing)."""
    w = timing_weights(s)
    cands = [c for c in candidates(rings, s, ring_list) if workspace_gb(rings, s, c) <= max_ws_gb
             and H.he_conv_check(rings.get(c.N, c.L), c.desc(s), w, c.mac_groups, c.mac_impl, c.tc_rows) == H.HE_OK]
    pred = model.predict_layers([features(rings, s, c) for c in cands])
    return cands[int(np.argmin(pred))]


def autotune(rings: Rings, s: Shape, cands: list, reps: int = 2):
    """Exhaustive search: (best config, best ms, {config: ms}) over the admissible candidates."""
    times = {}
    for c in cands:
        r = measure(rings, s, c, reps)
        if r is not None:
            times[c] = r[0]
    best = min(times, key=times.get)
    return best, times[best], times


STACKS = {
    "resnet20": (lambda sy: [Shape(c.C_in, c.C_out, c.H, c.W, c.k, c.stride, c.depthwise, 1)
                             for c in sy.resnet20_convs()], (8192, 3)),
    "vgg16": (lambda sy: [Shape(c.C_in, c.C_out, c.H, c.W, c.k, c.stride, c.depthwise, 8)
                          for c in sy.vgg16_convs()], (16384, 4)),
    "mobilenet": (lambda sy: [Shape(c.C_in, c.C_out, c.H, c.W, c.k, c.stride, c.depthwise, 32)
                              for c in sy.mobilenet_v1_convs()], (8192, 4)),
}


def evaluate(rings: Rings, model: CostModel, shapes: list, ring_default, max_ws_gb=60.0, log=None):
    """Per layer: the default configuration, the exhaustive optimum and the model's pick, all timed."""
    out = []
    for i, s in enumerate(shapes):
        cands = [c for c in candidates(rings, s) if workspace_gb(rings, s, c) <= max_ws_gb]
        best, best_ms, times = autotune(rings, s, cands)
        ok = [c for c in cands if c in times]
        pred = model.predict_layers([features(rings, s, c) for c in ok])
        pick = ok[int(np.argmin(pred))]
        d = default_config(s, *ring_default)
        dr = measure(rings, s, d)
        out.append({"layer": i, "shape": s.__dict__, "n_candidates": len(ok), "best": best.__dict__,
                    "best_ms": best_ms, "pick": pick.__dict__, "pick_ms": times[pick],
                    "pick_predicted_ms": float(pred.min()), "default_ms": dr[0] if dr else None,
                    "regret": times[pick] / best_ms - 1.0,
                    "rank_of_pick": sorted(times.values()).index(times[pick]) + 1})
        if log:
            log(f"layer {i}: {len(ok)} configs, best {best_ms:.3f} ms, pick {times[pick]:.3f} ms, "
                f"default {out[-1]['default_ms']}")
    return out


def main():
    import sys

    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=5000)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--out", default="costmodel_out")
    ap.add_argument("--stacks", default="resnet20,vgg16,mobilenet")
    ap.add_argument("--collect-seconds", type=float, default=600.0)
    ap.add_argument("--save-model", default=None, help="also write the trained weights (JSON) here")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    torch.cuda.set_device(0)

    def log(m):
        print(m, flush=True)

    rings = Rings()
    t0 = time.time()
    X, y, recs = collect(rings, args.samples, log=log, max_seconds=args.collect_seconds)
    t_collect = time.time() - t0
    np.savez_compressed(os.path.join(args.out, "latencies.npz"), X=X, y=y)
    # hold out every fifth layer to measure the model's error on unseen layers
    n = len(recs)
    hold = np.zeros(n, dtype=bool)
    hold[::5] = True
    rows_hold = np.repeat(hold, 4)
    model = CostModel()
    t1 = time.time()
    loss = model.train(X[~rows_hold], y[~rows_hold], steps=args.steps)
    t_train = time.time() - t1
    pr = model.predict_rows(X[rows_hold])
    err_stage = float(np.median(np.abs(2.0 ** (pr - y[rows_hold]) - 1.0)))
    lay_pred = (2.0 ** pr.reshape(-1, 4)).sum(1)
    lay_true = (2.0 ** y[rows_hold].reshape(-1, 4)).sum(1)
    err_layer = float(np.median(np.abs(lay_pred / lay_true - 1.0)))
    # retrain on everything for the selection
    model.close()
    model = CostModel()
    model.train(X, y, steps=args.steps)
    if args.save_model:
        model.save(args.save_model)
    report = {"samples_layers": n, "kernel_latencies": int(len(y)), "collect_s": t_collect, "train_s": t_train,
              "final_train_loss": loss, "holdout_median_rel_error_stage": err_stage,
              "holdout_median_rel_error_layer": err_layer, "stacks": {}}
    json.dump(report, open(os.path.join(args.out, "report.json"), "w"), indent=1)
    for name in [x for x in args.stacks.split(",") if x]:
        fn, ring = STACKS[name]
        res = evaluate(rings, model, fn(synth), ring, log=log)
        tot = {k: sum(r[k] for r in res) for k in ("best_ms", "pick_ms", "default_ms")}
        report["stacks"][name] = {
            "layers": res, "sum_ms": tot, "regret_total": tot["pick_ms"] / tot["best_ms"] - 1.0,
            "mean_regret": float(np.mean([r["regret"] for r in res])),
            "max_regret": float(np.max([r["regret"] for r in res])),
            "speedup_pick_vs_default": tot["default_ms"] / tot["pick_ms"],
            "speedup_best_vs_default": tot["default_ms"] / tot["best_ms"]}
        log(json.dumps({k: v for k, v in report["stacks"][name].items() if k != "layers"}))
        json.dump(report, open(os.path.join(args.out, "report.json"), "w"), indent=1)
    json.dump(report, open(os.path.join(args.out, "report.json"), "w"), indent=1)
    log(json.dumps({k: v for k, v in report.items() if k != "stacks"}))
    model.close()
    rings.close()


if __name__ == "__main__":
    main()
