"""Seeded synthetic workloads shared by the tests, bench.py and smoke().

This module holds none of the homomorphic method's arithmetic: it only draws
plaintext activations and integer filter weights and lists the layer shapes
of the networks the paper evaluates (VGG-16, ResNet-20, MobileNetV1; Sec. 4.1).
Both the CPU oracle and the CUDA library receive the same arrays from here.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014) evaluated at counter
positions, vectorised with numpy's wrapping uint64 arithmetic, so the arrays
are identical on every platform and numpy version.
Fixed seeds: 1 keys, 2 encryption, 3 activations, 4 weights.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_KEYS = 1
SEED_ENC = 2
SEED_ACT = 3
SEED_WEIGHTS = 4

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix(key: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 whose state begins at `key`."""
    with np.errstate(over="ignore"):
        n = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(key) + _GAMMA * n
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _stream(seed: int, label: int) -> int:
    return int(splitmix(int(splitmix(seed, 1)[0]) ^ label, 1)[0])


def uniform_int(seed: int, label: int, shape, lo: int, hi: int) -> np.ndarray:
    """Integers in [lo, hi] (x mod (hi - lo + 1), bias below 2^-40 for small ranges)."""
    n = int(np.prod(shape))
    x = splitmix(_stream(seed, label), n)
    span = np.uint64(hi - lo + 1)
    return (x % span).astype(np.int64).reshape(shape) + lo


def activations(shape, t: int, seed: int = SEED_ACT, label: int = 0) -> np.ndarray:
    """Client activations, uniform in [0, t)."""
    return uniform_int(seed, label, shape, 0, t - 1)


def weights(shape, seed: int = SEED_WEIGHTS, label: int = 0, wmax: int = 8) -> np.ndarray:
    """Integer filter weights, uniform in [-wmax, wmax]."""
    return uniform_int(seed, label, shape, -wmax, wmax)


@dataclass(frozen=True)
class ConvShape:
    """One convolution layer: channels, input size, square kernel, stride."""

    C_in: int
    C_out: int
    H: int
    W: int
    k: int = 3
    stride: int = 1
    depthwise: bool = False


def single_layer_16() -> list[ConvShape]:
    """16 channels, 16x16, 3x3, 16 outputs (the small single-layer case)."""
    return [ConvShape(16, 16, 16, 16)]


def resnet20_convs() -> list[ConvShape]:
    """The 19 3x3 convolutions of a CIFAR ResNet-20 on 32x32 inputs."""
    L = [ConvShape(3, 16, 32, 32)]
    L += [ConvShape(16, 16, 32, 32)] * 6
    L += [ConvShape(16, 32, 32, 32, stride=2)] + [ConvShape(32, 32, 16, 16)] * 5
    L += [ConvShape(32, 64, 16, 16, stride=2)] + [ConvShape(64, 64, 8, 8)] * 5
    return L


def vgg16_convs() -> list[ConvShape]:
    """The 13 3x3 convolutions of VGG-16 on 224x224 inputs."""
    spec = [(3, 64, 224), (64, 64, 224), (64, 128, 112), (128, 128, 112), (128, 256, 56), (256, 256, 56),
            (256, 256, 56), (256, 512, 28), (512, 512, 28), (512, 512, 28), (512, 512, 14), (512, 512, 14),
            (512, 512, 14)]
    return [ConvShape(a, b, h, h) for a, b, h in spec]


def mobilenet_v1_convs() -> list[ConvShape]:
    """The 27 convolutions of MobileNetV1 on 224x224 inputs (3x3 depthwise + 1x1 pointwise)."""
    L = [ConvShape(3, 32, 224, 224, stride=2)]
    spec = [(32, 64, 112, 1), (64, 128, 112, 2), (128, 128, 56, 1), (128, 256, 56, 2), (256, 256, 28, 1),
            (256, 512, 28, 2)] + [(512, 512, 14, 1)] * 5 + [(512, 1024, 14, 2), (1024, 1024, 7, 1)]
    for cin, cout, h, s in spec:
        L.append(ConvShape(cin, cin, h, h, k=3, stride=s, depthwise=True))
        ho = (h - 1) // s + 1
        L.append(ConvShape(cin, cout, ho, ho, k=1))
    return L


def sample_index(label: int, n: int, seed: int = 5) -> int:
    """A seeded index in [0, n): which output ciphertext of a layer a sampled comparison checks."""
    return int(uniform_int(seed, label, (1,), 0, n - 1)[0])


# the network stacks as the tests and the benchmark run them: shapes, ring, images per step
STACKS = {
    "resnet20": (resnet20_convs, 8192, 3, 1),
    "vgg16": (vgg16_convs, 16384, 4, 8),
    "mobilenet": (mobilenet_v1_convs, 8192, 4, 32),
}


def stack_layer(stack: str, i: int, polyphase: bool = False, dw_cn4: bool = False) -> dict:
    """Layer i of a stack as a layer description (3x3 or 1x1, Hyena packing c_n = 2); with
    `polyphase`, a 3x3 stride-2 layer is marked for polyphase packing; with `dw_cn4`, a depthwise
    layer not so marked packs four channels per ciphertext (c_n = 4)."""
    shapes, _, _, images = STACKS[stack]
    s = shapes()[i]
    d = dict(C_in=s.C_in, C_out=s.C_out, H=s.H, W=s.W, kh=s.k, stride=s.stride, depthwise=s.depthwise,
             n_images=images, c_n=2)
    if polyphase and s.stride == 2 and s.k == 3:
        d["polyphase"] = 1
    elif dw_cn4 and s.depthwise:
        d["c_n"] = 4
    return d


def stack_inputs(stack: str, i: int, t: int):
    """Activations, weights and encryption seed of layer i of a stack (the same for every caller)."""
    sp = stack_layer(stack, i)
    act = activations((sp["n_images"], sp["C_in"], sp["H"], sp["W"]), t, label=i)
    wt = weights((sp["C_out"], 1 if sp["depthwise"] else sp["C_in"], sp["kh"], sp["kh"]), label=i)
    return act, wt, SEED_ENC + i
