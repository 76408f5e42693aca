"""Builds and loads the oracle's C arithmetic core (hyena_oracle.c) with ctypes.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hyena_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_OUT = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
u64 = ctypes.c_uint64
i64 = ctypes.c_int64
cint = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle core with the host C compiler (plain -O2)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC)
    if stale:
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    sig = {
        "orc_splitmix_at": (u64, [u64, u64]),
        "orc_stream_key": (u64, [u64, u64, u64, u64]),
        "orc_sample_ternary": (None, [u64, cint, i64p]),
        "orc_sample_uniform": (None, [u64, cint, cint, u64p, u64p]),
        "orc_sample_gauss": (None, [u64, cint, u64, u64, i64, i64p]),
        "orc_ntt_fwd": (None, [u64p, cint, u64, u64]),
        "orc_ntt_inv": (None, [u64p, cint, u64, u64]),
        "orc_negacyclic_mul": (None, [u64p, u64p, u64p, cint, u64, u64]),
        "orc_automorphism": (None, [u64p, u64p, cint, u64, u64]),
        "orc_encrypt": (None, [u64p, i64p, u64p, i64p, u64p, u64p, u64p, cint, cint, u64p]),
        "orc_dot_secret": (None, [u64p, i64p, u64p, u64p, cint, cint, u64p]),
        "orc_galois_key": (None, [i64p, u64, u64p, i64p, u64p, u64p, cint, cint, cint, cint, u64p]),
        "orc_decompose": (None, [u64p, cint, cint, cint, cint, u64p]),
        "orc_rotate_hoisted": (None, [u64p, u64p, u64p, u64, u64p, u64p, cint, cint, cint, u64p]),
        "orc_cmult_add": (None, [u64p, u64p, i64, u64p, cint, cint]),
        "orc_pmult": (None, [u64p, i64p, u64p, u64p, cint, cint, u64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
