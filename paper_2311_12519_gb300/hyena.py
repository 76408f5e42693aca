"""Thin ctypes binding of libhyena (include/hyena.h).

Every function here has the name of the C entry point it calls and only
marshals arguments: host arrays are numpy arrays, device buffers are raw
pointers (e.g. ``tensor.data_ptr()`` of a torch CUDA tensor) and streams are
``cudaStream_t`` handles as integers (``torch.cuda.current_stream().cuda_stream``).
All computation happens in the library; if it cannot be loaded, importing
this module fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HE_OK, HE_EINVAL, HE_ENOMEM, HE_ECUDA, HE_ENOISE, HE_ETIMEOUT, HE_EMISSINGKEY = range(7)
HE_MAX_LIMBS = 8
STAGES = ("ntt_in", "keyswitch", "mac", "ntt_out")

u32, u64, i64, sz = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_size_t
vp = ctypes.c_void_p


class he_param_req(ctypes.Structure):
    _fields_ = [("N", u32), ("L", u32), ("limb_bits", u32), ("t_bits", u32), ("t", u64), ("decomp_bits", u32),
                ("k_max", u32), ("est_mac_terms", u32), ("est_weight_max", u32)]


class he_param_info(ctypes.Structure):
    _fields_ = [("N", u32), ("L", u32), ("w", u32), ("l", u32), ("t", u64), ("zeta", u64), ("h", u64), ("k", u64),
                ("kh", i64), ("log2_delta", ctypes.c_double), ("est_noise_log2", ctypes.c_double),
                ("q", u64 * HE_MAX_LIMBS), ("k4", u64)]


class he_conv_desc(ctypes.Structure):
    _fields_ = [(n, u32) for n in ("C_in", "C_out", "H", "W", "kh", "stride", "depthwise", "n_images", "c_n",
                                   "tile_h", "tile_w", "polyphase")]


class he_layout(ctypes.Structure):
    _fields_ = [(n, u32) for n in ("P", "T_h", "T_w", "W_b", "block_slots", "blocks_per_row", "n_ty", "n_tx",
                                   "units", "row_units", "in_groups", "out_groups", "n_ct_in", "n_ct_out", "Ho",
                                   "Wo", "n_galois")] + [("scale", u64)]


class he_tune(ctypes.Structure):
    _fields_ = [("mac_groups", u32), ("mac_impl", u32), ("tc_rows", u32), ("tc_cluster", u32), ("reserved", u32 * 4)]


class he_stage_times(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 4), ("launches", u64 * 4)]


class HyenaError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__(f"{fn} failed with code {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Loads libhyena.so, compiling it with nvcc first if it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libhyena.so not built at {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    A = {
        "he_last_error": (ctypes.c_char_p, []),
        "he_params_create": (ctypes.c_int, [P(he_param_req), P(vp)]),
        "he_params_info": (ctypes.c_int, [vp, P(he_param_info)]),
        "he_params_destroy": (None, [vp]),
        "he_keygen": (ctypes.c_int, [vp, u64, P(vp)]),
        "he_seckey_export": (ctypes.c_int, [vp, vp]),
        "he_seckey_destroy": (None, [vp]),
        "he_galois_keys": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, u64, P(vp)]),
        "he_galkeys_export": (ctypes.c_int, [vp, u32, vp]),
        "he_galkeys_destroy": (None, [vp]),
        "he_layout_for_layer": (ctypes.c_int, [vp, P(he_conv_desc), P(he_layout)]),
        "he_layer_galois": (ctypes.c_int, [vp, P(he_conv_desc), vp, ctypes.c_int, P(ctypes.c_int)]),
        "he_encrypt_image": (ctypes.c_int, [vp, vp, P(he_conv_desc), vp, u64, vp]),
        "he_decrypt_image": (ctypes.c_int, [vp, vp, P(he_conv_desc), vp, ctypes.c_int, vp]),
        "he_encrypt_slots": (ctypes.c_int, [vp, vp, vp, u64, u64, vp]),
        "he_decrypt_slots": (ctypes.c_int, [vp, vp, vp, vp]),
        "he_conv_plan": (ctypes.c_int, [vp, vp, P(he_conv_desc), vp, P(he_tune), P(vp)]),
        "he_conv_sizes": (ctypes.c_int, [vp, P(sz), P(sz), P(sz)]),
        "he_conv_forward": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "he_conv_forward_host": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp]),
        "he_plan_destroy": (None, [vp]),
        "he_conv_forward_noalloc": (ctypes.c_int, [vp, vp, vp, vp]),
        "he_conv_status": (ctypes.c_int, [vp]),
        "he_conv_info": (ctypes.c_int, [vp, P(ctypes.c_int)]),
        "he_selftest_bounded_wait": (ctypes.c_int, [vp]),
        "he_conv_check": (ctypes.c_int, [vp, P(he_conv_desc), vp, P(he_tune)]),
        "he_conv_time": (ctypes.c_int, [vp, P(he_conv_desc), vp, P(he_tune), ctypes.c_int, vp, vp, P(ctypes.c_float)]),
        "he_batch_create": (ctypes.c_int, [vp, ctypes.c_int, P(vp)]),
        "he_batch_create_limited": (ctypes.c_int, [vp, ctypes.c_int, sz, P(vp)]),
        "he_batch_waves": (ctypes.c_int, [vp, P(ctypes.c_int)]),
        "he_batch_workspace_bytes": (ctypes.c_int, [vp, P(sz)]),
        "he_batch_forward": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "he_batch_graph_launch": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "he_batch_forward_host": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp]),
        "he_batch_destroy": (None, [vp]),
        "he_ntt_forward": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
        "he_ntt_inverse": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
        "he_rotate_workspace_bytes": (ctypes.c_int, [vp, ctypes.c_int, P(sz)]),
        "he_rotate": (ctypes.c_int, [vp, vp, u32, vp, vp, ctypes.c_int, vp, vp]),
        "he_profile_enable": (ctypes.c_int, [ctypes.c_int]),
        "he_profile_collect": (ctypes.c_int, [P(he_stage_times)]),
        "he_mlp_create": (ctypes.c_int, [u32, u64, P(vp)]),
        "he_mlp_param_count": (ctypes.c_int, [vp, P(u32)]),
        "he_mlp_get_params": (ctypes.c_int, [vp, vp]),
        "he_mlp_set_params": (ctypes.c_int, [vp, vp]),
        "he_mlp_fit_scaling": (ctypes.c_int, [vp, vp, vp, u32, vp]),
        "he_mlp_step": (ctypes.c_int, [vp, vp, vp, u32, u32, ctypes.c_float, u64, vp, P(ctypes.c_float)]),
        "he_mlp_train": (ctypes.c_int, [vp, vp, vp, u32, u32, u32, ctypes.c_float, u64, vp, P(ctypes.c_float)]),
        "he_mlp_predict": (ctypes.c_int, [vp, vp, u32, vp, vp]),
        "he_mlp_destroy": (None, [vp]),
    }
    for name, (res, args) in A.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def exported_symbols():
    """Names of every entry point this binding declares (all must be exported)."""
    return [n for n in load.__code__.co_consts if isinstance(n, str) and n.startswith("he_")]


def _check(rc, fn):
    if rc != HE_OK:
        raise HyenaError(rc, fn, load().he_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(type(a))


# ---------------------------------------------------------------------- parameters
def he_params_create(N, L, limb_bits=50, t=0, t_bits=20, decomp_bits=0, k_max=32, est_mac_terms=0,
                     est_weight_max=8):
    req = he_param_req(N, L, limb_bits, t_bits, t, decomp_bits, k_max, est_mac_terms, est_weight_max)
    h = vp()
    _check(load().he_params_create(ctypes.byref(req), ctypes.byref(h)), "he_params_create")
    return h.value


def he_params_info(p) -> he_param_info:
    info = he_param_info()
    _check(load().he_params_info(p, ctypes.byref(info)), "he_params_info")
    return info


def he_params_destroy(p):
    load().he_params_destroy(p)


# ---------------------------------------------------------------------- keys
def he_keygen(p, seed):
    h = vp()
    _check(load().he_keygen(p, seed, ctypes.byref(h)), "he_keygen")
    return h.value


def he_seckey_export(sk, N):
    out = np.zeros(N, dtype=np.int64)
    _check(load().he_seckey_export(sk, _ptr(out)), "he_seckey_export")
    return out


def he_seckey_destroy(sk):
    load().he_seckey_destroy(sk)


def he_galois_keys(p, sk, galois, seed):
    g = np.ascontiguousarray(galois, dtype=np.uint32)
    h = vp()
    _check(load().he_galois_keys(p, sk, _ptr(g), len(g), seed, ctypes.byref(h)), "he_galois_keys")
    return h.value


def he_galkeys_export(gk, galois, info: he_param_info):
    out = np.zeros((info.L * info.l, 2, info.L, info.N), dtype=np.uint64)
    _check(load().he_galkeys_export(gk, galois, _ptr(out)), "he_galkeys_export")
    return out


def he_galkeys_destroy(gk):
    load().he_galkeys_destroy(gk)


# ---------------------------------------------------------------------- layout
def conv_desc(C_in, C_out, H, W, kh=3, stride=1, depthwise=False, n_images=1, c_n=2, tile_h=0,
              tile_w=0, polyphase=0) -> he_conv_desc:
    return he_conv_desc(C_in, C_out, H, W, kh, stride, int(depthwise), n_images, c_n, tile_h, tile_w, int(polyphase))


def he_layout_for_layer(p, d: he_conv_desc) -> he_layout:
    lay = he_layout()
    _check(load().he_layout_for_layer(p, ctypes.byref(d), ctypes.byref(lay)), "he_layout_for_layer")
    return lay


def he_layer_galois(p, d: he_conv_desc):
    n = ctypes.c_int()
    _check(load().he_layer_galois(p, ctypes.byref(d), None, 0, ctypes.byref(n)), "he_layer_galois")
    out = np.zeros(n.value, dtype=np.uint32)
    _check(load().he_layer_galois(p, ctypes.byref(d), _ptr(out), n.value, ctypes.byref(n)), "he_layer_galois")
    return out


# ---------------------------------------------------------------------- client
def he_encrypt_image(p, sk, d: he_conv_desc, act, seed, info: he_param_info):
    lay = he_layout_for_layer(p, d)
    a = np.ascontiguousarray(act, dtype=np.int64)
    out = np.zeros((lay.n_ct_in, 2, info.L, info.N), dtype=np.uint64)
    _check(load().he_encrypt_image(p, sk, ctypes.byref(d), _ptr(a), seed, _ptr(out)), "he_encrypt_image")
    return out


def he_decrypt_image(p, sk, d: he_conv_desc, ct, unscale=True):
    lay = he_layout_for_layer(p, d)
    c = np.ascontiguousarray(ct, dtype=np.uint64)
    out = np.zeros((d.n_images, d.C_out, lay.Ho, lay.Wo), dtype=np.int64)
    _check(load().he_decrypt_image(p, sk, ctypes.byref(d), _ptr(c), int(unscale), _ptr(out)), "he_decrypt_image")
    return out


def he_encrypt_slots(p, sk, slots, seed, index, info: he_param_info):
    s = np.ascontiguousarray(slots, dtype=np.int64)
    out = np.zeros((2, info.L, info.N), dtype=np.uint64)
    _check(load().he_encrypt_slots(p, sk, _ptr(s), seed, index, _ptr(out)), "he_encrypt_slots")
    return out


def he_decrypt_slots(p, sk, ct, N):
    c = np.ascontiguousarray(ct, dtype=np.uint64)
    out = np.zeros(N, dtype=np.int64)
    _check(load().he_decrypt_slots(p, sk, _ptr(c), _ptr(out)), "he_decrypt_slots")
    return out


# ---------------------------------------------------------------------- server
def he_conv_plan(p, gk, d: he_conv_desc, weights, mac_groups=0, mac_impl=0, tc_rows=0, tc_cluster=0):
    w = np.ascontiguousarray(weights, dtype=np.int32)
    t = he_tune(mac_groups, mac_impl, tc_rows, tc_cluster)
    h = vp()
    _check(load().he_conv_plan(p, gk, ctypes.byref(d), _ptr(w), ctypes.byref(t), ctypes.byref(h)), "he_conv_plan")
    return h.value


def he_selftest_bounded_wait(stream=0):
    """The status code of the bounded-wait self-test (HE_ETIMEOUT is the expected result)."""
    return load().he_selftest_bounded_wait(stream)


def he_conv_check(p, d: he_conv_desc, weights, mac_groups=0, mac_impl=0, tc_rows=0, tc_cluster=0):
    """HE_OK (0) if he_conv_plan would accept the configuration, else its error code (host only)."""
    w = np.ascontiguousarray(weights, dtype=np.int32)
    t = he_tune(mac_groups, mac_impl, tc_rows, tc_cluster)
    return load().he_conv_check(p, ctypes.byref(d), _ptr(w), ctypes.byref(t))


def he_conv_time(p, d: he_conv_desc, weights, mac_groups=0, mac_impl=0, tc_rows=0, reps=3, stream=0, tc_cluster=0):
    """(total ms, [ntt_in, keyswitch, mac, ntt_out] ms): medians over `reps` timed forwards."""
    w = np.ascontiguousarray(weights, dtype=np.int32)
    t = he_tune(mac_groups, mac_impl, tc_rows, tc_cluster)
    st = (ctypes.c_float * 4)()
    tot = ctypes.c_float()
    _check(load().he_conv_time(p, ctypes.byref(d), _ptr(w), ctypes.byref(t), reps, stream, st, ctypes.byref(tot)),
           "he_conv_time")
    return tot.value, list(st)


def he_conv_status(plan):
    _check(load().he_conv_status(plan), "he_conv_status")


def he_conv_info(plan):
    v = ctypes.c_int()
    _check(load().he_conv_info(plan, ctypes.byref(v)), "he_conv_info")
    return v.value


def he_conv_sizes(plan):
    a, b, c = sz(), sz(), sz()
    _check(load().he_conv_sizes(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "he_conv_sizes")
    return a.value, b.value, c.value


def he_conv_forward(plan, d_in, d_out, d_ws, stream=0):
    _check(load().he_conv_forward(plan, _ptr(d_in), _ptr(d_out), _ptr(d_ws), stream or None), "he_conv_forward")


def he_conv_forward_host(plan, h_in, h_out, d_in, d_out, d_ws, stream=0):
    _check(load().he_conv_forward_host(plan, _ptr(h_in), _ptr(h_out), _ptr(d_in), _ptr(d_out), _ptr(d_ws),
                                       stream or None), "he_conv_forward_host")


def he_plan_destroy(plan):
    load().he_plan_destroy(plan)


HE_NOALLOC_MAX_SCRATCH_BYTES = 33554432


def he_conv_forward_noalloc(plan, d_in, d_out, stream=0):
    """he_conv_forward with the library's static device scratch instead of a
    caller workspace, for callers that cannot allocate device memory."""
    _check(load().he_conv_forward_noalloc(plan, _ptr(d_in), _ptr(d_out), stream or None), "he_conv_forward_noalloc")


# ---------------------------------------------------------------------- batches
def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[_ptr(x) for x in ptrs])
    return arr


def he_batch_create(plans):
    arr = (ctypes.c_void_p * len(plans))(*plans)
    h = vp()
    _check(load().he_batch_create(arr, len(plans), ctypes.byref(h)), "he_batch_create")
    return h.value


def he_batch_create_limited(plans, max_workspace_bytes):
    arr = (ctypes.c_void_p * len(plans))(*plans)
    h = vp()
    _check(load().he_batch_create_limited(arr, len(plans), max_workspace_bytes, ctypes.byref(h)),
           "he_batch_create_limited")
    return h.value


def he_batch_waves(b):
    v = ctypes.c_int()
    _check(load().he_batch_waves(b, ctypes.byref(v)), "he_batch_waves")
    return v.value


def he_batch_workspace_bytes(b):
    v = sz()
    _check(load().he_batch_workspace_bytes(b, ctypes.byref(v)), "he_batch_workspace_bytes")
    return v.value


def he_batch_forward(b, d_ins, d_outs, d_ws, stream=0):
    a, o = _ptr_array(d_ins), _ptr_array(d_outs)
    _check(load().he_batch_forward(b, a, o, _ptr(d_ws), stream or None), "he_batch_forward")


def he_batch_graph_launch(b, d_ins, d_outs, d_ws, stream):
    a, o = _ptr_array(d_ins), _ptr_array(d_outs)
    _check(load().he_batch_graph_launch(b, a, o, _ptr(d_ws), stream or None), "he_batch_graph_launch")


def he_batch_forward_host(b, h_ins, h_outs, d_ins, d_outs, d_ws, stream):
    _check(load().he_batch_forward_host(b, _ptr_array(h_ins), _ptr_array(h_outs), _ptr_array(d_ins),
                                        _ptr_array(d_outs), d_ws, stream), "he_batch_forward_host")


def he_batch_destroy(b):
    load().he_batch_destroy(b)


# ---------------------------------------------------------------------- single steps
def he_ntt_forward(p, d_polys, n_polys, stream=0):
    _check(load().he_ntt_forward(p, _ptr(d_polys), n_polys, stream or None), "he_ntt_forward")


def he_ntt_inverse(p, d_polys, n_polys, stream=0):
    _check(load().he_ntt_inverse(p, _ptr(d_polys), n_polys, stream or None), "he_ntt_inverse")


def he_rotate_workspace_bytes(p, n_ct):
    b = sz()
    _check(load().he_rotate_workspace_bytes(p, n_ct, ctypes.byref(b)), "he_rotate_workspace_bytes")
    return b.value


def he_rotate(p, gk, galois, d_in, d_out, n_ct, d_ws, stream=0):
    _check(load().he_rotate(p, gk, galois, _ptr(d_in), _ptr(d_out), n_ct, _ptr(d_ws), stream or None), "he_rotate")


# ---------------------------------------------------------------------- timing
def he_profile_enable(on=True):
    _check(load().he_profile_enable(int(on)), "he_profile_enable")


def he_profile_collect():
    t = he_stage_times()
    _check(load().he_profile_collect(ctypes.byref(t)), "he_profile_collect")
    return {STAGES[i]: (t.ms[i], t.launches[i]) for i in range(4)}


# ------------------------------------------------------------------ cost model network
def he_mlp_create(n_features, seed):
    h = vp()
    _check(load().he_mlp_create(n_features, seed, ctypes.byref(h)), "he_mlp_create")
    return h.value


def he_mlp_params(m):
    n = u32()
    _check(load().he_mlp_param_count(m, ctypes.byref(n)), "he_mlp_param_count")
    out = np.zeros(n.value, dtype=np.float32)
    _check(load().he_mlp_get_params(m, _ptr(out)), "he_mlp_get_params")
    return out


def he_mlp_set_params(m, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().he_mlp_set_params(m, _ptr(a)), "he_mlp_set_params")


def he_mlp_fit_scaling(m, d_X, d_y, n, stream=0):
    _check(load().he_mlp_fit_scaling(m, d_X, d_y, n, stream), "he_mlp_fit_scaling")


def he_mlp_step(m, d_X, d_y, n, batch, lr, seed, stream=0):
    loss = ctypes.c_float()
    _check(load().he_mlp_step(m, d_X, d_y, n, batch, lr, seed, stream, ctypes.byref(loss)), "he_mlp_step")
    return loss.value


def he_mlp_train(m, d_X, d_y, n, steps, batch, lr, seed, stream=0):
    loss = ctypes.c_float()
    _check(load().he_mlp_train(m, d_X, d_y, n, steps, batch, lr, seed, stream, ctypes.byref(loss)), "he_mlp_train")
    return loss.value


def he_mlp_predict(m, d_X, n, d_y, stream=0):
    _check(load().he_mlp_predict(m, d_X, n, d_y, stream), "he_mlp_predict")


def he_mlp_destroy(m):
    load().he_mlp_destroy(m)
