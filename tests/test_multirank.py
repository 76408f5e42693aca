"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own image.

Ranks share keys and weights and exchange nothing on the data path; the only
collective is the max over ranks of the timed values.  Each rank encrypts its
own image with the library's client code, runs the oracle layer on it and
decrypts the plain convolution of its own image."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    from oracle import bfv, conv
    from oracle import params as prm
    from paper_2311_12519_gb300 import hyena as H

    # the first ResNet-20 layer (3 -> 16 channels, 32x32) on a small ring, with bench.py's per-rank inputs
    N, L, w = 4096, 2, 25
    spec = synth.stack_layer("resnet20", 0)
    p = H.he_params_create(N, L, decomp_bits=w)
    info = H.he_params_info(p)
    d = H.conv_desc(**spec)
    act, wt, enc_seed = bench.rank_inputs("resnet20", 0, rank, info.t)
    sk = H.he_keygen(p, synth.SEED_KEYS)
    cts = H.he_encrypt_image(p, sk, d, act, enc_seed, info)
    P = prm.make_params(N=N, L=L, w=w)
    s = bfv.keygen(P, synth.SEED_KEYS)
    lay = conv.Layout(N=N, **spec)
    ksk = {g: bfv.galois_key(P, s, g, synth.SEED_KEYS) for g in conv.galois_elements(P, lay)}
    out = conv.he_conv(P, lay, wt, cts, ksk)
    ok = bool((H.he_decrypt_image(p, sk, d, out) == conv.conv_plain(act, wt, 1, 1, False, P.t)).all())
    mx = bench.reduce_max([float(rank + 1), 10.0 * (rank + 1)], torch.device("cpu"), world)
    gathered = [None] * world
    dist.all_gather_object(gathered, {"ok": ok, "act0": int(act.reshape(-1)[0]), "ct0": int(cts.reshape(-1)[7])})
    if rank == 0:
        np.save(os.path.join(out_dir, "result.npy"), np.array([mx[0], mx[1], all(g["ok"] for g in gathered),
                                                              len({g["act0"] for g in gathered}),
                                                              len({g["ct0"] for g in gathered})], dtype=object))
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    mx0, mx1, ok, n_act, n_ct = np.load(tmp_path / "result.npy", allow_pickle=True)
    assert (mx0, mx1) == (2.0, 20.0)  # max over ranks
    assert ok  # every rank decrypts its own convolution
    assert n_act == 2 and n_ct == 2  # ranks hold different images and ciphertexts


def test_throughput_counts_every_rank():
    import bench

    import synth

    assert bench.layers_per_second(4, 19, 10, 2.0) == 4 * 19 * 10 / 2.0
    a0, w0, s0 = bench.rank_inputs("vgg16", 3, 0, 786433)
    a1, w1, s1 = bench.rank_inputs("vgg16", 3, 1, 786433)
    assert not (a0 == a1).all() and s0 != s1 and (w0 == w1).all()  # own images, shared weights
    a, w, s = synth.stack_inputs("vgg16", 3, 786433)
    assert (a == a0).all() and (w == w0).all() and s == s0  # rank 0 runs the stack's own seeds
