"""The cost model's GPU network against the float64 reference (oracle/mlp.py),
and the timing entry point it learns from.

The network runs in fp32, so the comparisons carry a tolerance: predictions to
1e-4 relative, one Adam step's weights to 1e-5 plus 1e-3 relative (a step moves
each weight by about lr, and fp32 gradient sums differ from float64 ones by
about 1e-6 relative)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import mlp  # noqa: E402
from paper_2311_12519_gb300 import hyena as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _data(n, F, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 2, (n, F)).astype(np.float32) + np.arange(F, dtype=np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2 - X[:, 2] + 3).astype(np.float32)
    return X, y


def test_predict_matches_reference():
    F, n = 11, 300
    X, _ = _data(n, F, 0)
    m = H.he_mlp_create(F, 7)
    rng = np.random.default_rng(3)
    p = H.he_mlp_params(m).astype(np.float64)
    p[mlp.n_weights(F):] = np.concatenate([rng.normal(0, 1, F), [4.0], rng.uniform(0.5, 2, F), [2.5]])
    p[:mlp.n_weights(F)] += rng.normal(0, 0.05, mlp.n_weights(F))
    H.he_mlp_set_params(m, p.astype(np.float32))
    p32 = H.he_mlp_params(m).astype(np.float64)
    dX = torch.from_numpy(X).cuda()
    dy = torch.empty(n, dtype=torch.float32, device="cuda")
    H.he_mlp_predict(m, dX.data_ptr(), n, dy.data_ptr())
    torch.cuda.synchronize()
    ref = mlp.predict(p32, F, X)
    assert np.allclose(dy.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)
    H.he_mlp_destroy(m)


@pytest.mark.parametrize("batch", [1, 37, 256])
def test_scaling_and_one_adam_step_match_reference(batch):
    F, n = 9, 500
    X, y = _data(n, F, 1)
    m = H.he_mlp_create(F, 11)
    dX, dY = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    H.he_mlp_fit_scaling(m, dX.data_ptr(), dY.data_ptr(), n)
    p0 = H.he_mlp_params(m).astype(np.float64)
    xm, ym, xs, ys = mlp.scaling(X, y)
    nw = mlp.n_weights(F)
    assert np.allclose(p0[nw:nw + F], xm, rtol=1e-5, atol=1e-5) and np.isclose(p0[nw + F], ym, rtol=1e-5)
    assert np.allclose(p0[nw + F + 1:nw + 2 * F + 1], xs, rtol=1e-5) and np.isclose(p0[-1], ys, rtol=1e-5)
    lr, seed = 3e-3, 1234
    loss = H.he_mlp_step(m, dX.data_ptr(), dY.data_ptr(), n, batch, lr, seed)
    p1 = H.he_mlp_params(m).astype(np.float64)
    rows = mlp.batch_rows(seed, 0, batch, n)
    ref_loss, g = mlp.loss_and_grad(p0, F, X, y, rows)
    w1, _, _ = mlp.adam(p0[:nw], np.zeros(nw), np.zeros(nw), g, 1, lr)
    assert np.isclose(loss, ref_loss, rtol=1e-4, atol=1e-6)
    # first Adam step: every weight with a non-negligible gradient moves by lr sign(g)
    assert np.allclose(p1[:nw], w1, rtol=1e-3, atol=1e-5)
    H.he_mlp_destroy(m)


def test_training_fits_a_smooth_function():
    F, n = 6, 4000
    X, y = _data(n, F, 2)
    m = H.he_mlp_create(F, 5)
    dX, dY = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    first = None
    H.he_mlp_fit_scaling(m, dX.data_ptr(), dY.data_ptr(), n)
    first = H.he_mlp_step(m, dX.data_ptr(), dY.data_ptr(), n, 256, 0.0, 9)  # loss before training
    H.he_mlp_train(m, dX.data_ptr(), dY.data_ptr(), n, 1500, 256, 3e-3, 9)
    pred = torch.empty(n, dtype=torch.float32, device="cuda")
    H.he_mlp_predict(m, dX.data_ptr(), n, pred.data_ptr())
    torch.cuda.synchronize()
    mse = float(np.mean((pred.cpu().numpy() - y) ** 2) / np.var(y))
    assert mse < 0.05 < first, (mse, first)
    # deterministic: the same seed gives the same weights
    m2 = H.he_mlp_create(F, 5)
    H.he_mlp_fit_scaling(m2, dX.data_ptr(), dY.data_ptr(), n)
    H.he_mlp_step(m2, dX.data_ptr(), dY.data_ptr(), n, 256, 0.0, 9)
    H.he_mlp_train(m2, dX.data_ptr(), dY.data_ptr(), n, 1500, 256, 3e-3, 9)
    assert (H.he_mlp_params(m) == H.he_mlp_params(m2)).all()
    H.he_mlp_destroy(m)
    H.he_mlp_destroy(m2)


def test_conv_time_reports_stages_and_rejects_bad_tunes():
    p = H.he_params_create(4096, 2, decomp_bits=25)
    d = H.conv_desc(16, 16, 16, 16)
    w = synth.weights((16, 16, 3, 3))
    total, st = H.he_conv_time(p, d, w, reps=3)
    assert total > 0 and all(s > 0 for s in st) and sum(st) <= total * 1.05
    for rows in (32, 64, 96):
        t, _ = H.he_conv_time(p, d, w, mac_impl=2, tc_rows=rows, reps=2)
        assert t > 0
    with pytest.raises(H.HyenaError):
        H.he_conv_time(p, d, w, mac_impl=2, tc_rows=40)
    H.he_params_destroy(p)


def test_tc_rows_tune_gives_identical_outputs():
    """Every rows-per-CTA choice of the tensor-core MAC computes the same words."""
    N, L = 1024, 2
    p = H.he_params_create(N, L, decomp_bits=25)
    info = H.he_params_info(p)
    spec = dict(C_in=8, C_out=70, H=6, W=6, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)
    d = H.conv_desc(**spec)
    sk = H.he_keygen(p, synth.SEED_KEYS)
    gk = H.he_galois_keys(p, sk, H.he_layer_galois(p, d), synth.SEED_KEYS)
    wt = synth.weights((70, 8, 3, 3))
    act = synth.activations((1, 8, 6, 6), info.t)
    cts = H.he_encrypt_image(p, sk, d, act, synth.SEED_ENC, info)
    d_in = torch.from_numpy(cts.reshape(-1).view(np.int64)).cuda()
    outs = []
    for rows in (0, 16, 32, 48, 80):
        plan = H.he_conv_plan(p, gk, d, wt, mac_impl=2, tc_rows=rows)
        _, n_out, ws = H.he_conv_sizes(plan)
        o = torch.full((n_out,), -1, dtype=torch.int64, device="cuda")
        w_ = torch.empty(ws // 8 + 1, dtype=torch.int64, device="cuda")
        H.he_conv_forward(plan, d_in.data_ptr(), o.data_ptr(), w_.data_ptr())
        torch.cuda.synchronize()
        H.he_conv_status(plan)
        outs.append(o.cpu())
        H.he_plan_destroy(plan)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    H.he_galkeys_destroy(gk)
    H.he_seckey_destroy(sk)
    H.he_params_destroy(p)


def test_autotuned_configuration_is_bit_exact():
    """The exhaustive search's choice for a layer, run with real keys, gives the oracle's words
    and decrypts to the plain convolution (every configuration is exact; this checks the one
    the tuner picked, layout and schedule as chosen)."""
    from oracle import bfv, conv
    from oracle import params as prm
    from paper_2311_12519_gb300 import costmodel as CM

    rings = CM.Rings()
    s = CM.Shape(6, 10, 20, 20, 3, 1, False, 2)
    best, best_ms, times = CM.autotune(rings, s, CM.candidates(rings, s, [(4096, 2)]))
    assert best_ms == min(times.values()) and len(times) >= 5
    p = rings.get(best.N, best.L)
    info = H.he_params_info(p)
    d = best.desc(s)
    spec = dict(C_in=s.C_in, C_out=s.C_out, H=s.H, W=s.W, kh=s.k, stride=s.stride, depthwise=s.depthwise,
                n_images=s.n_images, c_n=best.c_n, tile_h=best.tile[0], tile_w=best.tile[1])
    sk = H.he_keygen(p, synth.SEED_KEYS)
    gk = H.he_galois_keys(p, sk, H.he_layer_galois(p, d), synth.SEED_KEYS)
    act = synth.activations((s.n_images, s.C_in, s.H, s.W), info.t)
    wt = synth.weights((s.C_out, s.C_in, 3, 3))
    cts = H.he_encrypt_image(p, sk, d, act, synth.SEED_ENC, info)
    plan = H.he_conv_plan(p, gk, d, wt, mac_groups=best.mac_groups, mac_impl=best.mac_impl, tc_rows=best.tc_rows)
    _, n_out, ws = H.he_conv_sizes(plan)
    d_in = torch.from_numpy(cts.reshape(-1).view(np.int64)).cuda()
    d_out = torch.empty(n_out, dtype=torch.int64, device="cuda")
    d_ws = torch.empty(ws // 8 + 1, dtype=torch.int64, device="cuda")
    H.he_conv_forward(plan, d_in.data_ptr(), d_out.data_ptr(), d_ws.data_ptr())
    torch.cuda.synchronize()
    out = d_out.cpu().numpy().view(np.uint64).reshape(-1, 2, info.L, info.N)
    P = prm.make_params(N=best.N, L=best.L, w=info.w)
    s_or = bfv.keygen(P, synth.SEED_KEYS)
    ol = conv.Layout(N=best.N, **spec)
    ksk = {g: bfv.galois_key(P, s_or, g, synth.SEED_KEYS) for g in conv.galois_elements(P, ol)}
    ref = conv.he_conv(P, ol, wt, cts, ksk)
    assert (out == ref).all()
    dec = H.he_decrypt_image(p, sk, d, out)
    assert (dec == conv.conv_plain(act, wt, 1, 1, False, info.t)).all()
    H.he_plan_destroy(plan)
    H.he_galkeys_destroy(gk)
    H.he_seckey_destroy(sk)
    rings.close()


@pytest.mark.parametrize("stack,li", [("resnet20", 0), ("resnet20", 1), ("resnet20", 7), ("vgg16", 11)])
def test_learned_picks_are_bit_exact(stack, li):
    """The shipped cost model's configuration for a layer (ResNet-20: the first layer, a 16-channel
    layer, the first stride-2 layer; VGG-16: a 512 -> 512 layer on 8 images, K = 4608 terms), run
    with real keys, gives the oracle's words on sampled output ciphertexts, and every output
    decrypts to the plain convolution."""
    import os

    from oracle import bfv, conv
    from oracle import params as prm
    from paper_2311_12519_gb300 import costmodel as CM

    if not os.path.exists(CM.WEIGHTS):
        pytest.skip("no trained weights in the package")
    model = CM.CostModel.load(CM.WEIGHTS)
    rings = CM.Rings()
    sp = synth.stack_layer(stack, li)
    s = CM.Shape(sp["C_in"], sp["C_out"], sp["H"], sp["W"], sp["kh"], sp["stride"], sp["depthwise"], sp["n_images"])
    c = CM.pick(rings, model, s)
    p = rings.get(c.N, c.L)
    info = H.he_params_info(p)
    d = c.desc(s)
    spec = dict(sp, c_n=c.c_n, tile_h=c.tile[0], tile_w=c.tile[1])
    sk = H.he_keygen(p, synth.SEED_KEYS)
    gk = H.he_galois_keys(p, sk, H.he_layer_galois(p, d), synth.SEED_KEYS)
    act, wt, enc_seed = synth.stack_inputs(stack, li, info.t)
    cts = H.he_encrypt_image(p, sk, d, act, enc_seed, info)
    plan = H.he_conv_plan(p, gk, d, wt, mac_groups=c.mac_groups, mac_impl=c.mac_impl, tc_rows=c.tc_rows)
    _, n_out, ws = H.he_conv_sizes(plan)
    d_in = torch.from_numpy(cts.reshape(-1).view(np.int64)).cuda()
    d_out = torch.empty(n_out, dtype=torch.int64, device="cuda")
    d_ws = torch.empty(ws // 8 + 1, dtype=torch.int64, device="cuda")
    H.he_conv_forward(plan, d_in.data_ptr(), d_out.data_ptr(), d_ws.data_ptr())
    torch.cuda.synchronize()
    H.he_conv_status(plan)
    out = d_out.cpu().numpy().view(np.uint64).reshape(-1, 2, info.L, info.N)
    P = prm.make_params(N=c.N, L=c.L, w=info.w)
    s_or = bfv.keygen(P, synth.SEED_KEYS)
    ol = conv.Layout(N=c.N, **spec)
    ksk = {g: bfv.galois_key(P, s_or, g, synth.SEED_KEYS) for g in conv.galois_elements(P, ol)}
    sample = sorted({0, synth.sample_index(li, len(out)), len(out) - 1})
    ref = conv.he_conv(P, ol, wt, cts, ksk, out_cts=sample)
    for i in sample:
        assert (out[i] == ref[i]).all(), (stack, li, c, i)
    dec = H.he_decrypt_image(p, sk, d, out)
    assert (dec == conv.conv_plain(act, wt, s.stride, (s.k - 1) // 2, s.depthwise, info.t)).all(), (stack, li, c)
    H.he_plan_destroy(plan)
    H.he_galkeys_destroy(gk)
    H.he_seckey_destroy(sk)
    model.close()
    rings.close()
