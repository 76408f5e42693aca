"""Host side of the autotuner and cost model: the candidate configurations are
valid layouts, the features are finite and distinguish configurations, and the
random training shapes stay inside the documented ranges."""
import math

import numpy as np

from paper_2311_12519_gb300 import costmodel as CM
from paper_2311_12519_gb300 import hyena as H


def test_candidates_are_valid_layouts_with_distinct_features():
    rings = CM.Rings()
    for s in (CM.Shape(16, 16, 32, 32), CM.Shape(64, 128, 56, 56, 3, 2, False, 8),
              CM.Shape(32, 32, 112, 112, 3, 1, True, 32), CM.Shape(512, 512, 14, 14, 1, 1, False, 8)):
        cands = CM.candidates(rings, s)
        assert len(cands) == len(set(cands))
        feats = []
        for c in cands:
            lay = H.he_layout_for_layer(rings.get(c.N, c.L), c.desc(s))
            assert lay.n_ct_in > 0
            f = CM.features(rings, s, c)
            assert f.shape == (4, CM.N_FEATURES) and np.isfinite(f).all()
            feats.append(f.tobytes())
        assert len(set(feats)) == len(feats), "two configurations share a feature vector"
        if s.depthwise:
            assert all(c.mac_impl == 1 for c in cands)
    rings.close()


def test_tile_candidates_fit_and_follow_the_stride():
    for N in (4096, 8192, 16384):
        for s in (CM.Shape(3, 64, 224, 224), CM.Shape(8, 8, 57, 31, 3, 2), CM.Shape(4, 4, 7, 7, 1)):
            P = (s.k - 1) // 2
            for th, tw in CM.tile_candidates(N, s)[1:]:
                assert (th + 2 * P) * (tw + 2 * P) <= N // 2
                assert th % s.stride == 0 or th == s.H
                assert tw % s.stride == 0 or tw == s.W


def test_random_shapes_in_range():
    rng = np.random.default_rng(0)
    for _ in range(500):
        s = CM.random_shape(rng)
        assert 3 <= s.C_in <= 1024 and 3 <= s.C_out <= 1024 and 7 <= s.H <= 224 and s.H == s.W
        assert s.k in (1, 3) and s.stride in (1, 2) and s.n_images in (1, 2, 4, 8)
        assert not s.depthwise or (s.C_in == s.C_out and s.k == 3)


def test_training_rings_respect_the_security_bound():
    bound = {4096: 109, 8192: 218, 16384: 438}
    for N, L in CM.TRAIN_RINGS + CM.SELECT_RINGS:
        assert 50 * L <= bound[N]
        assert math.log2(N) in (12, 13, 14)


class _LinearModel:
    """Stand-in for the GPU network: least squares on the same features."""

    def __init__(self):
        self.w = None

    def train(self, X, y, **kw):
        A = np.c_[X, np.ones(len(X))]
        self.w = np.linalg.lstsq(A, y, rcond=None)[0]
        return float(np.mean((A @ self.w - y) ** 2))

    def predict_layers(self, feats):
        X = np.concatenate(feats)
        return (2.0 ** (np.c_[X, np.ones(len(X))] @ self.w).reshape(-1, 4)).sum(axis=1)


def test_collect_and_evaluate_pipeline_with_a_synthetic_clock(monkeypatch):
    """The collection, training and evaluation logic on the CPU, with he_conv_time replaced by a
    deterministic function of the layout (the GPU run uses the real timings)."""
    def fake_time(p, d, w, mac_groups=0, mac_impl=0, tc_rows=0, reps=3, stream=0):
        lay = H.he_layout_for_layer(p, d)
        info = H.he_params_info(p)
        if d.c_n == 1 and d.C_in > 200:
            raise H.HyenaError(H.HE_ENOISE, "he_conv_time", "fake noise limit")
        base = lay.n_ct_in * info.N * info.L * 1e-7
        st = [base, base * lay.n_galois / 4, base * (2.0 if mac_impl == 1 else 1.0) * d.C_out / 16,
              lay.n_ct_out * info.N * info.L * 1e-7]
        return sum(st), st

    monkeypatch.setattr(H, "he_conv_time", fake_time)
    rings = CM.Rings()
    X, y, recs = CM.collect(rings, 30, seed=2, max_ws_gb=2.0)
    assert X.shape == (120, CM.N_FEATURES) and y.shape == (120,) and len(recs) == 30
    assert np.isfinite(X).all() and np.isfinite(y).all()
    model = _LinearModel()
    model.train(X, y)
    shapes = [CM.Shape(16, 16, 32, 32), CM.Shape(16, 32, 32, 32, 3, 2)]
    res = CM.evaluate(rings, model, shapes, (8192, 3), max_ws_gb=8.0)
    assert len(res) == 2
    for r in res:
        assert r["regret"] >= 0 and r["pick_ms"] >= r["best_ms"] > 0 and 1 <= r["rank_of_pick"] <= r["n_candidates"]
        assert r["default_ms"] > 0
    rings.close()


def test_conv_check_matches_the_plan_rules_on_the_host():
    """he_conv_check runs the plan's host checks without a device: valid configurations pass,
    a tensor-core request beyond the exactness bound and a bad tune field are refused, and a
    layer whose weights exceed the noise budget is refused with HE_ENOISE."""
    p = H.he_params_create(4096, 2, decomp_bits=25)
    d = H.conv_desc(16, 16, 16, 16)
    w = np.full((16, 16, 3, 3), 8, dtype=np.int32)
    assert H.he_conv_check(p, d, w) == H.HE_OK
    assert H.he_conv_check(p, d, w, mac_impl=2, tc_rows=64) == H.HE_OK
    assert H.he_conv_check(p, d, w, mac_impl=2, tc_rows=40) == H.HE_EINVAL
    assert H.he_conv_check(p, d, np.full((16, 16, 3, 3), 9, dtype=np.int32), mac_impl=2) == H.HE_EINVAL
    H.he_params_destroy(p)
    # a 50-bit decomposition base at two limbs leaves no room for large weights
    p = H.he_params_create(4096, 2, decomp_bits=50)
    assert H.he_conv_check(p, H.conv_desc(64, 16, 7, 7), np.full((16, 64, 3, 3), 8, dtype=np.int32)) == H.HE_OK
    assert H.he_conv_check(p, H.conv_desc(64, 16, 7, 7), np.full((16, 64, 3, 3), 16000, dtype=np.int32)) == \
        H.HE_ENOISE
    H.he_params_destroy(p)


def test_tensor_core_needs_limbs_below_2_to_the_50():
    w = np.full((16, 16, 3, 3), 8, dtype=np.int32)
    d = H.conv_desc(16, 16, 16, 16)
    for bits, L, wb, ok in ((50, 2, 25, True), (54, 2, 27, False), (30, 4, 15, True)):
        p = H.he_params_create(4096, L, limb_bits=bits, decomp_bits=wb)
        assert (H.he_conv_check(p, d, w, mac_impl=2) == H.HE_OK) == ok, bits
        assert H.he_conv_check(p, d, w, mac_impl=1) == H.HE_OK
        H.he_params_destroy(p)
