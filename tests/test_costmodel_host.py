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
