"""he_conv_forward_noalloc: the forward pass for callers that cannot allocate
device memory (for example code running under a pool that owns all device
memory, or a service whose allocations are frozen after start-up).  It uses
the library's static device scratch instead of a caller workspace.

Checked through the C ABI against he_conv_forward, word for word (the
library's arithmetic is exact, so the tolerance is zero), on two calls in a
row with different inputs; a layer too large for the static scratch must be
rejected with HE_EINVAL.  The file is named so that pytest collects it last;
it builds all of its own state, so it also passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from paper_2311_12519_gb300 import hyena as H  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).view(np.int64)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("N,L,w,spec", [
    (4096, 2, 25, dict(C_in=16, C_out=16, H=16, W=16, kh=3, stride=1, depthwise=False, n_images=1, c_n=2)),
    (1024, 2, 25, dict(C_in=4, C_out=6, H=9, W=7, kh=3, stride=2, depthwise=False, n_images=2, c_n=2)),
])
def test_noalloc_matches_forward_on_two_calls(N, L, w, spec):
    p = H.he_params_create(N, L, decomp_bits=w)
    info = H.he_params_info(p)
    d = H.conv_desc(**spec)
    sk = H.he_keygen(p, synth.SEED_KEYS)
    gk = H.he_galois_keys(p, sk, H.he_layer_galois(p, d), synth.SEED_KEYS)
    wt = synth.weights((spec["C_out"], spec["C_in"], spec["kh"], spec["kh"]))
    plan = H.he_conv_plan(p, gk, d, wt)
    n_in, n_out, ws = H.he_conv_sizes(plan)
    assert ws <= H.HE_NOALLOC_MAX_SCRATCH_BYTES
    d_ws = torch.empty(ws // 8 + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        act = synth.activations((spec["n_images"], spec["C_in"], spec["H"], spec["W"]), info.t, label=100 + call)
        d_in = _dev(H.he_encrypt_image(p, sk, d, act, synth.SEED_ENC, info))
        ref = torch.empty(n_out, dtype=torch.int64, device="cuda")
        got = torch.full((n_out,), -1, dtype=torch.int64, device="cuda")
        H.he_conv_forward(plan, d_in.data_ptr(), ref.data_ptr(), d_ws.data_ptr(), stream)
        H.he_conv_forward_noalloc(plan, d_in.data_ptr(), got.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}: static-scratch output differs from he_conv_forward"
    H.he_plan_destroy(plan)
    H.he_galkeys_destroy(gk)
    H.he_seckey_destroy(sk)
    H.he_params_destroy(p)


def test_noalloc_rejects_layers_beyond_the_static_scratch():
    p = H.he_params_create(8192, 3, decomp_bits=50)
    d = H.conv_desc(64, 64, 8, 8)
    sk = H.he_keygen(p, synth.SEED_KEYS)
    gk = H.he_galois_keys(p, sk, H.he_layer_galois(p, d), synth.SEED_KEYS)
    plan = H.he_conv_plan(p, gk, d, synth.weights((64, 64, 3, 3)))
    n_in, n_out, ws = H.he_conv_sizes(plan)
    assert ws > H.HE_NOALLOC_MAX_SCRATCH_BYTES
    a = torch.zeros(n_in, dtype=torch.int64, device="cuda")
    b = torch.zeros(n_out, dtype=torch.int64, device="cuda")
    with pytest.raises(H.HyenaError) as e:
        H.he_conv_forward_noalloc(plan, a.data_ptr(), b.data_ptr())
    assert e.value.code == H.HE_EINVAL
    H.he_plan_destroy(plan)
