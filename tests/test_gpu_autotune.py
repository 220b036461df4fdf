"""The autotuner picks among valid configurations only: results stay the same up to the FP32
summation order of the symmetric product's split-K partial sums (tolerance 1e-4, far inside the
1e-2 Hessian tolerance), and its JSON cache is written and reused."""
import json
import os

import numpy as np
import pytest

import synth
from synth.nets import MLPSpec, make_mlp

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results_and_caches(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22462_gb300 import build, nnc
    build.build()
    mlp = make_mlp(MLPSpec([784, 1024, 1024, 1024, 10], ["tanh", "tanh", "tanh", "identity"]), seed=2)
    d = synth.adversarial_data(seed=1)
    net = nnc.Net.from_mlp(mlp, precision="bf16x3")
    H0 = net.hessian_lag(d.x0, d.lam)
    path = str(tmp_path / "tune.json")
    net.autotune(path)
    choices = [net.tuning(l) for l in range(4)]
    print("[autotune] (tangent N tile, symmetric-product splits) per layer:", choices)
    H1 = net.hessian_lag(d.x0, d.lam)
    # a different split-K count reorders FP32 partial sums of the symmetric product (the
    # split-BF16x3 form itself is ~1e-5 from the FP64 oracle); nothing else may change
    assert np.linalg.norm(H1 - H0) <= 1e-4 * np.linalg.norm(H0)
    cache = json.load(open(path))
    assert any(k.startswith("sm10") and "tangent" in k for k in cache)
    assert any("syrk" in k for k in cache)
    net2 = nnc.Net.from_mlp(mlp, precision="bf16x3")
    net2.autotune(path)                       # served from the cache
    assert [net2.tuning(l) for l in range(4)] == choices
    assert os.path.getsize(path) > 0
    net.free()
    net2.free()


def test_tune_set_pins_tiles_and_keeps_results():
    """nnc_tune_set: every candidate N tile gives the same tangents (the K order of one output is
    the same in every tile), so H changes only through the symmetric product's splits."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22462_gb300 import build, nnc
    build.build()
    mlp = make_mlp(MLPSpec([300, 512, 512, 7], ["tanh", "sigmoid", "identity"]), seed=5)
    x = synth.uniform01(synth.derive_key(5, "tune-x"), 300)
    lam = synth.normal(synth.derive_key(5, "tune-lam"), 7)
    net = nnc.Net.from_mlp(mlp, precision="bf16x3")
    H0 = net.hessian_lag(x, lam)
    for bn in (112, 128, 208, 256):
        net.tune_set(tangent_bn=bn)
        assert net.tuning(1)[0] == bn
        assert np.array_equal(net.hessian_lag(x, lam), H0), bn
    # SM-pair tiles (cta_group::2, 256-row tiles): the same products in the same K order
    for bn in (-128, -160, -208, -256):
        net.tune_set(tangent_bn=bn)
        assert net.tuning(1)[0] == bn
        H = net.hessian_lag(x, lam)
        assert np.linalg.norm(H - H0) <= 1e-6 * np.linalg.norm(H0), (bn, np.linalg.norm(H - H0))
    net.tune_set(syrk_splits=1)
    assert net.tuning(0)[1] == 1
    H1 = net.hessian_lag(x, lam)
    assert np.linalg.norm(H1 - H0) <= 1e-4 * np.linalg.norm(H0)
    with pytest.raises(nnc.NNCError):
        net.tune_set(tangent_bn=100)
    with pytest.raises(nnc.NNCError):
        net.tune_set(tangent_bn=-112)
    net.free()
