"""nnc_residual_noalloc, the entry point for callers that cannot allocate device memory (a host
framework that owns the device memory budget, or a control loop that must not call cudaMalloc,
which can synchronise the device): it must give the same FP64 residual y - NN(x) as nnc_residual
on a net built with nnc_load_weights, and as the FP64 oracle, on two calls in a row (its fixed
scratch array keeps the previous call's contents, which must not leak into the next result).
Collected last on purpose."""
import numpy as np
import pytest

import synth
from oracle import nn as onn
from synth.nets import MLPSpec, make_mlp

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_nnc_residual():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22462_gb300 import build, nnc
    build.build()
    spec = MLPSpec([33, 300, 129, 10], ["tanh", "softplus", "identity"])
    mlp = make_mlp(spec, seed=11, tag="noalloc", bias_std=0.2)
    net = nnc.Net.from_mlp(mlp, precision="fp64")
    dev = torch.device("cuda:0")
    W_dev = [torch.tensor(w, device=dev) for w in mlp.W]
    b_dev = [torch.tensor(b, device=dev) for b in mlp.b]
    for call in range(2):
        x = synth.uniform01(synth.derive_key(call, "noalloc-x"), 33)
        y = synth.normal(synth.derive_key(call, "noalloc-y"), 10)
        ref = net.residual(x, y)
        xd, yd = torch.tensor(x, device=dev), torch.tensor(y, device=dev)
        rd = torch.full((10,), float("nan"), dtype=torch.float64, device=dev)
        nnc.residual_noalloc(spec.widths, spec.acts, W_dev, b_dev, xd, yd, rd)
        torch.cuda.synchronize()
        r = rd.cpu().numpy()
        # the FP64 tolerance of the other GPU tests: 1e-10 relative, against the existing entry
        # point and against the oracle's r = y - NN(x)
        assert np.linalg.norm(r - ref) <= 1e-10 * max(np.linalg.norm(ref), 1.0), (call, r, ref)
        r_or = y - onn.value(mlp, x)
        assert np.linalg.norm(r - r_or) <= 1e-10 * max(np.linalg.norm(r_or), 1.0), (call, r, r_or)
    net.free()


def test_noalloc_rejects_widths_beyond_its_array():
    from paper_2509_22462_gb300 import nnc
    lib = nnc.load_library()
    import ctypes
    wid = (ctypes.c_int * 2)(70000, 3)
    act = (ctypes.c_int * 1)(1)
    fake = ctypes.c_void_p(16)          # never dereferenced: the size check comes first
    Wp = (ctypes.c_void_p * 1)(fake)
    assert lib.nnc_residual_noalloc(1, wid, act, Wp, None, fake, fake, fake, None) == -1
    assert b"65536" in lib.nnc_last_error()


def test_noalloc_rejects_softmax_output():
    from paper_2509_22462_gb300 import nnc
    lib = nnc.load_library()
    import ctypes
    wid = (ctypes.c_int * 2)(4, 3)
    act = (ctypes.c_int * 1)(5)         # NNC_SOFTMAX
    fake = ctypes.c_void_p(16)          # never dereferenced: the activation check comes first
    Wp = (ctypes.c_void_p * 1)(fake)
    assert lib.nnc_residual_noalloc(1, wid, act, Wp, None, fake, fake, fake, None) == -6
    assert b"softmax" in lib.nnc_last_error()
