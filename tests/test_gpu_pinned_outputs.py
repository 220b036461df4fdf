"""Host calls with outputs in page-locked memory: the Hessian is written there by the kernel that
forms it (no device copy and no transfer after it), so the results must equal, bit for bit, those
of the same call with pageable outputs, in every form and on repeated calls."""
import numpy as np
import pytest

import synth
from synth.nets import MLPSpec, make_mlp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["bf16", "bf16x3", "fp64"])
def test_pinned_outputs_equal_pageable(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22462_gb300 import build, nnc
    build.build()
    n, m = 96, 5
    mlp = make_mlp(MLPSpec([n, 256, 128, m], ["tanh", "sigmoid", "identity"]), seed=11, tag="pin")
    x = synth.uniform01(synth.derive_key(11, "pin-x"), n)
    y = synth.uniform01(synth.derive_key(11, "pin-y"), m)
    lam = synth.normal(synth.derive_key(11, "pin-lam"), m)
    net = nnc.Net.from_mlp(mlp, precision=precision)
    ref = net.eval_kkt(x, y, lam)

    def pin(*shape):
        a = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        a[...] = np.nan
        return a

    outs = (pin(m), pin(m, n), pin(n, n), pin(n))
    for _ in range(2):
        got = net.eval_kkt(x, y, lam, out=outs)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        for a in outs:
            a[...] = np.nan
    # a later pageable call is unaffected
    for a, b in zip(net.eval_kkt(x, y, lam), ref):
        assert np.array_equal(a, b)
    net.free()


def test_pinned_outputs_of_the_other_host_calls():
    """nnc_eval (y), nnc_jacobian and nnc_hessian_lag (H and the gradient) with page-locked
    outputs give the pageable results."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from paper_2509_22462_gb300 import build, nnc
    build.build()
    n, m = 64, 4
    mlp = make_mlp(MLPSpec([n, 128, m], ["tanh", "identity"]), seed=12, tag="pin2")
    x = synth.uniform01(synth.derive_key(12, "pin2-x"), n)
    lam = synth.normal(synth.derive_key(12, "pin2-lam"), m)
    net = nnc.Net.from_mlp(mlp, precision="bf16")
    lib = nnc.load_library()
    dp = ctypes.POINTER(ctypes.c_double)

    def pin(*shape):
        a = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        a[...] = np.nan
        return a

    yp, Jp, Hp, gp = pin(m), pin(m, n), pin(n, n), pin(n)
    assert lib.nnc_eval(net.handle, x.ctypes.data_as(dp), yp.ctypes.data_as(dp), 0) == 0
    assert np.array_equal(yp, net.eval(x))
    assert lib.nnc_jacobian(net.handle, x.ctypes.data_as(dp), Jp.ctypes.data_as(dp)) == 0
    assert np.array_equal(Jp, net.jacobian(x))
    assert lib.nnc_hessian_lag(net.handle, x.ctypes.data_as(dp), lam.ctypes.data_as(dp),
                               Hp.ctypes.data_as(dp), gp.ctypes.data_as(dp)) == 0
    H, g = net.hessian_lag(x, lam, want_grad=True)
    assert np.array_equal(Hp, H) and np.array_equal(gp, g)
    net.free()
