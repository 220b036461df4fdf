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
