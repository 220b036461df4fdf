"""Failure detection on the GPU without a fault: every device-side wait is bounded, so a wait that
nothing satisfies ends with NNC_ERR_TIMEOUT and a recorded wait code, and the context stays usable
(the next evaluation is correct)."""
import numpy as np
import pytest

import synth
from synth.nets import MLPSpec, make_mlp
from oracle import nn as onn

pytestmark = pytest.mark.gpu

NNC_ERR_TIMEOUT = -4


@pytest.fixture(scope="module")
def nnc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22462_gb300 import build, nnc as m
    build.build()
    return m


@pytest.mark.parametrize("which,code", [(0, 91), (1, 93)])
def test_bounded_wait_gives_up_and_context_survives(nnc, which, code):
    st, got = nnc.selftest_bounded_wait(which, 2_000_000)   # about a millisecond
    assert st == NNC_ERR_TIMEOUT and got == code
    mlp = make_mlp(MLPSpec([30, 40, 7], ["tanh", "identity"]), seed=6, tag="fail")
    x = synth.uniform01(synth.derive_key(6, "fail-x"), 30)
    net = nnc.Net.from_mlp(mlp, precision="bf16x3")
    y = net.eval(x)
    assert np.max(np.abs(y - onn.value(mlp, x))) < 1e-12
    net.free()


def test_selftest_argument_errors(nnc):
    assert nnc.selftest_bounded_wait(2, 1000)[0] != 0
    assert nnc.selftest_bounded_wait(0, 0)[0] != 0
