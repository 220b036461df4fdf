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


@pytest.mark.parametrize("which,code", [(0, 91), (1, 93)])
def test_host_call_reports_a_timeout_then_recovers(nnc, which, code):
    """A bounded wait that ran out inside a net's work (queued on its stream, recording into the
    net's error word) is reported by the next host call, which reads the word back with its outputs;
    the call after it is correct again."""
    mlp = make_mlp(MLPSpec([30, 40, 7], ["tanh", "identity"]), seed=7, tag="fail2")
    x = synth.uniform01(synth.derive_key(7, "fail2-x"), 30)
    y0 = synth.uniform01(synth.derive_key(7, "fail2-y"), 7)
    lam = synth.normal(synth.derive_key(7, "fail2-lam"), 7)
    net = nnc.Net.from_mlp(mlp, precision="bf16")
    r_ref, J_ref, H_ref, g_ref = net.eval_kkt(x, y0, lam)
    net.selftest_wait(which, 2_000_000)   # about a millisecond
    with pytest.raises(nnc.NNCError) as e:
        net.eval_kkt(x, y0, lam)
    assert e.value.code == NNC_ERR_TIMEOUT and f"code {code}" in str(e.value)
    r, J, H, g = net.eval_kkt(x, y0, lam)
    assert np.array_equal(r, r_ref) and np.array_equal(J, J_ref)
    assert np.array_equal(H, H_ref) and np.array_equal(g, g_ref)
    net.selftest_wait(which, 2_000_000)
    with pytest.raises(nnc.NNCError) as e:
        net.residual(x, y0)
    assert e.value.code == NNC_ERR_TIMEOUT
    assert np.max(np.abs(net.residual(x, y0) - (y0 - onn.value(mlp, x)))) < 1e-10
    with pytest.raises(nnc.NNCError):
        net.selftest_wait(2, 1000)
    net.free()
