"""The algorithmic work that bench.py divides by measured time (the roofline's `achieved`),
against the closed forms written out by hand for the workloads it reports."""
import types

import numpy as np

import bench
import synth
from synth.nets import MLPSpec


def test_hessian_flops_104m_closed_form():
    """784 -> 4096 x 7 -> 10 tanh, linear output: six 4096 x 4096 tangent GEMMs with 784 tangent
    columns (2 n m k each) and the lower triangles of seven symmetric products n (n + 1) m."""
    n, w = 784, 4096
    per_launch = 2 * n * w * w
    assert per_launch == 26_306_674_688
    assert bench.tangent_gemm_flops(synth.PAPER_104M) == [per_launch] * 6
    assert bench.hessian_flops(synth.PAPER_104M) == 6 * per_launch + 7 * n * (n + 1) * w
    assert bench.hessian_flops(synth.PAPER_104M) == 175_485_943_808


def test_hessian_flops_curved_output_layer():
    """With a curved output layer the last layer adds a tangent GEMM and a symmetric product;
    identity hidden layers add no symmetric product."""
    spec = MLPSpec([5, 7, 9, 3], ["tanh", "identity", "sigmoid"])
    n = 5
    tangents = 2 * n * 9 * 7 + 2 * n * 3 * 9        # layers 2 and 3 (layer 1 is W_1 itself)
    syrk = n * (n + 1) * 7 + n * (n + 1) * 3         # layers 1 and 3 have curvature
    assert bench.tangent_gemm_flops(spec) == [2 * n * 9 * 7, 2 * n * 3 * 9]
    assert bench.hessian_flops(spec) == tangents + syrk


def test_tangent_shape_key():
    assert bench.tangent_shape(synth.PAPER_104M) == (4096, 784, 4096)
    assert bench.tangent_shape(synth.PAPER_274M) == (8192, 784, 8192)
    assert bench.tangent_shape(MLPSpec([5, 7, 9, 3], ["tanh", "tanh", "identity"])) == (9, 5, 7)
    assert bench.tangent_shape(MLPSpec([5, 7, 9, 11, 3], ["tanh"] * 3 + ["identity"])) is None
    # the measured traffic applies to its own shape only
    assert bench.TANGENT_TRAFFIC.get((bench.tangent_shape(synth.PAPER_274M), "bf16x3", -208)) is None


def test_scopf_weight_bytes():
    """8 B (double-float value pass) + 4 B (FP32 reverse) per weight, plus the tangent operand: the
    FP32 first layer (4 B) and the hidden layers' BF16 hi + lo (4 B, split form), BF16 hi (2 B) or
    e4m3 (1 B); the linear output layer takes no tangent."""
    rng = np.random.default_rng(0)
    nets = []
    for n_k in (20, 137, 200):
        shapes = [(16, n_k), (16, 16), (16, 16), (1, 16)]
        nets.append(types.SimpleNamespace(W=[rng.standard_normal(s) for s in shapes]))
    for prec, tb in (("bf16x3", 4), ("bf16", 2), ("fp8", 1)):
        expect = 0
        for net in nets:
            P = sum(w.size for w in net.W)
            first, hidden = net.W[0].size, net.W[1].size + net.W[2].size
            assert P == first + hidden + net.W[-1].size
            expect += 12 * P + 4 * first + tb * hidden
        assert bench.scopf_weight_bytes(nets, prec) == expect, prec
    # the bench's own surrogates (8 of them here; the bench runs 256): n_k -> 1024 x 5 -> 1
    data, d, raw = bench._scopf_workload(8)
    P = sum(sum(w.size for w in m.W) for m in raw)
    n_k = [len(s) for s in data.subsets]
    assert P == sum(n * 1024 + 4 * 1024 * 1024 + 1024 for n in n_k)
    assert bench.scopf_weight_bytes(raw, "bf16x3") == 16 * P - 4 * 1024 * len(raw)
    hidden = 4 * 1024 * 1024 * len(raw)
    assert bench.scopf_weight_bytes(raw, "bf16") == 16 * P - 4 * 1024 * len(raw) - 2 * hidden


def test_clock_samples():
    """The clocks record of a bench line: median SM clock, its maximum, and every throttle reason
    seen active in any sample (sw_power_cap kept, hardware slowdowns reported)."""
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, N/A, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = bench.parse_clock_samples(lines)
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.parse_clock_samples([lines[0], "0, 1200, 2070, 1400, 0x48, Active, Active, Not Active, Active"])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    assert bench.parse_clock_samples(["garbage"]) is None
