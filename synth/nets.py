"""Seeded multilayer perceptrons shaped like the paper's networks (Eq. 3, Table 1).

Weights are drawn N(0, 1/fan_in) and biases are zero.  The trained MNIST and SCOPF
networks of the paper are not available, so these random networks stand in for them
with the same widths, depths and activations.
"""
from dataclasses import dataclass, field
from typing import List, Optional
import numpy as np

from .rng import derive_key, normal

ACTIVATIONS = ("identity", "tanh", "sigmoid", "softplus", "gelu", "softmax")


@dataclass
class MLPSpec:
    """Widths d_0 = n_in, d_1, ..., d_L = n_out and one activation name per layer."""
    widths: List[int]
    acts: List[str]
    name: str = "mlp"

    def __post_init__(self):
        assert len(self.acts) == len(self.widths) - 1
        for a in self.acts:
            assert a in ACTIVATIONS, a
        assert "softmax" not in self.acts[:-1], "softmax is an output-layer activation"

    @property
    def n_layers(self) -> int:
        return len(self.widths) - 1

    @property
    def n_in(self) -> int:
        return self.widths[0]

    @property
    def n_out(self) -> int:
        return self.widths[-1]

    @property
    def n_weights(self) -> int:
        return sum(self.widths[l] * self.widths[l + 1] for l in range(self.n_layers))

    @property
    def n_params(self) -> int:
        return self.n_weights + sum(self.widths[1:])


@dataclass
class MLP:
    spec: MLPSpec
    W: List[np.ndarray]            # W[l] has shape (d_{l+1}, d_l), row-major, float64
    b: List[np.ndarray]            # b[l] has shape (d_{l+1},)
    seed: int = 0
    extra: dict = field(default_factory=dict)


def make_mlp(spec: MLPSpec, seed: int = 0, tag: str = "mlp", bias_std: float = 0.0) -> MLP:
    W, b = [], []
    for l in range(spec.n_layers):
        m, k = spec.widths[l + 1], spec.widths[l]
        key = derive_key(seed, tag, "W", l)
        W.append(normal(key, m * k).reshape(m, k) / np.sqrt(k))
        if bias_std > 0.0:
            b.append(bias_std * normal(derive_key(seed, tag, "b", l), m))
        else:
            b.append(np.zeros(m))
    return MLP(spec, W, b, seed)


def make_classifier(spec: MLPSpec, seed: int = 0, tag: str = "clf", out_scale: float = 3.0) -> MLP:
    """A random stand-in for a trained softmax classifier (Section 4.1): hidden weights
    N(0, g^2 / fan_in) with g = 4 for sigmoid layers (the reciprocal of sigmoid'(0), so the
    layer gain stays near one through five wide layers) and g = 1 for tanh, sigmoid biases
    -W 0.5 (centring inputs that average one half), and the output logits scaled by `out_scale`
    so that the class probabilities are peaked as a trained classifier's are.  With these
    settings a confidence of 0.6 on any class is reachable from x ~ U[0,1]^784 inside the box."""
    mlp = make_mlp(spec, seed=seed, tag=tag)
    for l in range(spec.n_layers - 1):
        if spec.acts[l] == "sigmoid":
            mlp.W[l] = 4.0 * mlp.W[l]
            mlp.b[l] = -0.5 * mlp.W[l].sum(axis=1)
    mlp.W[-1] = out_scale * mlp.W[-1]
    return mlp


def mnist_like_spec(hidden: int, n_hidden_layers: int, act: str = "tanh",
                    out_act: str = "identity", n_in: int = 784, n_out: int = 10) -> MLPSpec:
    """784 -> hidden x n_hidden_layers -> 10.  The output layer is linear (logits) by default."""
    widths = [n_in] + [hidden] * n_hidden_layers + [n_out]
    acts = [act] * n_hidden_layers + [out_act]
    return MLPSpec(widths, acts, name=f"mnist_{n_in}_{hidden}x{n_hidden_layers}_{n_out}_{act}")


def surrogate_spec(n_in: int, hidden: int = 1024, depth: int = 5, act: str = "sigmoid") -> MLPSpec:
    """A stability-margin surrogate: n_in setpoints -> hidden x depth -> 1 margin."""
    return MLPSpec([n_in] + [hidden] * depth + [1], [act] * depth + ["identity"],
                   name=f"surrogate_{n_in}_{hidden}x{depth}")


# Named workloads (synthetic stand-ins for the paper's MNIST classifiers).
TINY = mnist_like_spec(128, 2)                 # 784 -> 128 -> 128 -> 10, 118,016 weights
PAPER_104M = mnist_like_spec(4096, 7)          # 784 -> 4096 x 7 -> 10, 103,944,202 params
PAPER_87M = mnist_like_spec(4096, 6)           # literal "6 hidden layers" reading, 87,162,890 params


# The paper's softmax classifiers (Table 1): seven layers in all, so five hidden layers; 4096 wide
# tanh gives 70.4M parameters (the 70M row), 8192 wide sigmoid 275.0M (the 274M row).
PAPER_70M_SOFTMAX = mnist_like_spec(4096, 5, out_act="softmax")
PAPER_274M = mnist_like_spec(8192, 5, act="sigmoid", out_act="softmax")


# SCOPF-shaped single network (Section 4.2): 117 inputs (generator setpoints and loads), 37 outputs
# (stability margins), deep tanh; [117, 4096 x 5, 37] has 67.7M parameters, the size of the
# paper's 68M SCOPF net.  Its Jacobian has 37 seed rows and its Hessian 117 tangents.
SCOPF_68M = MLPSpec([117] + [4096] * 5 + [37], ["tanh"] * 5 + ["identity"],
                    name="scopf_117_4096x5_37_tanh")


def spec_by_name(name: str) -> Optional[MLPSpec]:
    return {"tiny": TINY, "104m": PAPER_104M, "87m": PAPER_87M, "scopf68m": SCOPF_68M,
            "70m": PAPER_70M_SOFTMAX, "274m": PAPER_274M}.get(name)


def warmstart_params(n_in: int, h1: int, h2: int, n_out: int, seed: int = 0):
    """Initial weights of the warm-start MLP n_in -> h1 -> h2 -> n_out: N(0, 2/fan_in) (He et al.
    2015, suited to GELU layers), zero biases.  Returned as [W1, b1, W2, b2, W3, b3]."""
    out = []
    for l, (m, k) in enumerate(((h1, n_in), (h2, h1), (n_out, h2))):
        out.append(normal(derive_key(seed, "warmstart", "W", l), m * k).reshape(m, k) * np.sqrt(2.0 / k))
        out.append(np.zeros(m))
    return out
