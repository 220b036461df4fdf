"""Seeded problem data for the two problem families of Section 4.

* Adversarial example (synthetic variant of Eq. 7): minimise ||x - x0||^2 subject to
  y = NN(x), y_t >= y_j + margin for j != t, 0 <= x <= 1.  x0 ~ U[0,1]^n_in stands in for an
  MNIST image; lambda ~ N(0,1) is a multiplier draw for derivative checks.
* SCOPF-shaped batch (synthetic variant of Eq. 8): G generator setpoints x in [0,1]^G, K
  contingencies each with a stability-margin surrogate that sees the setpoints x[S_k] and,
  through its first-layer bias, the loads of a few buses.  Only random draws live here;
  the calibration of each surrogate's output bias (which evaluates a network) is done by
  the problem builder on each side.
"""
from dataclasses import dataclass
from typing import List
import numpy as np

from .rng import derive_key, uniform01, normal, randint, permutation
from .nets import MLP, make_mlp, surrogate_spec


@dataclass
class AdversarialData:
    x0: np.ndarray          # reference image, U[0,1]^n_in
    target: int             # class that must win by `margin`
    margin: float
    lam: np.ndarray         # N(0,1) multipliers of the network outputs (for oracle checks)


def adversarial_data(n_in: int = 784, n_out: int = 10, seed: int = 0, target: int = 3,
                     margin: float = 0.1) -> AdversarialData:
    x0 = uniform01(derive_key(seed, "x0"), n_in)
    lam = normal(derive_key(seed, "lambda"), n_out)
    return AdversarialData(x0, target, margin, lam)


@dataclass
class ScopfData:
    G: int                          # generators (decision variables)
    n_bus: int                      # load buses
    nets: List[MLP]                 # one surrogate per contingency, output bias not calibrated
    subsets: List[np.ndarray]       # S_k: generator indices seen by surrogate k (length n_k)
    load_buses: List[np.ndarray]    # buses whose loads shift surrogate k's first-layer bias
    load_proj: List[np.ndarray]     # A_k, shape (hidden, n_load_buses), N(0, 1/n_load_buses)
    cost: np.ndarray                # c ~ U[1,10]^G, objective sum_i c_i x_i^2
    delta: np.ndarray               # calibration offsets delta_k ~ U[0.05, 0.2]


def scopf_data(K: int = 256, G: int = 200, n_bus: int = 512, seed: int = 0,
               n_min: int = 20, n_max: int = 200, hidden: int = 1024, depth: int = 5,
               n_load_buses: int = 16, act: str = "sigmoid") -> ScopfData:
    n_k = randint(derive_key(seed, "scopf", "n_k"), K, n_min, n_max)
    nets, subsets, buses, projs = [], [], [], []
    for k in range(K):
        spec = surrogate_spec(int(n_k[k]), hidden, depth, act)
        nets.append(make_mlp(spec, seed, tag=f"scopf_net_{k}"))
        subsets.append(np.sort(permutation(derive_key(seed, "scopf", "S", k), G)[: n_k[k]]))
        buses.append(np.sort(permutation(derive_key(seed, "scopf", "bus", k), n_bus)[:n_load_buses]))
        projs.append(normal(derive_key(seed, "scopf", "A", k), hidden * n_load_buses)
                     .reshape(hidden, n_load_buses) / np.sqrt(n_load_buses))
    cost = 1.0 + 9.0 * uniform01(derive_key(seed, "scopf", "cost"), G)
    delta = 0.05 + 0.15 * uniform01(derive_key(seed, "scopf", "delta"), K)
    return ScopfData(G, n_bus, nets, subsets, buses, projs, cost, delta)


def load_vectors(n: int, n_bus: int = 512, seed: int = 0, tag: str = "loads") -> np.ndarray:
    """n load vectors d ~ N(1, 0.1^2) per bus, shape (n, n_bus)."""
    return 1.0 + 0.1 * normal(derive_key(seed, tag), n * n_bus).reshape(n, n_bus)


def scopf_first_bias(data: ScopfData, k: int, d: np.ndarray) -> np.ndarray:
    """First-layer bias of surrogate k under the load vector d: b_1^(k) + A_k d[B_k] -- the load
    dependence of the stability map G_k(S^g, S^d) in Eq. 8 (problem data, not network work)."""
    return data.nets[k].b[0] + data.load_proj[k] @ d[data.load_buses[k]]


def scopf_demand(data: ScopfData, d: np.ndarray) -> float:
    """Total demand D(d) = 0.5 G mean(d): the generators run at half capacity on average."""
    return 0.5 * data.G * float(np.mean(d))
