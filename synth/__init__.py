"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module draws random numbers and shapes them into networks and problem data.
It holds none of the method's arithmetic (no network evaluation, no derivative,
no interior-point step), so both sides of every parity test can import it.

Generator: splitmix64 used as a counter-based generator (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): output i of the
stream with key k is mix64(k + (i + 1) * 0x9E3779B97F4A7C15).  Uniforms take the
top 53 bits, normals use the Box-Muller transform (one normal per pair of
uniforms).  Everything is vectorised numpy, so the draw is identical on every
machine and library version.
"""
from .rng import derive_key, uniform01, normal, randint, permutation  # noqa: F401
from .nets import (MLP, MLPSpec, make_mlp, make_classifier, mnist_like_spec, surrogate_spec, spec_by_name, TINY,  # noqa: F401
                   PAPER_104M, PAPER_87M, PAPER_70M_SOFTMAX, PAPER_274M, SCOPF_68M,
                   warmstart_params)
from .problems import (AdversarialData, adversarial_data, ScopfData, scopf_data, load_vectors,  # noqa: F401
                       scopf_first_bias, scopf_demand)
