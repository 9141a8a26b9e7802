"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws random numbers and lays them out: latent pyramids,
Glorot-initialised MLP weights, per-query (uv, lod, wi, wo, xi) arrays and the
procedural training target.  It contains none of the neural-BRDF evaluation
itself (no filtering, no frame construction, no MLP).
"""
from .synth import *  # noqa: F401,F403
