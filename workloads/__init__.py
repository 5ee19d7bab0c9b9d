"""Seeded synthetic populations and inputs shaped like the TensorNEAT workloads.

This package only draws random numbers and lays them out in the padded
tensor encoding of Sec. 3.1 (node rows [key, bias, response, act, agg],
connection rows [in key, out key, weight, enabled], NaN rows for padding).
It holds none of the network arithmetic: both the FP64 oracle and the CUDA
library consume what it produces, and neither is imported here.
"""
from .generators import (  # noqa: F401
    ACT, AGG, GenomeSpec, random_genome, make_population, CONFIGS,
    population_for, xor_inputs, locomotion_inputs, uneven_inputs,
    regression_batch, random_ops,
)
