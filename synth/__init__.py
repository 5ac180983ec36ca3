"""Seeded synthetic Fock matrices shared by the tests, the oracle checks and the benchmark.

This package only draws random numbers and lays them out; it holds none of the
density-matrix arithmetic (no Gershgorin bounds, no polynomial expansion, no
truncation).  Both the CPU oracle and the CUDA path receive the same arrays
from here.
"""
from .fock import (  # noqa: F401
    BLOCK,
    BlockSparse,
    CONFIGS,
    dense_gapped,
    water_like,
    helix_like,
    make_config,
    random_symmetric_on_pattern,
    to_dense,
    from_dense,
)
