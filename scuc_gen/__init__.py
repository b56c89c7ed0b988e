"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

Nothing in this package computes any step of the solver or of the fixing
method; it only produces instances (and seeded random vectors) that both
sides consume.
"""
from .scuc import (PRESETS, SCUCConfig, SCUCInstance, batch_configs, make_preset, make_scuc,
                   split_network_rows)
from .randlp import random_lp, seeded_vector

__all__ = ["PRESETS", "SCUCConfig", "SCUCInstance", "batch_configs", "make_preset", "make_scuc",
           "random_lp", "seeded_vector", "split_network_rows"]
