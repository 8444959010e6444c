"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

Only input construction lives here (circuit text, shot index ranges); no step of the sampling
method is computed in this package.
"""
from .circuits import WORKLOADS, cultivation_circuit, tiny_circuit, workload_circuit
from .random_circuits import random_circuit

__all__ = ["WORKLOADS", "cultivation_circuit", "tiny_circuit", "workload_circuit", "random_circuit"]
