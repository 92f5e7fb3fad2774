"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random numbers and nothing else of the propagation method:
no Fock matrix, residual, integrator or cumulant arithmetic lives here.
"""
from .generators import Problem, gen_problem, random_amplitudes, WORKLOADS, workload  # noqa: F401
