"""Seeded synthetic inputs shared by the oracle tests and the CUDA path (graphs and workload parameters only)."""
from . import graphs, workloads  # noqa: F401
