"""Seeded synthetic workloads for the out-of-core executor and its oracle.

Each module builds plain-data chains (see `spec`) and seeded initial arrays with the
shapes and value distributions of the workloads the paper measures (arXiv
1709.02125, Sec. 5.1). Nothing here performs the method's arithmetic.
"""
from . import spec  # noqa: F401
