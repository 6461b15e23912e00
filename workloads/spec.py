"""Plain-data description of stencil loop chains (no arithmetic of the method).

A chain is what a user of the executor enqueues (arXiv 1709.02125, Sec. 3): datasets
declared on a structured block, then parallel loops, each naming a kernel, an
iteration range and a list of arguments (dataset + stencil + access mode). Both the
oracle and the CUDA binding consume these records and map the kernel names onto
their own implementations; this module only holds shapes, names and seeded numbers.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

READ, WRITE, RW, REDUCE = "r", "w", "rw", "red"


@dataclass
class DatSpec:
    """A dataset: interior size per axis (x first), halo depths, dtype name,
    periodic axes, and the dense initial array of the full extent (slowest axis
    first, halos included) or None for zeros."""
    name: str
    size: Tuple[int, ...]
    halo_lo: Tuple[int, ...]
    halo_hi: Tuple[int, ...]
    dtype: str = "f64"
    periodic: Tuple[int, ...] = ()
    init: Optional[np.ndarray] = None

    @property
    def ndim(self) -> int:
        return len(self.size)

    @property
    def shape(self) -> Tuple[int, ...]:
        """numpy shape of the dense full-extent array (slowest axis first)."""
        return tuple(self.size[a] + self.halo_lo[a] + self.halo_hi[a]
                     for a in reversed(range(self.ndim)))


@dataclass
class Arg:
    """One loop argument. `name` is a dataset (or, for REDUCE, a reduction) name;
    `offsets` is a list of per-point offset tuples (x, y[, z])."""
    name: str
    access: str
    offsets: Sequence[Tuple[int, ...]] = ((0, 0),)


@dataclass
class Loop:
    kernel: str
    lo: Tuple[int, ...]
    hi: Tuple[int, ...]
    args: List[Arg]
    params: List[float] = field(default_factory=list)


@dataclass
class RedSpec:
    name: str
    op: str  # "sum" | "max" | "min"
