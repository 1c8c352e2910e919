"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Holds none of the method's arithmetic: Philox4x32-10 draws, Irwin-Hall
Gaussians, SPD metrics X X^T + 0.1 I from integer X, QR-orthonormalised PNO
coefficients, pair lists and the packed ragged layout.
"""
from .workloads import (Workload, WORKLOADS, tiny, c40h81, c160h321, lattice_quartet, custom,
                        pair_inputs, packed_inputs, packed_offsets, pack_lower, unpack, ALIGN)
