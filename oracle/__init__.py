"""FP64 CPU oracle of the pair-F12 path -- test infrastructure, not product code.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline/reference leg
may import it.  It shares no code with the CUDA path; its inputs come from the
synthetic/ generator alone.
"""
from .pairf12 import (DOMO, SOMO, local_fit, robust_kernel, pno_transform,
                      amplitude_contractions, spin_multiplicities, pair_energies,
                      pair_forward, energy_weights, pair_gradient, run, kahan_total,
                      augment_pno, virtual_spaces, opposite_spin_orientations,
                      spin_case_weights, spin_case_energies)
