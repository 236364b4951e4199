"""SU(2) lattice gauge theory heat bath for GB300 (sm_103a).

A CUDA implementation of the quenched SU(2) Monte Carlo of Cardoso & Bicudo,
"SU(2) Lattice Gauge Theory Simulations on Fermi GPUs" (arXiv:1010.4834): the
checkerboard heat-bath sweep, over-relaxation, plaquette, Polyakov loop, APE
smearing and Wilson loops, behind the C ABI of include/su2.h.
"""
from ._lib import SU2Error, load as load_library  # noqa: F401
from .lattice import Batch, Lattice, kernel_launches, probe_fma  # noqa: F401
