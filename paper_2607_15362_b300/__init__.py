"""B300-native GOC-LBM: the central-moment MRT lattice Boltzmann method in
general orthogonal coordinates with the D2Q5 magnetic-induction scheme,
behind the C ABI of include/goc.h (libgoc.so, CUDA kernels for sm_103a)."""
from ._abi import GocError, lib  # noqa: F401
from .build import build  # noqa: F401
from .lattice import Batch, Lattice, Slab, metric_info, structs_from_spec  # noqa: F401
