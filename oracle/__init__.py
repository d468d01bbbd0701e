"""FP64 CPU oracle of the GOC-LBM hot path -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  It shares no code with the CUDA library.
"""
from .metric import Metric, map_metric, map_position, axis_tables  # noqa: F401
from .oracle import Oracle, build, build_metric, derived_parameters  # noqa: F401
