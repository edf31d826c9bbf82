"""GB300-native flow-based hypergraph refinement (push-relabel max flow on the
Lawler expansion, minimal min cuts, FlowCutter), after Gottesbueren, Heuer and
Sanders, "Parallel Flow-Based Hypergraph Partitioning".

The compute path is libhfp.so (hand-written sm_103a CUDA behind the C ABI in
include/hfp.h); ``hfp`` is its thin Python binding.
"""
from . import hfp  # noqa: F401
from ._build import build  # noqa: F401
