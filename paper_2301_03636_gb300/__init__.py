"""GB300-native (sm_103a) cost-model hot path of the OpenMP Advisor method
(arXiv 2301.03636): descriptor -> integer features -> MLP regression ->
per-kernel argmin, behind the C ABI declared in include/advisor.h.

Submodules are imported lazily: `workloads` (seeded synthetic inputs) needs
only numpy; `advisor` loads the CUDA library and fails loudly without it.
"""
__all__ = ["workloads", "advisor", "metrics"]
