"""GB300-native adiabatic 3-SAT state-vector evolution (C-ABI library + thin binding).

``from paper_1103_1399_gb300 import Instance`` loads ``libqaa.so`` (built
in-tree by ``paper_1103_1399_gb300.build.build()``); if it is missing the import
raises ImportError -- there is no CPU fallback.  The ``build`` submodule itself
imports without the library.
"""

_EXPORTS = ("Instance", "QaaError", "lib", "flatten_clauses", "SIGNATURES", "MAX_QUBITS", "MAX_CLAUSES",
            "LIB_PATH", "Obs", "KERNEL_KINDS", "Server", "tune_candidates", "forget_tuned_plans",
            "LAUNCH_PASSES", "LAUNCH_GRAPH")

__all__ = list(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        from . import _binding
        return getattr(_binding, name)
    raise AttributeError(name)
