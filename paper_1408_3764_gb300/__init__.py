"""GB300-native grand canonical Monte Carlo hot path for Lennard-Jones fluids with
cell lists (after Schwiebert et al., arXiv 1408.3764).

The compute path is the CUDA library built from ``csrc/`` for sm_103a behind
the C ABI of ``include/gcmc.h``; ``gcmc.Box`` is its Python front end.  The
library is loaded lazily, so ``workloads`` imports without a GPU.
"""
__all__ = ["Box", "Batch", "Mix", "cell_list_energy", "workloads"]


def __getattr__(name):
    if name in ("Box", "Batch", "Mix", "cell_list_energy", "species_major_order", "TRACE_DTYPE"):
        from . import gcmc
        return getattr(gcmc, name)
    raise AttributeError(name)
