"""GB300-native contact SPH (CSPH) hot path with Voronoi work-unit balancing
(arXiv 1805.05128).  The computation lives in libcsph.so (CUDA, sm_103a)
behind the C ABI of include/csph.h; this package marshals torch tensors to it.
"""
from . import abi
from .abi import (CsphError, sph_build_cells, sph_conservation, sph_destroy, sph_eval_rates, sph_init,
                  sph_last_error, sph_pair_counts, sph_read_status, sph_step, sph_unit_stats, voronoi_assign,
                  voronoi_balance)


def __getattr__(name):
    if name == "Simulation":
        from .sim import Simulation
        return Simulation
    raise AttributeError(name)
