"""GB300 (sm_103a) walk-on-spheres / local-BIE Dirichlet-to-Neumann library.

The numerical path lives in libdtn.so (CUDA kernels behind the C ABI of
include/dtn.h); this package only binds it.  Build with
``python -c "import __graft_entry__ as g; g.build()"`` or
``python paper_1210_1491_gb300/build.py``.
"""
from .binding import (  # noqa: F401
    DATA_CONSTANT, DATA_HARMONIC_SH, DATA_POINT_SOURCE, EXPORTS, GEOM_BALL_INTERIOR,
    GEOM_BOX_INTERIOR, GEOM_BALL_EXTERIOR, GEOM_BOX_MINUS_BOXES, GEOM_DISK_EXTERIOR, GEOM_HALF_SPACE, LIB_PATH, PREC_FP64, PREC_MIXED, DtnError, Geometry,
    HostBatch, Server, alloc_result, autotune_walks, distance, eval_dirichlet, eval_potential, eval_potential_fmm,
    fmm_opts, gather_owned, load,
    philox, philox_fields21, single_point_neumann, solve_opts, solve_patches, wos_points, wos_points_noalloc,
)
