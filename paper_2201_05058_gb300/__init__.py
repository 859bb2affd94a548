"""Predicted composite distance fields on GB300 (sm_103a).

A small library for the mapping hot path of Finean et al. (arXiv 2201.05058):
the exact signed EDT of a static voxel map, the fields of predicted human
capsules, their per-voxel composite (Sec. 6, Sec. 8) and the hinge obstacle
cost at robot body spheres with its gradient (Sec. 7).  The compute runs in the
hand-written CUDA kernels of ``libpcdf.so`` behind the C ABI of
``include/pcdf.h``; PyTorch supplies device memory and streams only.
"""
from .api import (  # noqa: F401
    SurrogateMLP,
    surrogate_features,
    surrogate_finish,
    surrogate_query,
    surrogate_step,
    surrogate_select,
    surrogate_samples,
    Batch,
    Context,
    batch_autotune,
    Grid,
    HingeCost,
    build_from_scratch,
    build_template,
    composite_translated,
    lattice_placements,
    template_box,
    template_radius,
    build_predicted_composite,
    build_static_sdf,
    CYLINDER,
    capsule_fixed,
    composite_finish,
    predicted_fields,
    update_workspace,
    filter_voxels,
    collapse_2d,
    edt_2d,
    update_to_host,
    composite_prepare,
    composite_slab,
    composite_workspace,
    hinge_cost,
    query_cost,
    query_cost_backward,
)
from .build import build_library  # noqa: F401
