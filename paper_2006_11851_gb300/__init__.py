"""GB300 (sm_103a) library for perspective texture synthesis by energy optimisation.

Bashir & Ghouri, "Perspective Texture Synthesis Based on Improved Energy
Optimization" (arXiv:2006.11851).  The compute path is the C-ABI CUDA library
``libpts`` (include/pts.h); this package is a thin ctypes binding with the same
entry-point names that takes torch CUDA tensors and passes their pointers,
sizes and the current stream (the batched entry points are in ``batched``).  There is no CPU fallback: every call raises if
the CUDA library is not built or no GPU is present.
"""
from ._binding import (  # noqa: F401
    MODES,
    ExemplarIndex,
    PtsError,
    build_exemplar_index,
    build_kmeans_tree,
    downsample2,
    fp32_fma_peak,
    gemm_selftest,
    histogram_match,
    index_load,
    index_pca,
    index_save,
    irls_weights,
    kmeans,
    kmtree_export,
    kmtree_info,
    kmtree_last_leaves,
    lib,
    live_allocations,
    m_step,
    m_step_hist,
    mlp_grad,
    nn_search,
    pca_fit,
    project_queries,
    proposal_info,
    query_rows_f16,
    proposal_top4,
    rgb_of,
    rgbs,
    scale_guided_init,
    scale_map,
    scale_resample,
    set_allocator,
    synthesize_level,
    synthesize_level_async,
    synthesize_level_converge,
    train_proposal,
    upsample2,
    use_torch_allocator,
    wait_selftest,
)
from .pyramid import synthesize_pyramid, synthesize_pyramid_rgbs  # noqa: F401
