"""GB300 (sm_103a) implementation of the Direct Voxel Grid Optimization render step.

The compute lives in ``libdvgo.so`` (CUDA, C ABI in ``include/dvgo.h``).  This package only
marshals torch tensors into that ABI: ``dvgo_*`` functions with the C names, a
``torch.autograd.Function`` over the forward / backward pair, and a small ``Renderer`` helper
that owns descriptors and the workspace.  There is no CPU fallback: every call fails loudly when
the library is missing or a tensor is not on a CUDA device.
"""
from .binding import (  # noqa: F401
    DVGO_DTYPE_BF16, DVGO_DTYPE_F32, DVGO_MLP_BF16, DVGO_MLP_FP32, DVGO_MODE_COARSE, DVGO_MODE_FINE,
    DVGOError, GridDesc, Params, dvgo_abi_version, dvgo_adam_step, dvgo_adam_step_multi, dvgo_lr_at, dvgo_render_bwd,
    dvgo_render_fwd, dvgo_sample_counts, dvgo_shift_from_alpha_init, dvgo_status_string, dvgo_workspace_size,
    dvgo_workspace_status, lib, library_path, EXPORTED_SYMBOLS, KERNEL_KINDS, dvgo_profile_enable,
    dvgo_profile_read, dvgo_profile_trace, dvgo_launch_counter, dvgo_render_fwd_noalloc, dvgo_weight_bins, dvgo_proposal_fwd,
    dvgo_proposal_bwd, dvgo_sample_pdf, PROP_KEYS, FreeSpace, dvgo_unknown_bbox, DVGO_ACT_POST, DVGO_ACT_PRE,
    DVGO_ACT_IN, DVGO_LAYOUT_CANONICAL, DVGO_LAYOUT_PACKED, dvgo_grid_elements, dvgo_pack_grid, dvgo_resize_grid,
    dvgo_fit2d, dvgo_touched_points, dvgo_view_counts,
)
from .render import (  # noqa: F401
    AdamState, BatchStager, CoarseModel, FineModel, FrameRenderer, Proposal, ProposalTrainer, Renderer, RenderFunction,
    mlp_flat_size, mlp_views,
)
