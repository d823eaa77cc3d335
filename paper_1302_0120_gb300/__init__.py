"""GB300 (sm_103a) Gerchberg-Saxton phase masks.

The method of alternating projections of Kramer, Hagemann and Luke,
"Real-Time Phase Masks for Interactive Stimulation of Optogenetic Neurons",
as a C-ABI CUDA library (include/gs.h) with a thin Python binding.
"""

from ._binding import (  # noqa: F401
    GS_ECUDA,
    GS_EINVAL,
    GS_ENOMEM,
    GS_ENUMERIC,
    GS_ETIMEOUT,
    GS_FINAL_RESIDUAL,
    GS_INIT_FROM_TARGET,
    GS_OK,
    GS_TENSOR_CORE,
    GSError,
    gs_create,
    gs_create_batched,
    gs_create_mixed,
    gs_destroy,
    gs_get_grid,
    gs_run,
    gs_run_batched,
    gs_run_mixed,
    gs_run_host,
    gs_set_grid,
    gs_set_slm_amplitude,
    gs_status,
    gs_strerror,
    gs_workspace_bytes,
    gs_workspace_bytes_batched,
)
from .solver import GerchbergSaxton, MixedGerchbergSaxton  # noqa: F401
