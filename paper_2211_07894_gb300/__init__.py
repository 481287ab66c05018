"""GB300 (sm_103a) implementation of the batched Gateaux derivative of the
Kohn-Sham SCF residual used by the low-rank dielectric-matrix (LRDM)
preconditioner of Das & Gavini (arXiv 2211.07894, §II).

The computation lives in the C-ABI library ``lib/liblrdm.so`` (declared in
``include/lrdm.h``); ``binding`` marshals torch tensors into it.
"""

from .binding import (  # noqa: F401
    Context,
    KpContext,
    Lrdma,
    LrdmError,
    gateaux_function,
    load,
    lrdm_apply,
    lrdm_backward,
    lrdm_create,
    lrdm_create_rows,
    lrdm_default_options,
    lrdm_destroy,
    lrdm_gateaux_batch,
    lrdm_get_density,
    lrdm_get_mu,
    lrdm_get_projection,
    lrdm_get_tuning,
    lrdm_kp_create,
    lrdm_kp_gateaux,
    lrdm_krylov_step,
    lrdm_profile_enable,
    lrdm_profile_read,
    lrdm_status_query,
    lrdm_status_string,
    rows_callback,
    torch_allreduce,
)
