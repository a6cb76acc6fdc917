"""Implicit distance-matrix products on GB300 (sm_103a).

``A Z`` with ``A_ij = ||x_i - x_j||_1`` (sort + prefix sums, Algorithms 1-2 of
Indyk & Silwal, arXiv 2210.15114) or ``||x_i - x_j||_2^2`` (the rank-(d+2)
identity of Appendix A), computed by the CUDA kernels of libdm without ever
forming A.  ``binding`` exposes the C ABI of include/dm.h under the same names.
"""
from .binding import (DMError, dm_batch_create, dm_batch_destroy, dm_batch_lanes, dm_batch_run,
                      dm_bruteforce, dm_create, dm_destroy, dm_grad, dm_launch_count,
                      dm_matmat, dm_matmat_host, dm_matvec_l1, dm_matvec_l2sq, dm_plan_destroy,
                      dm_plan_export, dm_prepare, dm_prepare_l2_embed, dm_prepare_lpp, dm_profile_enable, dm_profile_read,
                      dm_set_deterministic, dm_set_stream, dm_status_string, dm_sync)

__all__ = ["DMError", "dm_batch_create", "dm_batch_destroy", "dm_batch_lanes", "dm_batch_run",
           "dm_bruteforce", "dm_create", "dm_destroy", "dm_grad", "dm_launch_count",
           "dm_matmat", "dm_matmat_host", "dm_matvec_l1", "dm_matvec_l2sq", "dm_plan_destroy",
           "dm_plan_export", "dm_prepare", "dm_prepare_l2_embed", "dm_prepare_lpp", "dm_profile_enable", "dm_profile_read",
           "dm_set_deterministic", "dm_set_stream", "dm_status_string", "dm_sync"]
