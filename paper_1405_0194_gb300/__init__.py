"""GB300 (sm_103a) PEXSI hot path: supernodal LDL^T + selected inversion +
pole sum for DM / EDM / FDM, and LDL^T inertia counts (see
include/pexsi_gb300.h for the C ABI this package binds)."""
from .capi import (  # noqa: F401
    PexsiError,
    library_path,
    pexsi_dm,
    pexsi_dm_device,
    pexsi_dm_poles,
    pexsi_profile_enable,
    pexsi_profile_read,
    pexsi_profile_reset,
    pexsi_inertia,
    pexsi_inertia_device,
    pexsi_last_error_detail,
    pexsi_opts_default,
    pexsi_plan_destroy,
    pexsi_plan_get_perm,
    pexsi_plan_get_stats,
    pexsi_plan_get_supernodes,
    pexsi_pole_table,
    pexsi_selinv,
    pexsi_setup,
    pexsi_strerror,
    pexsi_trace_noalloc,
)
