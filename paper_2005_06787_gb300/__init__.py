"""GB300-native stem contraction for random-circuit amplitudes.

The work happens in ``lib/libtnstem.so`` (CUDA kernels for sm_103a behind a
C interface, ``include/tnstem.h``); ``binding`` exposes the same entry points
to Python. There is no CPU path: calls fail if the library is missing.
"""

from .binding import (  # noqa: F401
    Network, Plan, TnError, load, make_opts, tn_build_network, tn_cgemm, tn_contract_stem, tn_contract_stem_noalloc,
    tn_linear_xeb, tn_permute, tn_plan_create, tn_plan_export, tn_plan_info, tn_plan_prepare,
    tn_plan_steps, tn_plan_profile, tn_version, tn_plan_features, tn_plan_search, Mlp, N_FEATURES, EXPORTED, PREC, MODE,
    tn_set_prefix, tn_destroy_plan, tn_destroy_network, tn_frugal_sample,
    tn_device_status, tn_fp32_fma_peak, tn_build_hypernetwork,
)


def build(force: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force)
