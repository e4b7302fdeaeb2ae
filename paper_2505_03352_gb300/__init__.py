"""GB300 (sm_103a) library for the differentiable control-variables ->
Yee-grid permittivity chain of arXiv 2505.03352 and its Eq. 1 adjoint.

The CUDA kernels live in csrc/ behind the C ABI of include/epschain.h;
`epschain` is the thin ctypes binding (same function names), `autograd`
wraps it as torch.autograd.Functions, `synth` draws the seeded inputs.
"""

from .epschain import (BatchedVjp, eps_batched_workspace_size, eps_forward_batched,
                       EPS_BC_CLAMP, EPS_BC_PERIODIC, EPS_FIELD_C64, EPS_FIELD_BF16X2_SCALED,
                       EPS_FIELD_F16X2_SCALED, EPS_FLAG_OFFDIAG, EPS_FLAG_NORMALS_3D, EpsError, PreparedVjp, Problem,
                       eps_field_pack, eps_forward, eps_packed_field_bytes,
                       eps_profile_start, eps_profile_stop, eps_launch_count,
                       eps_set_l2_fetch_granularity,
                       eps_selftest_timeout, eps_selftest_bounds,
                       eps_status_string, eps_sync_status,
                       eps_vjp, eps_vjp_real, eps_vjp_surrogate, eps_workspace_size, lib,
                       CLOSE_THEN_OPEN, EPS_MORPH_DILATE, EPS_MORPH_ERODE, Morph,
                       eps_forward_morph, eps_morph_workspace_size, eps_vjp_morph,
                       eps_vjp_real_morph, PreparedVjpMorph,
                       OptParams, eps_opt_init, eps_opt_step, read_opt_state,
                       Coarse, eps_coarse_workspace_size, eps_forward_coarse, eps_vjp_coarse,
                       eps_vjp_real_coarse)

__all__ = [
    "BatchedVjp", "eps_batched_workspace_size", "eps_forward_batched",
    "EPS_BC_CLAMP", "EPS_BC_PERIODIC", "EPS_FIELD_C64", "EPS_FIELD_BF16X2_SCALED",
    "EPS_FIELD_F16X2_SCALED", "EPS_FLAG_OFFDIAG", "EPS_FLAG_NORMALS_3D", "EpsError", "PreparedVjp", "Problem", "eps_forward",
    "eps_field_pack", "eps_packed_field_bytes",
    "eps_profile_start", "eps_profile_stop", "eps_launch_count",
    "eps_set_l2_fetch_granularity",
    "eps_selftest_timeout", "eps_selftest_bounds", "eps_status_string",
    "eps_sync_status", "eps_vjp",
    "eps_vjp_real", "eps_vjp_surrogate", "eps_workspace_size", "lib",
    "CLOSE_THEN_OPEN", "EPS_MORPH_DILATE", "EPS_MORPH_ERODE", "Morph", "eps_forward_morph",
    "eps_morph_workspace_size", "eps_vjp_morph", "eps_vjp_real_morph", "PreparedVjpMorph",
    "OptParams", "eps_opt_init", "eps_opt_step", "read_opt_state",
    "Coarse", "eps_coarse_workspace_size", "eps_forward_coarse", "eps_vjp_coarse",
    "eps_vjp_real_coarse",
]

from . import autograd  # noqa: E402  (torch.autograd wrappers)
