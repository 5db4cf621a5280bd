"""GB300-native (sm_103a) hot path of the COLA N-body method (Tassev, Zaldarriaga &
Eisenstein 2013, arXiv:1301.0322): 2LPT initial conditions, the particle-mesh force and the
modified COLA kick/drift, as a C-ABI CUDA library with a thin Python binding."""
from .cola import (COLA_NCOEF, ColaDensity, ColaError, Ensemble, Plan, cola_coeffs, cola_config_default, cola_density,
                   cola_density_adjoint, cola_density_from_noise, cola_fft_r2c, cola_force, cola_ic_2lpt,
                   cola_ic_2lpt_adjoint, cola_noise, cola_plan_create, cola_plan_destroy, cola_power,
                   cola_power_noalloc, cola_set_workspace, cola_status, cola_step, cola_step_adjoint,
                   cola_workspace_bytes, load_library, cola_ensemble_create, cola_ensemble_destroy,
                   cola_ensemble_workspace_bytes, cola_ensemble_set_workspace, cola_ensemble_offsets,
                   cola_ensemble_noise, cola_ensemble_ic_2lpt, cola_ensemble_step, cola_ensemble_density,
                   cola_ensemble_power, cola_ensemble_tune, cola_ensemble_get_tuning, cola_ensemble_set_tuning,
                   cola_ensemble_use_graphs, cola_ensemble_status, cola_cross_power, cola_fof,
                   cola_set_fof_union_tries, cola_density_power)

__all__ = ["Plan", "Ensemble", "ColaError", "ColaDensity", "COLA_NCOEF", "load_library", "cola_config_default",
           "cola_plan_create", "cola_plan_destroy", "cola_workspace_bytes", "cola_set_workspace", "cola_coeffs",
           "cola_noise", "cola_ic_2lpt", "cola_step", "cola_force", "cola_density", "cola_power", "cola_fft_r2c",
           "cola_status", "cola_step_adjoint", "cola_density_adjoint", "cola_ic_2lpt_adjoint",
           "cola_density_from_noise", "cola_power_noalloc", "cola_ensemble_create", "cola_ensemble_destroy",
           "cola_ensemble_workspace_bytes", "cola_ensemble_set_workspace", "cola_ensemble_offsets",
           "cola_ensemble_noise", "cola_ensemble_ic_2lpt", "cola_ensemble_step", "cola_ensemble_density",
           "cola_ensemble_power", "cola_ensemble_tune", "cola_ensemble_get_tuning", "cola_ensemble_set_tuning",
           "cola_ensemble_use_graphs", "cola_ensemble_status", "cola_cross_power", "cola_fof",
           "cola_set_fof_union_tries", "cola_density_power"]
