"""GB300-native (sm_103a) path-integral Monte Carlo estimator of transition
amplitudes with level-p effective actions (SPEEDUP method).

The compute path lives in libspeedup_gb300.so (C ABI: include/speedup.h);
this package is its ctypes binding.  There is no CPU fallback: without the
built library or a CUDA device the entry points raise.
"""
from ._binding import (  # noqa: F401
    BatchPlan, EXPORTS, GENERAL_MAX_P, MAX_D, MLP_PARAMS, MODELS, PRECISIONS, Plan, PlanND, Proposal, SpeedupError, library_path, load,
    general_params, options, speedup_amplitude, speedup_amplitude_batch, speedup_amplitude_nd, speedup_amplitude_noalloc,
    speedup_amplitude_proposal, speedup_amplitude_judged,
    speedup_evolution_matrix, speedup_evolution_band, speedup_evolution_spectrum, su_evolution_band_size, speedup_generate_coeffs, speedup_generate_nd, speedup_logweights,
    speedup_logweights_nd, speedup_normals, speedup_philox_words,
    speedup_proposal_logweights, speedup_train_proposal, speedup_wp, speedup_wp_nd, su_autotune, su_autotune_clear, su_batch_autotune,
    su_fault_inject, su_fit_continuum, su_fixed_shape,
    su_fma_peak,
    su_last_error, su_mlp_loss_grad, su_version,
)
