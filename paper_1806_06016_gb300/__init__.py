"""GB300-native population-annealing molecular dynamics (arXiv:1806.06016).

The compute path is the CUDA library ``lib/libpamd.so`` (sources in
``csrc/``, interface in ``include/pamd.h``); ``pamd`` is its ctypes binding.
"""
from .pamd import (  # noqa: F401
    PAMD_EINVAL, PAMD_ENOMEM, PAMD_ECUDA, PAMD_ETIMEOUT, PAMD_ENONFINITE, PAMD_ESTATE,
    PAMD_EUNSUPPORTED, PAMD_MAX_ATOMS, PAMD_OK, PAMD_PREC_FP64, PAMD_PREC_MIXED,
    PamdError, PamdObs, PamdOptions, PamdTune, Population, load, pamd_anneal, pamd_autotune, pamd_destroy, pamd_forces,
    pamd_batch_size, pamd_batch_sub, pamd_get_counters, pamd_get_state, pamd_info, pamd_init,
    pamd_init_batch, pamd_last_error, pamd_launch_count,
    pamd_observables, pamd_options_default, pamd_propagate, pamd_reset, pamd_resample, pamd_set_counters,
    pamd_set_state, pamd_sync, torch_options, pamd_checkpoint, pamd_restore,
)
