"""ggeval: batched GP-GOMEA fitness evaluation on NVIDIA GB300 (sm_103a).

The compute path is the CUDA library built from ``csrc/`` (see
``include/ggeval.h``); :mod:`.ggeval` is its Python binding.
"""
from .ggeval import (  # noqa: F401
    ERR_ARG, ERR_CHECKED, ERR_CUDA, ERR_OOM, ERR_TEMPLATE, ERR_TIMEOUT, ERR_UNSUPPORTED,
    F_EXACT, F_GRAD_MSE, F_GRAPH, F_NO_FOLD, F_POW, F_PROFILE, F_TEST_STALL, LAYOUT_HEAP,
    LAYOUT_PREFIX, PIPE_KINDS, Dataset, GGEvalError, ScaledMSE, adam_step, batch_stats,
    gom_accept, gom_changed, gom_donate, lib, make_batch, pack_host, pipe_rates, trial_sizes)
from .build import build  # noqa: F401
