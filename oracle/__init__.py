"""FP64 CPU oracle (test infrastructure only; see ntt_oracle.py)."""

from .ntt_oracle import *  # noqa: F401,F403
from .ntt_oracle import (  # noqa: F401
    BCD_DELTA,
    EPS_MU,
    bcd_nmf,
    select_rank,
    singular_values,
    spectral_norm_sym,
    compression_ratio,
    handoff_normalize,
    init_columns_H,
    init_factors,
    mu_update_H,
    mu_update_W,
    nmf_mu,
    ntt_decompose,
    objective,
    rel_error,
    splitmix64_outputs,
    stream_key,
    tt_entry,
    tt_full,
    uniform01,
    unfold,
)
