"""GB300 (sm_103a) tensor-train contraction library.

Contracts two tensors held in tensor-train format along a set of common modes
(the Tensor-Train Contraction Product of Kisil et al., arXiv 2109.00626).  The
compute path is the C-ABI library ``libttc.so`` (``include/ttc.h``, CUDA
kernels under ``csrc/``); this package only marshals arguments.

``inputs`` (seeded synthetic TTs) is numpy-only and imports nothing else.
"""
from ._binding import (  # noqa: F401
    EXPORTS,
    BatchedContraction,
    autotune,
    backward,
    tt_full,
    tt_partial,
    tt_sum,
    LAYOUT,
    PREC,
    Desc,
    FullContraction,
    PairsContraction,
    PartialContraction,
    TTError,
    Decomposition,
    FactoredContraction,
    Rounding,
    round_merged,
    tt_round,
    contract_dense_pairs,
    contract_factored,
    contract_full,
    contract_pairs,
    contract_partial,
    error_string,
    launch_count,
    lib,
    partial_k,
    pairs_shape,
    partial_shape,
    dense_permute,
    svd_workspace,
    tt_decompose,
    workspace_bytes,
)
