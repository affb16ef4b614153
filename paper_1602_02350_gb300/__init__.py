"""Sketched-preconditioned SVRG for ridge regression on GB300 (sm_103a).

The compute path is the CUDA library ``librs.so`` behind the C ABI of
``include/rs.h``; this package is its thin Python binding (``rs_*`` functions
taking CUDA tensors, same names as the C entry points) plus the seeded
synthetic-input generator ``synth``.
"""

from ._lib import (  # noqa: F401
    Context, RsError, declared_symbols, lib, matrix, Fp8Rows,
    RS_F64, RS_F32, RS_BF16, RS_FP8E4M3, RS_SKETCH_GAUSSIAN, RS_SKETCH_COUNTSKETCH,
    RS_SAMPLE_IMPORTANCE, RS_SAMPLE_UNIFORM,
    rs_philox_words, rs_gaussian, rs_countsketch, rs_range_sketch, rs_orthonormalize, rs_sym_eig,
    rs_ritz, rs_sketch, rs_precondition, rs_map_output, rs_sampling_weights, rs_sampling_table,
    rs_index_stream, rs_full_gradient, rs_full_gradient_static, rs_svrg_epoch, rs_svrg_solve, rs_solve,
    rs_objective, rs_trace_c, rs_speedup_ratio, rs_wait_probe, rs_autotune, rs_catalyst_solve, rs_solve_batched, rs_solve_proposed, rs_mlp_forward, rs_mlp_train_step, rs_propose, mlp_norm, MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_NPARAM,
)
