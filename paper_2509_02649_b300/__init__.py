"""B300 (sm_103a) path of Fourier-represented kernel regression (arXiv 2509.02649).

The compute lives in libfk.so (CUDA kernels behind the C-ABI of include/fk.h);
this package is its thin binding.  Import fails loudly at first use when the
library is missing: there is no CPU fallback.
"""
from ._lib import (FK_FP64, FK_MIXED, FK_PEN_LOWBIAS, FK_PEN_SOBOLEV, FK_SOLVER_AUTO, FK_SOLVER_CG,
                   FK_SOLVER_CHOL, FK_SOLVER_EIG, FK_SPREAD_ATOMIC, FK_SPREAD_AUTO, FK_SPREAD_BINNED, FK_SPREAD_FIXED,
                   FK_SPREAD_FIXED_SHARED, Accumulator,
                   FkError, Opts, default_opts, fk_build_system, fk_fit_additive, fk_fit_pik, fk_fit_sobolev,
                   fk_hypergrad, fk_launch_count, fk_peak_fp32, fk_peak_smem_atomics, fk_heldout_loss, fk_adjoint, fk_autotune_clear, fk_autotune_table, fk_box_moments, fk_fit_pik_general, fk_fit_sobolev_pairs, Graph, capture, fk_penalty_grads, fk_penalty_weights, fk_predict, fk_solve,
                   fk_type1,
                   fk_type1_noalloc, fk_type2, generate_sweep_1d, lib)

__all__ = ["FK_FP64", "FK_MIXED", "FK_PEN_SOBOLEV", "FK_PEN_LOWBIAS", "FK_SOLVER_AUTO", "FK_SOLVER_CHOL",
           "FK_SOLVER_CG", "FK_SOLVER_EIG", "FK_SPREAD_AUTO", "FK_SPREAD_ATOMIC", "FK_SPREAD_BINNED", "FK_SPREAD_FIXED",
           "FK_SPREAD_FIXED_SHARED", "Accumulator",
           "FkError", "Opts", "default_opts", "fk_build_system", "fk_fit_sobolev", "fk_fit_pik", "fk_fit_additive",
           "fk_predict", "fk_type1", "fk_type1_noalloc", "fk_type2", "fk_penalty_weights", "fk_solve", "fk_hypergrad",
           "fk_launch_count", "fk_peak_fp32", "fk_peak_smem_atomics", "fk_heldout_loss", "fk_adjoint", "fk_penalty_grads", "fk_autotune_table", "fk_autotune_clear", "fk_box_moments", "fk_fit_pik_general", "fk_fit_sobolev_pairs", "Graph", "capture", "generate_sweep_1d", "lib", "HeldOutLoss", "heldout_loss", "ChunkedHeldOutLoss", "heldout_loss_chunked"]
from .autograd import ChunkedHeldOutLoss, HeldOutLoss, heldout_loss, heldout_loss_chunked  # noqa: E402
