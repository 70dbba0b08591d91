"""FP64 CPU DirectLiNGAM oracle (test infrastructure only).

Only tests/, the smoke check in __graft_entry__ and bench.py's CPU-baseline
leg may import this package.  It shares no code with the CUDA path.
"""
from .oracle import (build, lib_path, fit, fit_B, pair_measure, pair_measures, entropy, standardize,
                     covariance, regress, find_root_scores, constants, num_threads,
                     variable_scores)

__all__ = ["build", "lib_path", "fit", "fit_B", "pair_measure", "pair_measures", "entropy", "standardize",
           "covariance", "regress", "find_root_scores", "constants", "num_threads", "variable_scores"]
