"""GB300 (sm_103a) SVD-PHAT hot path: PHAT cross spectra, the rank-K projection Z = V^H X,
the exhaustive Re{D Z} argmax or the k-d tree search, and plain SRP-PHAT beside them, all in
hand-written CUDA behind the C ABI of ``include/svdphat.h`` (libsvdphat.so)."""
from .api import (MODE, PREC, Basis, Batch, Proposal, Steering, SvdPhatError, build_steering, build_steering_nearfield,
                  apply_mask, check_status, exported_symbols, fp32_fma_peak, kdtree_search,
                  localize_samples, n_frames, stft, weighted_doa_error,
                  lib, load_basis, localize, localize_batched, localize_host, localize_noalloc, localize_srp, phat, project,
                  save_basis, set_tune_cache, set_wait_budget, svd_reduce, tune_cache_get, tune_cache_put)

__all__ = ["MODE", "PREC", "Basis", "Batch", "Proposal", "Steering", "SvdPhatError", "build_steering",
           "build_steering_nearfield", "check_status", "fp32_fma_peak", "kdtree_search", "apply_mask", "localize_samples",
           "n_frames", "stft", "weighted_doa_error",
           "exported_symbols", "lib", "load_basis", "localize", "localize_batched", "localize_host", "localize_noalloc", "localize_srp", "phat", "project",
           "save_basis", "set_tune_cache", "set_wait_budget", "svd_reduce", "tune_cache_get", "tune_cache_put"]
