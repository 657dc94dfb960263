"""GB300-native (sm_103a) FP64 complex GEMM emulated on tensor cores by the Ozaki-I slicing
scheme with a tunable slice count S, and the block-LU solve for the central block tau_00 of
an LSMS-style KKR matrix M = I - t G built on it, with a learned slice-count selector.

The compute path is libozk.so (CUDA kernels behind the C ABI in include/ozk.h);
``binding`` is its ctypes binding.  Build with ``python paper_2603_29975_gb300/build.py``.
"""
from .binding import (OZK_ERR_TIMEOUT, OZK_NB_MAX, OZK_PAIRS_FULL, OZK_PAIRS_TRI, OZK_PANEL_MAX, OZK_SEL_FEATURES,
                      OZK_SEL_NO_FALLBACK, OZK_SEL_NPARAMS, OZK_SEL_OUTPUTS, OZK_SEL_SMAX, OZK_SEL_SMIN,
                      SELECTOR_WEIGHTS, Handle, OzkError, colmajor_cuda, kkr_build_m, kkr_build_m_batched_ptrs,
                      kkr_build_m_shared_ptrs, kkr_build_m_shared_sizes_ptrs, kkr_contour_trace, kkr_tau00,
                      kkr_tau00_autotune, kkr_tau00_autotune_panels, kkr_tau00_batched, kkr_tau00_batched_ptrs,
                      kkr_tau00_lu, launch_count, lib, ozaki2_zgemm, ozaki_zgemm, ozaki_zgemm_noalloc,
                      ozaki_zgemm_vbatched, ozaki_ztrsm, ozk_group_sums_debug, ozk_split_debug, ozk_zgemm_dmma,
                      rel_diff, selector_features, selector_gradient, selector_predict, selector_train_step,
                      to_numpy)

__all__ = ["OZK_ERR_TIMEOUT", "OZK_NB_MAX", "OZK_PAIRS_FULL", "OZK_PAIRS_TRI", "OZK_PANEL_MAX", "OZK_SEL_FEATURES",
           "OZK_SEL_NO_FALLBACK", "OZK_SEL_NPARAMS", "OZK_SEL_OUTPUTS", "OZK_SEL_SMAX", "OZK_SEL_SMIN",
           "SELECTOR_WEIGHTS", "Handle", "OzkError", "colmajor_cuda", "kkr_build_m", "kkr_build_m_batched_ptrs",
           "kkr_build_m_shared_ptrs", "kkr_build_m_shared_sizes_ptrs", "kkr_contour_trace", "kkr_tau00",
           "kkr_tau00_autotune", "kkr_tau00_autotune_panels", "kkr_tau00_batched", "kkr_tau00_batched_ptrs",
           "kkr_tau00_lu", "launch_count", "lib", "ozaki2_zgemm", "ozaki_zgemm", "ozaki_zgemm_noalloc",
           "ozaki_zgemm_vbatched", "ozaki_ztrsm", "ozk_group_sums_debug", "ozk_split_debug", "ozk_zgemm_dmma",
           "rel_diff", "selector_features", "selector_gradient", "selector_predict", "selector_train_step",
           "to_numpy"]
