"""GB300-native Cholesky-factorised second-order electron propagator.

The compute path lives in ``libcdsigma.so`` (CUDA, sm_103a) behind the C ABI
of ``include/cdsigma.h``; ``cdsigma`` is its thin binding.
"""
from .cdsigma import (CdsError, cds_acd_aux_pairs, cds_cd_decompose, cds_cd_decompose_shells,
                      cds_cd_decompose_to_mo, cds_cd_gemm_time, cds_cd_gemm_timing, cds_cd_stats, cds_cd_to_mo, cds_eri_columns, cds_eri_diag, cds_launch_count,
                      cds_mp2_energy, cds_qp_solve, cds_qp_solve_bracketed,
                      cds_qp_solve_bracketed_cached, cds_qp_solve_cached, cds_ri_factors,
                      cds_sigma2_diag, cds_sigma2_diag_cache, cds_version, cds_wait_check,
                      declared_symbols, load, npair)

__all__ = ["CdsError", "cds_acd_aux_pairs", "cds_cd_decompose", "cds_cd_decompose_shells",
           "cds_cd_decompose_to_mo", "cds_cd_gemm_time", "cds_cd_gemm_timing", "cds_cd_stats", "cds_cd_to_mo", "cds_eri_columns", "cds_eri_diag", "cds_launch_count",
           "cds_mp2_energy", "cds_qp_solve", "cds_qp_solve_bracketed",
           "cds_qp_solve_bracketed_cached", "cds_qp_solve_cached", "cds_ri_factors",
           "cds_sigma2_diag", "cds_sigma2_diag_cache", "cds_version", "cds_wait_check",
           "declared_symbols", "load", "npair"]
