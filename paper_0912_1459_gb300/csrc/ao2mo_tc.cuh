// Tensor-core (tcgen05, split-precision TF32X3 / BF16X3) AO->MO transform.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace cds {

// Workspace for batches of at most kb_max vectors (precision CDS_PREC_TF32X3
// or CDS_PREC_BF16X3).
size_t tr_tc_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max,
                             int32_t precision);
// Split C into the operand rows (once per call; also clears the error word).
int tr_tc_columns(int32_t nbf, int32_t nmo, int32_t nocc, const double* C, const int32_t* orb,
                  int32_t np, int32_t kb_max, int32_t precision, void* ws, cudaStream_t stream);
// Vectors [K0, K0 + kb) (FP64 rows of L, or float-pair rows Lf when given)
// into Lov[i][a][K] and Lp[t][q][K], K stride ldK.
int tr_tc_batch(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, const double* L,
                const float2* Lf, int32_t K0, int32_t kb, int64_t ldK, double* Lov, double* Lp,
                int32_t kb_max, int32_t precision, void* ws, cudaStream_t stream);
// Blocking: the kernels' error word (0, or CDS_ERR_TIMEOUT from a bounded wait).
int tr_tc_status(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max,
                 int32_t precision, void* ws, cudaStream_t stream);

// The split-precision GEMM of the transform as a building block (precision
// CDS_PREC_TF32X3 or CDS_PREC_BF16X3): D[m][c] = sum_k A[m][k] B[c][k] with
// both operands given as split hi/lo rows (k contiguous, row stride ld
// elements, 16-byte aligned rows), a_rows x kdim and b_rows x kdim; FP64
// output element (m, c) at out[(m / kdiv) rs_hi + (m % kdiv) rs_lo + c cs],
// written or (accumulate) added.  Asynchronous; the kernel's error word is
// err (device int32, cleared by the caller).
int tr_split_gemm(int32_t precision, const void* a_hi, const void* a_lo, int64_t a_rows,
                  const void* b_hi, const void* b_lo, int64_t b_rows, int32_t kdim, int32_t ld,
                  int64_t kdiv, int64_t rs_hi, int64_t rs_lo, int64_t cs, double* out,
                  bool accumulate, int32_t* err, cudaStream_t stream);

// Exact-slice (Ozaki) form, CDS_PREC_OZAKI: nbf <= 1040.
size_t tr_oz_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max);
int tr_oz_columns(int32_t nbf, int32_t nmo, int32_t nocc, const double* C, const int32_t* orb,
                  int32_t np, int32_t kb_max, void* ws, cudaStream_t stream);
int tr_oz_batch(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, const double* L,
                const float2* Lf, int32_t K0, int32_t kb, int64_t ldK, double* Lov, double* Lp,
                int32_t kb_max, void* ws, cudaStream_t stream);
int tr_oz_status(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max, void* ws,
                 cudaStream_t stream);

// Tensor-core transform of any kind: columns once, then batches, then the
// error word (precision CDS_PREC_TF32X3, CDS_PREC_BF16X3 or CDS_PREC_OZAKI).
inline int tr_any_columns(int32_t precision, int32_t nbf, int32_t nmo, int32_t nocc,
                          const double* C, const int32_t* orb, int32_t np, int32_t kb_max, void* ws,
                          cudaStream_t stream) {
    return precision == CDS_PREC_OZAKI
               ? tr_oz_columns(nbf, nmo, nocc, C, orb, np, kb_max, ws, stream)
               : tr_tc_columns(nbf, nmo, nocc, C, orb, np, kb_max, precision, ws, stream);
}
inline int tr_any_batch(int32_t precision, int32_t nbf, int32_t nmo, int32_t nocc, int32_t np,
                        const double* L, const float2* Lf, int32_t K0, int32_t kb, int64_t ldK,
                        double* Lov, double* Lp, int32_t kb_max, void* ws, cudaStream_t stream) {
    return precision == CDS_PREC_OZAKI
               ? tr_oz_batch(nbf, nmo, nocc, np, L, Lf, K0, kb, ldK, Lov, Lp, kb_max, ws, stream)
               : tr_tc_batch(nbf, nmo, nocc, np, L, Lf, K0, kb, ldK, Lov, Lp, kb_max, precision, ws,
                             stream);
}
inline int tr_any_status(int32_t precision, int32_t nbf, int32_t nmo, int32_t nocc, int32_t np,
                         int32_t kb_max, void* ws, cudaStream_t stream) {
    return precision == CDS_PREC_OZAKI
               ? tr_oz_status(nbf, nmo, nocc, np, kb_max, ws, stream)
               : tr_tc_status(nbf, nmo, nocc, np, kb_max, precision, ws, stream);
}
inline size_t tr_any_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np,
                                     int32_t kb_max) {
    return std::max(tr_tc_workspace_bytes(nbf, nmo, nocc, np, kb_max, CDS_PREC_TF32X3),
                    tr_oz_workspace_bytes(nbf, nmo, nocc, np, kb_max));
}

inline bool is_tr_tc(int32_t precision) {
    return precision == CDS_PREC_TF32X3 || precision == CDS_PREC_BF16X3 ||
           precision == CDS_PREC_OZAKI;
}

}  // namespace cds
