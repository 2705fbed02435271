// Tensor-core (tcgen05, split-precision BF16X3 / FP16X3 / TF32X3) path of the
// self-energy.
#pragma once

#include "sigma.cuh"

namespace cds {

size_t tc_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE,
                          bool tf32 = false);

// resplit = false reuses the 16-bit operand splits a previous call with the
// same Lov, Lp and workspace left in ws (the Newton iterations of one solve).
// cache (may be null): receives every work item's numerators
// (tc_cache_bytes), for sigma2_cached.
int sigma2_tc(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
              int32_t np, const double* eps, const double* E, int32_t nE,
              const int32_t* active, int32_t precision, double* sigma, double* dsigma, void* ws,
              cudaStream_t stream, bool resplit = true, float* cache = nullptr);
size_t tc_cache_bytes(int32_t nmo, int32_t nocc, int32_t np);
// Sigma and dSigma/dE at one energy per orbital (E [np]) from cached
// numerators; first = the first call of a solve (stages eps).
size_t tc_cached_workspace_bytes(int32_t nmo, int32_t nocc, int32_t np);
int sigma2_cached(int32_t nmo, int32_t nocc, int32_t np, const double* eps, const double* E,
                  const int32_t* active, const float* cache, double* sigma, double* dsigma,
                  void* ws, cudaStream_t stream, bool first);

// FP64 form of the same: k_sigma_fp64 stores each 32 x 32 item's numerators
// (fp64_cache_bytes) when given a cache, and sigma2_cached_fp64 evaluates
// Sigma at one energy per orbital from them (workspace
// fp64_cached_workspace_bytes).
size_t fp64_cache_bytes(int32_t nmo, int32_t nocc, int32_t np);
size_t fp64_cached_workspace_bytes(int32_t nmo, int32_t nocc, int32_t np);
int sigma2_cached_fp64(int32_t nmo, int32_t nocc, int32_t np, const double* eps, const double* E,
                       const int32_t* active, const double* cache, double* sigma, double* dsigma,
                       double* part, cudaStream_t stream);

// MP2 correlation energy (Eq. MP2) on the tensor-core kernel: e_pair[i] =
// sum_{j,a,b}, e_total = sum_i e_pair[i] (either may be null).
size_t tc_mp2_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M);
int mp2_tc(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* eps,
           int32_t precision, double* e_pair, double* e_total, void* ws, cudaStream_t stream);
// out[0] = sum of x[0..n) in a fixed order (nothing if out is null).
int sum_fixed(const double* x, int32_t n, double* out, cudaStream_t stream);

// One molecule of a batch (host side) and the element offsets of its arrays
// in the concatenated batch buffers.
struct BatchMol {
    int32_t nbf, nocc, np, nE, max_rank;
};
struct BatchOffsets {
    int64_t basis, pair, L, piv, C, eps, orb, E, ov, p;
};

size_t tc_batch_workspace_bytes(int32_t nmol, const BatchMol* mols);
int tc_batch_setup(int32_t nmol, const BatchMol* mols, const int32_t* M, int32_t precision,
                   void* ws, cudaStream_t stream);
int tc_batch_split(int32_t nmol, const BatchMol* mols, const int32_t* M, const BatchOffsets* off,
                   const double* Lov, const double* Lp, const double* eps, int32_t precision,
                   void* ws, cudaStream_t stream);
// cache_mode: 0 none, 1 the tensor-core pass also stores the numerators,
// 2 Sigma from the stored numerators (Newton passes only).
int tc_batch_pass(int32_t nmol, const BatchMol* mols, int32_t pass, int64_t nE_total,
                  int32_t max_nE, int64_t np_total, const double* E, const int32_t* active,
                  int32_t precision, double* sigma, double* dsigma, unsigned long long* stamps,
                  void* ws, cudaStream_t stream, int32_t cache_mode);
namespace tc {
int tune_newton_cache();   // CDS_TUNE_NEWTON_CACHE
int tune_cd_graph();       // CDS_TUNE_CD_GRAPH
int tune_pipe_split();     // CDS_TUNE_PIPE_SPLIT
int tune_grid_ec();        // CDS_TUNE_GRID_EC
}

inline bool is_split16(int32_t precision) {
    return precision == CDS_PREC_BF16X3 || precision == CDS_PREC_FP16X3;
}
// Split precisions of the single-molecule self-energy (also TF32X3).
inline bool is_split_tc(int32_t precision) {
    return is_split16(precision) || precision == CDS_PREC_TF32X3;
}

size_t sigma_ws_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE,
                      int32_t precision);

int sigma2_dispatch(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                    int32_t np, const double* eps, const double* E, int32_t nE,
                    int32_t precision, const int32_t* active, double* sigma, double* dsigma,
                    void* ws, cudaStream_t stream, bool resplit = true);

}  // namespace cds
