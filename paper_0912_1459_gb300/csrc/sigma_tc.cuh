// Tensor-core (tcgen05, BF16 split-precision) path of the self-energy.
#pragma once

#include "sigma.cuh"

namespace cds {

size_t tc_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE);

int sigma2_tc(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
              int32_t np, const double* eps, const double* E, int32_t nE,
              const int32_t* active, double* sigma, double* dsigma, void* ws,
              cudaStream_t stream);

size_t sigma_ws_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE,
                      int32_t precision);

int sigma2_dispatch(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                    int32_t np, const double* eps, const double* E, int32_t nE,
                    int32_t precision, const int32_t* active, double* sigma, double* dsigma,
                    void* ws, cudaStream_t stream);

}  // namespace cds
