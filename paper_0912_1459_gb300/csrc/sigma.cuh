// Work decomposition of the diagonal self-energy (paper Eq. SE), shared by the
// FP64 and tensor-core paths.
//
// Both sums of Eq. SE have one shape.  For orbital q, a "spectator" index s
// and two "pair" indices x, y from the other orbital space,
//   X_xy = sum_J L^J_qx L^J_sy,
//   term = sum_s sum_{x,y} (2 X_xy - X_yx) X_xy / (E + e_s - e_x - e_y),
// first sum (2h1p): s = a (virtual), x, y = i, j (occupied);
// second sum (2p1h): s = i (occupied), x, y = a, b (virtual).
//
// Exchange pairing: the x range is cut into blocks of TB; a work item is
// (orbital t, spectator s, block pair A <= B).  It computes the two tiles
//   X1[x][y] = sum_J Aq[x][J] Bs[y][J]    (x in A, y in B)  = X_xy
//   X2[x][y] = sum_J Bs[x][J] Aq[y][J]    (x in A, y in B)  = X_yx
// so every thread sees X_xy and X_yx of the same (x, y).  For A < B the item
// covers the ordered pairs (x,y) and (y,x) at once with the shared
// denominator and numerator 2 X_xy^2 + 2 X_yx^2 - 2 X_xy X_yx; for A == B it
// uses (2 X_xy - X_yx) X_xy over all (x, y) in the block.
#pragma once

#include "common.cuh"

namespace cds {

struct SigmaTerm {
    const double* Aq;   // orbital rows: Aq + t*sAt + x*sAx + J
    int64_t sAt, sAx;
    const double* Bk;   // spectator rows: Bk + s*sBs + y*sBy + J
    int64_t sBs, sBy;
    const double* eps_s;  // [ns]
    const double* eps_x;  // [nx]
    int32_t nx, ns;
};

__host__ __device__ inline int32_t nblocks_of(int32_t nx, int32_t tb) { return (nx + tb - 1) / tb; }
__host__ __device__ inline int64_t npairs_of(int32_t nb) { return (int64_t)nb * (nb + 1) / 2; }

// Block pair (A <= B) of a pair index, rows of the upper triangle in order.
__host__ __device__ inline void block_pair(int64_t pb, int32_t nb, int32_t& A, int32_t& B) {
    int32_t a = 0;
    int64_t rem = pb;
    while (rem >= nb - a) { rem -= nb - a; ++a; }
    A = a;
    B = a + (int32_t)rem;
}

}  // namespace cds
