// Shared device/host helpers of libcdsigma (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <climits>
#include <algorithm>
#include <functional>

#include "cdsigma.h"
#include "boys_table.h"

#define CDS_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return CDS_ERR_CUDA;          \
    } while (0)

namespace cds {
// Kernel launches issued by this library in this process (see cds_launch_count).
void count_launches(unsigned long long n);
}

// Counts one launch and turns a launch error into CDS_ERR_CUDA.
#define CDS_LAUNCH_CHECK()                 \
    do {                                   \
        cds::count_launches(1);            \
        CDS_CUDA_TRY(cudaGetLastError());  \
    } while (0)

namespace cds {

constexpr double kTwoPi52 = 34.98683665524972;      // 2 pi^(5/2)
constexpr double kHalfSqrtPi = 0.88622692545275801;  // sqrt(pi)/2
constexpr double kPi = 3.14159265358979323846;

inline int64_t npair_of(int32_t nbf) { return (int64_t)nbf * (nbf + 1) / 2; }

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Carves consecutive 256-byte-aligned regions out of a caller workspace.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* p) : base(static_cast<char*>(p)) {}
    template <class T> T* take(size_t n) {
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off = align_up(off + n * sizeof(T));
        return p;
    }
};

// Gaussian-product data of every product density (Sec. II.A), structure of
// arrays so a warp reads consecutive pairs with coalesced loads.
struct PairSoA {
    double* p;    // exponent sum a_mu + a_nu
    double* Px;   // product centre
    double* Py;
    double* Pz;
    double* Kp;   // N_mu N_nu exp(-a_mu a_nu |A-B|^2 / p) / p
};

// Above T = 36 the Boys function needs no error function: erfc(6) ~ 2.2e-17 is
// below half an ulp of 1, so erf(sqrt T) rounds to exactly 1 in binary64.
constexpr double kErfOneT = 36.0;
constexpr double kPi3 = 31.006276680299816;   // pi^3 = 2 pi^(5/2) * sqrt(pi)/2

// (rho_I|rho_J) = 2 pi^(5/2) K_I K_J / (p q sqrt(p+q)) F0(T), T = x / s with
// x = p q |P-Q|^2 and s = p + q (Eq. integral, s-type).  The pair data hold
// K/p, so no division is needed.
__device__ __forceinline__ void eri_xs(double p, double px, double py, double pz, double q,
                                       double qx, double qy, double qz, double& x, double& s) {
    const double dx = px - qx, dy = py - qy, dz = pz - qz;
    x = p * q * (dx * dx + dy * dy + dz * dz);
    s = p + q;
}
// T >= kErfOneT: F0(T) = (1/2) sqrt(pi/T) exactly, and the integral reduces to
// pi^3 (K_I/p)(K_J/q) / sqrt(x) (the point-charge form).
__device__ __forceinline__ bool eri_is_far(double x, double s) { return x >= kErfOneT * s; }
__device__ __forceinline__ double eri_far(double kk, double x) { return kPi3 * kk * rsqrt(x); }
// T < kErfOneT: F0(T) from its Taylor expansion around the nearest point of a
// 1/16 grid (boys_table.h: F_0(T_i + d) = sum_m F_m(T_i) (-d)^m / m!, eight
// terms, truncation below 2e-18).  kk = (K_I/p)(K_J/q).
__device__ __forceinline__ double eri_near(double kk, double x, double s) {
    const double rs = rsqrt(s);
    const double T = x * (rs * rs);
    const int i = min(max(__double2int_rn(T * kBoysPerUnit), 0), kBoysPoints - 1);
    const double d = T - (double)i * (1.0 / kBoysPerUnit);
    const double* c = kBoysTaylor[i];
    double f = c[kBoysOrder - 1];
#pragma unroll
    for (int m = kBoysOrder - 2; m >= 0; --m) f = fma(f, d, c[m]);
    return kTwoPi52 * kk * rs * f;
}

// (rho_I|rho_J) from the pair data of both densities (Eq. integral, s-type).
__device__ __forceinline__ double eri_pair(double p, double px, double py, double pz,
                                           double kp, double q, double qx, double qy,
                                           double qz, double kq) {
    double x, s;
    eri_xs(p, px, py, pz, q, qx, qy, qz, x, s);
    return eri_is_far(x, s) ? eri_far(kp * kq, x) : eri_near(kp * kq, x, s);
}

// Decode a packed pair index I = nu(nu+1)/2 + mu into (mu, nu).
__device__ __forceinline__ void unpack_pair(int64_t I, int32_t& mu, int32_t& nu) {
    double r = sqrt(8.0 * (double)I + 1.0);
    int64_t n = (int64_t)((r - 1.0) * 0.5);
    while (n * (n + 1) / 2 > I) --n;
    while ((n + 1) * (n + 2) / 2 <= I) ++n;
    nu = (int32_t)n;
    mu = (int32_t)(I - n * (n + 1) / 2);
}

}  // namespace cds

// Internal entry points shared across translation units (not exported).
namespace cds {
int build_pairs(int32_t nbf, const double* xyz, const double* alpha, PairSoA pd,
                cudaStream_t stream);
// Workspace of cds_cd_decompose for one precision (f32x2 needs the candidate
// projections as well).
size_t cd_workspace_bytes_for(int32_t nbf, bool f32x2);
// Workspace of cds_cd_decompose for a precision (FP64, F32X2, or OZAKI: the
// tensor-core form, whose slice store holds max_rank columns).
size_t cd_workspace_bytes_prec(int32_t nbf, int32_t max_rank, int32_t precision);
// SM split of the pipelined decomposition + transform (cds_cd_decompose_to_mo
// sets it for the calling thread while it runs): the transform's tensor-core
// GEMMs take at most this many CTAs, the decomposition's projection GEMM the
// rest of the SMs; 0 = no split.
int& pipe_tr_ctas();
// Called after each host check of the decomposition: (rows of L final, stopped).
using CdChunkHook = std::function<int(int32_t, bool)>;
int cd_decompose_run(int32_t nbf, const double* xyz, const double* alpha, const int32_t* atom,
                     double delta, int32_t scheme, int32_t max_rank, int32_t precision, double* L,
                     int32_t* piv, double* D, int32_t* M_out, double* delta_eff_out,
                     void* workspace, size_t workspace_bytes, cudaStream_t stream,
                     const CdChunkHook* on_chunk, cudaStream_t convert_after,
                     bool chunk_graph = true, bool convert = true);
// Float pairs (hi, lo) of the first count elements of L back to FP64, in place.
int pairs_to_fp64(double* L, int64_t count, cudaStream_t stream);
}
