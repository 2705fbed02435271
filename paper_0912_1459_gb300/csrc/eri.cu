// Electron-repulsion integrals over s-type Gaussians (paper Sec. II.A,
// Eq. integral): pair data, the diagonal and on-the-fly columns.
#include "common.cuh"

namespace cds {

// Gaussian-product data of pair I from the basis (Sec. II.A).
__device__ __forceinline__ void pair_of(int64_t I, const double* __restrict__ xyz,
                                        const double* __restrict__ alpha, double& p,
                                        double& px, double& py, double& pz, double& kp) {
    int32_t mu, nu;
    unpack_pair(I, mu, nu);
    double am = alpha[mu], an = alpha[nu];
    double ax = xyz[3 * mu], ay = xyz[3 * mu + 1], az = xyz[3 * mu + 2];
    double bx = xyz[3 * nu], by = xyz[3 * nu + 1], bz = xyz[3 * nu + 2];
    p = am + an;
    double dx = ax - bx, dy = ay - by, dz = az - bz;
    double r2 = dx * dx + dy * dy + dz * dz;
    // normalisation (2a/pi)^(3/4) of each primitive
    double nm = pow(2.0 * am / kPi, 0.75), nn = pow(2.0 * an / kPi, 0.75);
    px = (am * ax + an * bx) / p;
    py = (am * ay + an * by) / p;
    pz = (am * az + an * bz) / p;
    kp = nm * nn * exp(-am * an / p * r2) / p;
}

__global__ void k_build_pairs(int32_t nbf, const double* __restrict__ xyz,
                              const double* __restrict__ alpha, PairSoA pd, int64_t npair) {
    int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= npair) return;
    double p, px, py, pz, k;
    pair_of(I, xyz, alpha, p, px, py, pz, k);
    pd.p[I] = p; pd.Px[I] = px; pd.Py[I] = py; pd.Pz[I] = pz; pd.Kp[I] = k;
}

int build_pairs(int32_t nbf, const double* xyz, const double* alpha, PairSoA pd,
                cudaStream_t stream) {
    int64_t n = npair_of(nbf);
    if (n == 0) return CDS_OK;
    int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    k_build_pairs<<<(unsigned)blocks, threads, 0, stream>>>(nbf, xyz, alpha, pd, n);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

__global__ void k_eri_diag(const double* __restrict__ xyz, const double* __restrict__ alpha,
                           int64_t npair, double* __restrict__ D) {
    int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= npair) return;
    double p, px, py, pz, k;
    pair_of(I, xyz, alpha, p, px, py, pz, k);
    D[I] = eri_pair(p, px, py, pz, k, p, px, py, pz, k);
}

__global__ void k_eri_columns(const double* __restrict__ xyz, const double* __restrict__ alpha,
                              int64_t npair, const int32_t* __restrict__ piv, int32_t ncol,
                              double* __restrict__ cols) {
    int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (I >= npair || c >= ncol) return;
    int64_t P = piv[c];
    double* out = cols + (int64_t)c * npair;
    if (P < 0 || P >= npair) { out[I] = __longlong_as_double(0x7ff8000000000000LL); return; }
    double p, px, py, pz, k, q, qx, qy, qz, kq;
    pair_of(I, xyz, alpha, p, px, py, pz, k);
    pair_of(P, xyz, alpha, q, qx, qy, qz, kq);
    out[I] = eri_pair(p, px, py, pz, k, q, qx, qy, qz, kq);
}

}  // namespace cds

using namespace cds;

extern "C" int cds_eri_diag(int32_t nbf, const double* xyz, const double* alpha, double* D,
                            cudaStream_t stream) {
    if (nbf < 0 || (nbf > 0 && (!xyz || !alpha || !D))) return CDS_ERR_ARG;
    int64_t n = npair_of(nbf);
    if (n == 0) return CDS_OK;
    k_eri_diag<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(xyz, alpha, n, D);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

extern "C" int cds_eri_columns(int32_t nbf, const double* xyz, const double* alpha,
                               const int32_t* piv, int32_t ncol, double* cols,
                               cudaStream_t stream) {
    if (nbf < 0 || ncol < 0 || ncol > 65535) return CDS_ERR_ARG;
    int64_t n = npair_of(nbf);
    if (n == 0 || ncol == 0) return CDS_OK;
    if (!xyz || !alpha || !piv || !cols) return CDS_ERR_ARG;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)ncol);
    k_eri_columns<<<grid, 256, 0, stream>>>(xyz, alpha, n, piv, ncol, cols);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}
