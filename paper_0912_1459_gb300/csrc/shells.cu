// Electron-repulsion integrals over contracted Cartesian Gaussians (s, p, d),
// FP64, for the decomposition's on-the-fly columns (paper Eq. integral over
// the contracted shells of Sec. III).
//
// A basis function is chi(r) = sum_k c_k x_A^l y_A^m z_A^n exp(-a_k |r - A|^2)
// (l + m + n <= 2, coefficients carrying the normalisation).  Per primitive
// quartet the integral is the McMurchie-Davidson sum
//   (ab|cd) = 2 pi^(5/2) / (p q sqrt(p+q)) sum_tuv E^ab_tuv
//             sum_t'u'v' (-1)^(t'+u'+v') E^cd_t'u'v' R_{t+t', u+u', v+v'},
// with the Hermite expansion coefficients E_t^{ij} of each Cartesian
// product (one axis at a time, by their two-term recurrences) and the
// Hermite Coulomb integrals R_tuv = R^0_tuv, R^n_000 = (-2 alpha)^n F_n(T),
// R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{t,u,v} (u, v alike).
// The levels n are built from n = L down to 0 in one array, each level's
// entries in decreasing total order, which only reads lower totals of the
// level above.  The Boys function F_n(T), n <= 8: its power series
// F_n(T) = e^-T sum_k (2T)^k / ((2n+1)(2n+3)...(2n+2k+1)) for the highest n
// and the downward recurrence F_m = (2T F_{m+1} + e^-T) / (2m+1) for T <= 50,
// F_0 = sqrt(pi/T)/2 and the upward recurrence above (erf(sqrt T) = 1 to
// double precision there).  One thread per pair of basis functions.
#include <cmath>

#include "common.cuh"

namespace cds {
namespace sh {

constexpr int LMAX = 2;              // per function
constexpr int LTOT = 4 * LMAX;       // per quartet
constexpr int NR = (LTOT + 1) * (LTOT + 2) * (LTOT + 3) / 6;   // t + u + v <= 8

struct Basis {
    const double* xyz;     // [nbf][3]
    const int32_t* lmn;    // [nbf][3]
    const int32_t* start;  // [nbf + 1]
    const double* exps;
    const double* coefs;
};

__device__ __forceinline__ int ridx(int t, int u, int v) {
    const int s = t + u + v, w = u + v;
    return s * (s + 1) * (s + 2) / 6 + w * (w + 1) / 2 + v;
}

__device__ void boys_all(int nmax, double T, double* F) {
    if (T < 1e-14) {
        for (int m = 0; m <= nmax; ++m) F[m] = 1.0 / (2 * m + 1) - T / (2 * m + 3);
        return;
    }
    const double et = exp(-T);
    if (T > 50.0) {
        F[0] = 0.5 * sqrt(3.141592653589793 / T);
        for (int m = 0; m < nmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - et) / (2.0 * T);
        return;
    }
    double term = 1.0 / (2 * nmax + 1), sum = term;
    for (int k = 1; k < 400; ++k) {
        term *= 2.0 * T / (2 * nmax + 2 * k + 1);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    F[nmax] = et * sum;
    for (int m = nmax - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + et) / (2 * m + 1);
}

// E_t^{ij}, t = 0 .. i + j, for one axis (i, j <= LMAX).
__device__ void hermite_e(int i, int j, double a, double b, double A, double B, double* E) {
    const double p = a + b, P = (a * A + b * B) / p;
    const double XA = P - A, XB = P - B, h = 0.5 / p;
    double cur[2 * LMAX + 1], nxt[2 * LMAX + 1];
    for (int t = 0; t <= 2 * LMAX; ++t) cur[t] = 0.0;
    cur[0] = exp(-a * b / p * (A - B) * (A - B));
    int n = 0;   // cur holds E^{ii', 0}, degree n
    for (int ii = 0; ii < i; ++ii) {
        for (int t = 0; t <= n + 1; ++t) {
            double v = XA * (t <= n ? cur[t] : 0.0);
            if (t >= 1) v += h * cur[t - 1];
            if (t + 1 <= n) v += (t + 1) * cur[t + 1];
            nxt[t] = v;
        }
        ++n;
        for (int t = 0; t <= n; ++t) cur[t] = nxt[t];
    }
    for (int jj = 0; jj < j; ++jj) {
        for (int t = 0; t <= n + 1; ++t) {
            double v = XB * (t <= n ? cur[t] : 0.0);
            if (t >= 1) v += h * cur[t - 1];
            if (t + 1 <= n) v += (t + 1) * cur[t + 1];
            nxt[t] = v;
        }
        ++n;
        for (int t = 0; t <= n; ++t) cur[t] = nxt[t];
    }
    for (int t = 0; t <= i + j; ++t) E[t] = cur[t];
}

// (mu nu|lam sig) over the contracted functions.
__device__ double contracted_eri(const Basis& b, int mu, int nu, int lam, int sig) {
    const int la[3] = {b.lmn[3 * mu], b.lmn[3 * mu + 1], b.lmn[3 * mu + 2]};
    const int lb[3] = {b.lmn[3 * nu], b.lmn[3 * nu + 1], b.lmn[3 * nu + 2]};
    const int lc[3] = {b.lmn[3 * lam], b.lmn[3 * lam + 1], b.lmn[3 * lam + 2]};
    const int ld[3] = {b.lmn[3 * sig], b.lmn[3 * sig + 1], b.lmn[3 * sig + 2]};
    const double* A = b.xyz + 3 * mu;
    const double* B = b.xyz + 3 * nu;
    const double* C = b.xyz + 3 * lam;
    const double* D = b.xyz + 3 * sig;
    int nab[3], ncd[3];
    for (int x = 0; x < 3; ++x) { nab[x] = la[x] + lb[x]; ncd[x] = lc[x] + ld[x]; }
    const int L = nab[0] + nab[1] + nab[2] + ncd[0] + ncd[1] + ncd[2];
    double total = 0.0;
    double R[NR], F[LTOT + 1];
    for (int i = b.start[mu]; i < b.start[mu + 1]; ++i)
        for (int j = b.start[nu]; j < b.start[nu + 1]; ++j) {
            const double ea = b.exps[i], eb = b.exps[j], p = ea + eb;
            double Eab[3][2 * LMAX + 1];
            for (int x = 0; x < 3; ++x) hermite_e(la[x], lb[x], ea, eb, A[x], B[x], Eab[x]);
            double P[3];
            for (int x = 0; x < 3; ++x) P[x] = (ea * A[x] + eb * B[x]) / p;
            const double cij = b.coefs[i] * b.coefs[j];
            for (int k = b.start[lam]; k < b.start[lam + 1]; ++k)
                for (int l = b.start[sig]; l < b.start[sig + 1]; ++l) {
                    const double ec = b.exps[k], ed = b.exps[l], q = ec + ed;
                    double Ecd[3][2 * LMAX + 1];
                    for (int x = 0; x < 3; ++x) hermite_e(lc[x], ld[x], ec, ed, C[x], D[x], Ecd[x]);
                    double X[3];
                    for (int x = 0; x < 3; ++x) X[x] = P[x] - (ec * C[x] + ed * D[x]) / q;
                    const double alpha = p * q / (p + q);
                    boys_all(L, alpha * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]), F);
                    // R^n for n = L .. 0 in place: totals L - n down to 0
                    double pw = 1.0;
                    for (int n = 0; n < L; ++n) pw *= -2.0 * alpha;
                    R[0] = pw * F[L];
                    for (int n = L - 1; n >= 0; --n) {
                        for (int s = L - n; s >= 1; --s)
                            for (int t = s; t >= 0; --t)
                                for (int u = s - t; u >= 0; --u) {
                                    const int v = s - t - u;
                                    double val;
                                    if (t > 0)
                                        val = (t > 1 ? (t - 1) * R[ridx(t - 2, u, v)] : 0.0) +
                                              X[0] * R[ridx(t - 1, u, v)];
                                    else if (u > 0)
                                        val = (u > 1 ? (u - 1) * R[ridx(t, u - 2, v)] : 0.0) +
                                              X[1] * R[ridx(t, u - 1, v)];
                                    else
                                        val = (v > 1 ? (v - 1) * R[ridx(t, u, v - 2)] : 0.0) +
                                              X[2] * R[ridx(t, u, v - 1)];
                                    R[ridx(t, u, v)] = val;
                                }
                        pw /= -2.0 * alpha;
                        R[0] = pw * F[n];
                    }
                    double sum = 0.0;
                    for (int t = 0; t <= nab[0]; ++t)
                        for (int u = 0; u <= nab[1]; ++u)
                            for (int v = 0; v <= nab[2]; ++v) {
                                const double e1 = Eab[0][t] * Eab[1][u] * Eab[2][v];
                                double inner = 0.0;
                                for (int t2 = 0; t2 <= ncd[0]; ++t2)
                                    for (int u2 = 0; u2 <= ncd[1]; ++u2)
                                        for (int v2 = 0; v2 <= ncd[2]; ++v2) {
                                            const double e2 = Ecd[0][t2] * Ecd[1][u2] * Ecd[2][v2];
                                            const double r = R[ridx(t + t2, u + u2, v + v2)];
                                            inner += ((t2 + u2 + v2) & 1) ? -e2 * r : e2 * r;
                                        }
                                sum += e1 * inner;
                            }
                    total += cij * b.coefs[k] * b.coefs[l] * 2.0 * 3.141592653589793 *
                             3.141592653589793 * sqrt(3.141592653589793) /
                             (p * q * sqrt(p + q)) * sum;
                }
        }
    return total;
}

__global__ void k_shell_diag(Basis b, int64_t n, double* __restrict__ D) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= n) return;
    int32_t mu, nu;
    unpack_pair(I, mu, nu);
    D[I] = contracted_eri(b, mu, nu, mu, nu);
}

// ecol[I] = (rho_I | rho_P), P read from the pivot slot (skipped once the
// decomposition has stopped, *done != 0).
__global__ void k_shell_column(Basis b, int64_t n, const int64_t* __restrict__ Pp,
                               const int32_t* __restrict__ done, double* __restrict__ ecol) {
    if (*done) return;
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= n) return;
    int32_t mu, nu, lam, sig;
    unpack_pair(I, mu, nu);
    unpack_pair(*Pp, lam, sig);
    ecol[I] = contracted_eri(b, mu, nu, lam, sig);
}

}  // namespace sh

int shell_diag(int32_t nbf, const double* xyz, const int32_t* lmn, const int32_t* start,
               const double* exps, const double* coefs, double* D, cudaStream_t stream) {
    const sh::Basis b{xyz, lmn, start, exps, coefs};
    const int64_t n = npair_of(nbf);
    sh::k_shell_diag<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(b, n, D);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

int shell_column(int32_t nbf, const double* xyz, const int32_t* lmn, const int32_t* start,
                 const double* exps, const double* coefs, const int64_t* P, const int32_t* done,
                 double* ecol, cudaStream_t stream) {
    const sh::Basis b{xyz, lmn, start, exps, coefs};
    const int64_t n = npair_of(nbf);
    sh::k_shell_column<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(b, n, P, done, ecol);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

}  // namespace cds
