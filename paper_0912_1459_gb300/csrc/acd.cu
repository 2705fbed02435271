// Atomic Cholesky basis and the V-approximation built on it (paper Sec. II.A,
// atomic CD; Eq. int_approx, Eq. error_approx).
//
// The basis: for every unique atom (the exponents of the functions on one
// centre) the isolated atom's one-centre ERI matrix is decomposed with the
// threshold-delta pivoted Cholesky decomposition of cds_cd_decompose (same
// pivot rule); its pivots, as densities on each atom of that type, are the
// molecule's basis densities rho~_K.
// The factors: with the Coulomb metric V_KL = (rho~_K|rho~_L) = L_m L_m^T,
//   B = L_m^-1 (rho~|rho_I),   (rho_I|rho_J) ~ sum_K B^K_I B^K_J,
// the same factor form as Eq. CD, so the transform and the self-energy take
// B in place of the Cholesky vectors.
#include <algorithm>
#include <map>
#include <vector>

#include "common.cuh"
#include "eri_col.cuh"

namespace cds {
namespace {

struct AcdLayout {
    double* xyz;     // [na][3] zeros: the isolated atom at the origin
    double* alpha;   // [na]
    double* L;       // [npa][npa]
    int32_t* piv;    // [npa]
    double* D;       // [npa]
    void* cd;        // the isolated atom's decomposition workspace
    size_t cd_bytes;
    size_t bytes;
};

AcdLayout acd_layout(void* ws, int32_t na) {
    const int64_t npa = npair_of(na);
    Carver c(ws);
    AcdLayout l;
    l.xyz = c.take<double>((size_t)3 * std::max(na, 1));
    l.alpha = c.take<double>((size_t)std::max(na, 1));
    l.L = c.take<double>((size_t)std::max<int64_t>(npa * npa, 1));
    l.piv = c.take<int32_t>((size_t)std::max<int64_t>(npa, 1));
    l.D = c.take<double>((size_t)std::max<int64_t>(npa, 1));
    l.cd_bytes = cd_workspace_bytes_for(std::max(na, 1), false);
    l.cd = c.take<unsigned char>(l.cd_bytes);
    l.bytes = c.off;
    return l;
}

// The factors by forward substitution with the basis as fixed pivots:
//   B[k][I] = (X[k][I] - sum_{j<k} Lm[k][j] B[j][I]) / Lm[k][k],
// X[k] = (rho~_k|rho).  The metric's factor need not be formed first: B
// restricted to the basis' own columns is L_m^T, so Lm[k][j] = B[j][aux[k]]
// (j < k) once row j is final, and Lm[k][k] is the square root of the Schur
// complement X[k][aux[k]] - sum_j Lm[k][j]^2.  Rows go kRiR at a time:
// k_ri_panel gathers the finished part of their Lm rows and factors the
// kRiR x kRiR block of the Schur complement (FP64, a few hundred values);
// k_ri_rows then streams every earlier row once for all kRiR new rows.
// FP64 form: X is made in B and replaced row by row.  Float-pair form: X and
// the finished rows live as float pairs in the workspace (the operand the
// stream reads), and each finished row is also written to B in FP64.
constexpr int kRiR = 8;      // rows per pass
constexpr int kRiJ = 256;    // earlier rows staged per shared-memory tile
constexpr int kRiT = 256;    // threads per block
constexpr int kRiEriPasses = 4;   // integral kernel: passes of kRiT pairs per block

// A Cholesky pivot at or below kSingular x its metric diagonal: the metric is
// singular to working precision (e.g. a basis density listed twice) and B
// would carry 1e6 x the rounding or more.
constexpr double kSingular = 1e-12;

struct RiLayout {
    PairSoA pd;
    PairF2 pf;        // float-pair form only
    float2* Xf;       // [naux][n], float-pair form only
    double* Lrow;     // [kRiR][naux]
    float2* Lrowf;    // [kRiR][naux], float-pair form only
    double* Lblk;     // [kRiR][kRiR]: the block's factor (FP64 form)
    float2* Lblkf;    // [kRiR][kRiR]: -factor below the diagonal, 1/diagonal on it
    int32_t* status;
    size_t bytes;
};

RiLayout ri_layout(void* ws, int64_t n, int32_t naux, bool df) {
    Carver c(ws);
    RiLayout l{};
    const size_t nn = (size_t)std::max<int64_t>(n, 1), na = (size_t)std::max(naux, 1);
    l.pd = PairSoA{c.take<double>(nn), c.take<double>(nn), c.take<double>(nn),
                   c.take<double>(nn), c.take<double>(nn)};
    if (df) {
        l.pf = PairF2{c.take<float2>(nn), c.take<float2>(nn), c.take<float2>(nn),
                      c.take<float2>(nn), c.take<float2>(nn)};
        l.Xf = c.take<float2>(na * nn);
        l.Lrowf = c.take<float2>((size_t)kRiR * na);
        l.Lblkf = c.take<float2>((size_t)kRiR * kRiR);
    }
    l.Lrow = c.take<double>((size_t)kRiR * na);
    l.Lblk = c.take<double>((size_t)kRiR * kRiR);
    l.status = c.take<int32_t>(4);
    l.bytes = c.off;
    return l;
}

// Row y of X: (rho~_{aux[y]}|rho_I) for all I, FP64 into B or float pairs
// into Xf.
template <bool DF>
__global__ void __launch_bounds__(kRiT) k_ri_eri(PairSoA pd, PairF2 pf, int64_t n,
                                                 const int32_t* __restrict__ aux,
                                                 double* __restrict__ B, float2* __restrict__ Xf) {
    const int64_t P = aux[blockIdx.y];
    if (DF) eri_column_df<kRiT>(pd, pf, n, P, Xf + (int64_t)blockIdx.y * n, blockIdx.x, gridDim.x);
    else eri_column_fp64<kRiT>(pd, n, P, B + (int64_t)blockIdx.y * n, blockIdx.x, gridDim.x);
}

template <bool DF>
__device__ __forceinline__ double x_at(const double* B, const float2* Xf, int64_t e) {
    if (DF) {
        const float2 v = Xf[e];
        return (double)v.x + (double)v.y;
    }
    return B[e];
}

// Lrow[r][j] = B[j][aux[k0+r]] for j < k0 (final rows); the lower Cholesky
// factor of S[r][s] = X[k0+r][aux[k0+s]] - sum_j Lrow[r][j] Lrow[s][j]
// (s <= r < nr) into Lblk / Lblkf.  status = 1 on a pivot that is not finite
// or falls to kSingular x X[k0+r][aux[k0+r]].
template <bool DF>
__global__ void __launch_bounds__(kRiT) k_ri_panel(const double* __restrict__ B,
                                                   const float2* __restrict__ Xf, int64_t n,
                                                   const int32_t* __restrict__ aux, int32_t k0,
                                                   int32_t nr, RiLayout lay, int32_t naux_ld) {
    __shared__ double S[kRiR][kRiR];
    __shared__ double d0[kRiR];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int64_t e = tid; e < (int64_t)nr * k0; e += blockDim.x) {
        const int r = (int)(e / k0), j = (int)(e - (int64_t)r * k0);
        const double v = B[(int64_t)j * n + aux[k0 + r]];
        lay.Lrow[(int64_t)r * naux_ld + j] = v;
        if (DF) lay.Lrowf[(int64_t)r * naux_ld + j] = to_f2(v);
    }
    __syncthreads();
    // one warp per lower-triangle entry (r, s)
    for (int e = warp; e < nr * (nr + 1) / 2; e += blockDim.x / 32) {
        int r = 0;
        while ((r + 1) * (r + 2) / 2 <= e) ++r;
        const int s2 = e - r * (r + 1) / 2;
        const double* a = lay.Lrow + (int64_t)r * naux_ld;
        const double* b = lay.Lrow + (int64_t)s2 * naux_ld;
        double acc = 0.0;
        for (int j = lane; j < k0; j += 32) acc = fma(a[j], b[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double x = x_at<DF>(B, Xf, (int64_t)(k0 + r) * n + aux[k0 + s2]);
            S[r][s2] = x - acc;
            if (s2 == r) d0[r] = x;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int bad = 0;
        for (int j = 0; j < nr; ++j) {
            double d = S[j][j];
            for (int q = 0; q < j; ++q) d -= S[j][q] * S[j][q];
            if (!(d > kSingular * d0[j]) || !(d < INFINITY)) { bad = 1; d = 1.0; }
            S[j][j] = sqrt(d);
            for (int i = j + 1; i < nr; ++i) {
                double v = S[i][j];
                for (int q = 0; q < j; ++q) v -= S[i][q] * S[j][q];
                S[i][j] = v / S[j][j];
            }
        }
        for (int i = 0; i < kRiR; ++i)
            for (int j = 0; j < kRiR; ++j) {
                const bool in = i < nr && j <= i;
                lay.Lblk[i * kRiR + j] = in ? S[i][j] : 0.0;
                if (DF)
                    lay.Lblkf[i * kRiR + j] =
                        !in ? make_float2(0.f, 0.f) : (i == j ? to_f2(1.0 / S[i][i]) : to_f2(-S[i][j]));
            }
        if (bad) *lay.status = 1;
    }
}

// Rows k0 .. k0+nr-1 from X (in those rows) and the final rows j < k0.  One
// pair column I per thread: each earlier row is read once for all nr rows,
// then the kRiR x kRiR block is solved in registers.
__global__ void __launch_bounds__(kRiT) k_ri_rows(double* __restrict__ B, int64_t n, int32_t k0,
                                                  int32_t nr, const double* __restrict__ Lrow,
                                                  int32_t ldr, const double* __restrict__ Lblk) {
    __shared__ double ls[kRiJ][kRiR];
    __shared__ double lb[kRiR][kRiR];
    const int tid = threadIdx.x;
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + tid;
    const bool valid = I < n;
    double s[kRiR];
#pragma unroll
    for (int r = 0; r < kRiR; ++r) s[r] = 0.0;
    for (int j0 = 0; j0 < k0; j0 += kRiJ) {
        const int jn = min(kRiJ, k0 - j0);
        __syncthreads();
        for (int e = tid; e < kRiJ * kRiR; e += blockDim.x) {
            const int r = e / kRiJ, jj = e - r * kRiJ;
            ls[jj][r] = (r < nr && jj < jn) ? Lrow[(int64_t)r * ldr + j0 + jj] : 0.0;
        }
        __syncthreads();
        if (valid) {
            const double* col = B + (int64_t)j0 * n + I;
            for (int jj = 0; jj < jn; ++jj) {
                const double b = col[(int64_t)jj * n];
#pragma unroll
                for (int r = 0; r < kRiR; ++r) s[r] = fma(ls[jj][r], b, s[r]);
            }
        }
    }
    if (tid < kRiR * kRiR) lb[tid / kRiR][tid % kRiR] = Lblk[tid];
    __syncthreads();
    if (!valid) return;
    double bv[kRiR];
#pragma unroll
    for (int r = 0; r < kRiR; ++r) {
        if (r < nr) {
            double* out = B + (int64_t)(k0 + r) * n + I;
            double x = *out - s[r];
#pragma unroll
            for (int q = 0; q < r; ++q) x = fma(-lb[r][q], bv[q], x);
            bv[r] = x / lb[r][r];
            *out = bv[r];
        }
    }
}

// The same in float pairs: the earlier rows and X are read from Xf, each new
// row is written to Xf (float pairs) and to B (FP64).
__global__ void __launch_bounds__(kRiT) k_ri_rows_df(double* __restrict__ B,
                                                     float2* __restrict__ Xf, int64_t n,
                                                     int32_t k0, int32_t nr,
                                                     const float2* __restrict__ Lrowf, int32_t ldr,
                                                     const float2* __restrict__ Lblkf) {
    __shared__ float2 ls[kRiJ][kRiR];
    __shared__ float2 lb[kRiR][kRiR];
    const int tid = threadIdx.x;
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + tid;
    const bool valid = I < n;
    const float2 zero = make_float2(0.f, 0.f);
    float2 s[kRiR];
#pragma unroll
    for (int r = 0; r < kRiR; ++r) s[r] = zero;
    for (int j0 = 0; j0 < k0; j0 += kRiJ) {
        const int jn = min(kRiJ, k0 - j0);
        __syncthreads();
        for (int e = tid; e < kRiJ * kRiR; e += blockDim.x) {
            const int r = e / kRiJ, jj = e - r * kRiJ;
            ls[jj][r] = (r < nr && jj < jn) ? Lrowf[(int64_t)r * ldr + j0 + jj] : zero;
        }
        __syncthreads();
        if (valid) {
            const float2* col = Xf + (int64_t)j0 * n + I;
            for (int jj = 0; jj < jn; ++jj) {
                const float2 b = col[(int64_t)jj * n];
#pragma unroll
                for (int r = 0; r < kRiR; ++r) df_fma(s[r], ls[jj][r], b);
            }
        }
    }
    if (tid < kRiR * kRiR) lb[tid / kRiR][tid % kRiR] = Lblkf[tid];
    __syncthreads();
    if (!valid) return;
    float2 bv[kRiR];
#pragma unroll
    for (int r = 0; r < kRiR; ++r) {
        if (r < nr) {
            const int64_t e = (int64_t)(k0 + r) * n + I;
            float2 x = df_add(Xf[e], df_neg(s[r]));
#pragma unroll
            for (int q = 0; q < r; ++q) df_fma(x, lb[r][q], bv[q]);
            x = df_add(x, zero);   // renormalise after the accumulation
            bv[r] = df_mul(x, lb[r][r]);
            Xf[e] = bv[r];
            B[e] = (double)bv[r].x + (double)bv[r].y;
        }
    }
}

}  // namespace
}  // namespace cds

using namespace cds;

extern "C" size_t cds_acd_workspace_bytes(int32_t max_atom_funcs) {
    if (max_atom_funcs <= 0) return 0;
    return acd_layout(nullptr, max_atom_funcs).bytes;
}

extern "C" int cds_acd_aux_pairs(int32_t nbf, const double* alpha, const int32_t* atom,
                                 double delta, int32_t* aux, int32_t capacity, int32_t* naux,
                                 void* workspace, size_t workspace_bytes, cudaStream_t stream) {
    if (nbf <= 0 || !alpha || !atom || !aux || !naux || capacity < 0 || !(delta >= 0.0))
        return CDS_ERR_ARG;
    std::vector<double> a(nbf);
    std::vector<int32_t> at(nbf);
    CDS_CUDA_TRY(cudaMemcpyAsync(a.data(), alpha, sizeof(double) * nbf, cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaMemcpyAsync(at.data(), atom, sizeof(int32_t) * nbf, cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    // functions of each centre, centres ascending
    std::map<int32_t, std::vector<int32_t>> funcs;
    for (int32_t f = 0; f < nbf; ++f) funcs[at[f]].push_back(f);
    int32_t na_max = 0;
    for (auto& kv : funcs) na_max = std::max(na_max, (int32_t)kv.second.size());
    AcdLayout lay = acd_layout(workspace, na_max);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    std::map<std::vector<double>, std::vector<std::pair<int32_t, int32_t>>> picks;   // per type
    int32_t count = 0;
    for (auto& kv : funcs) {
        const std::vector<int32_t>& fs = kv.second;
        const int32_t na = (int32_t)fs.size();
        std::vector<double> key(na);
        for (int32_t i = 0; i < na; ++i) key[i] = a[fs[i]];
        auto it = picks.find(key);
        if (it == picks.end()) {
            // the isolated atom's decomposition, in this call's own workspace
            const int64_t npa = npair_of(na);
            std::vector<double> zeros(3 * (size_t)na, 0.0);
            CDS_CUDA_TRY(cudaMemcpyAsync(lay.xyz, zeros.data(), sizeof(double) * 3 * na,
                                         cudaMemcpyHostToDevice, stream));
            CDS_CUDA_TRY(cudaMemcpyAsync(lay.alpha, key.data(), sizeof(double) * na,
                                         cudaMemcpyHostToDevice, stream));
            int32_t M = 0;
            double de = 0.0;
            int st = cds_cd_decompose(na, lay.xyz, lay.alpha, nullptr, delta, CDS_SCHEME_FULL,
                                      (int32_t)npa, CDS_PREC_FP64, lay.L, lay.piv, lay.D, &M, &de,
                                      lay.cd, lay.cd_bytes, stream);
            if (st) return st;
            std::vector<int32_t> piv(M);
            if (M > 0)
                CDS_CUDA_TRY(cudaMemcpyAsync(piv.data(), lay.piv, sizeof(int32_t) * M,
                                             cudaMemcpyDeviceToHost, stream));
            CDS_CUDA_TRY(cudaStreamSynchronize(stream));
            std::vector<std::pair<int32_t, int32_t>> loc;
            for (int32_t P : piv) {   // packed local index -> (mu, nu), mu <= nu
                int32_t nu = 0;
                while ((int64_t)(nu + 1) * (nu + 2) / 2 <= P) ++nu;
                loc.push_back({P - nu * (nu + 1) / 2, nu});
            }
            it = picks.emplace(key, loc).first;
        }
        for (auto& mn : it->second) {
            const int32_t g1 = fs[mn.first], g2 = fs[mn.second];
            const int32_t lo = std::min(g1, g2), hi = std::max(g1, g2);
            if (count < capacity) aux[count] = (int32_t)((int64_t)hi * (hi + 1) / 2 + lo);
            ++count;
        }
    }
    *naux = count;
    return count > capacity ? CDS_ERR_CAPACITY : CDS_OK;
}

extern "C" size_t cds_ri_workspace_bytes(int32_t nbf, int32_t naux, int32_t precision) {
    if (nbf <= 0 || naux < 0) return 0;
    if (precision != CDS_PREC_FP64 && precision != CDS_PREC_F32X2) return 0;
    return ri_layout(nullptr, npair_of(nbf), naux, precision == CDS_PREC_F32X2).bytes;
}

extern "C" int cds_ri_factors(int32_t nbf, const double* xyz, const double* alpha,
                              const int32_t* aux, int32_t naux, int32_t precision, double* B,
                              void* workspace, size_t workspace_bytes, cudaStream_t stream) {
    if (nbf <= 0 || naux < 0 || !xyz || !alpha || (naux > 0 && (!aux || !B)))
        return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && precision != CDS_PREC_F32X2) return CDS_ERR_UNSUPPORTED;
    if (naux == 0) return CDS_OK;
    const bool df = precision == CDS_PREC_F32X2;
    const int64_t n = npair_of(nbf);
    RiLayout lay = ri_layout(workspace, n, naux, df);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    {   // every basis density must be a pair of this basis
        std::vector<int32_t> h(naux);
        CDS_CUDA_TRY(cudaMemcpyAsync(h.data(), aux, sizeof(int32_t) * naux, cudaMemcpyDeviceToHost,
                                     stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
        for (int32_t P : h)
            if (P < 0 || P >= n) return CDS_ERR_ARG;
    }
    int st = build_pairs(nbf, xyz, alpha, lay.pd, stream);
    if (st) return st;
    const unsigned gn = (unsigned)((n + kRiT - 1) / kRiT);
    if (df) {
        k_pairs_to_f2<<<gn, kRiT, 0, stream>>>(lay.pd, lay.pf, n);
        CDS_LAUNCH_CHECK();
    }
    // X = (rho~_K|rho_I), one block row of grid per basis density
    const unsigned ge = (unsigned)std::max<int64_t>(1, (n + (int64_t)kRiT * kRiEriPasses - 1) /
                                                           ((int64_t)kRiT * kRiEriPasses));
    for (int32_t y0 = 0; y0 < naux; y0 += 65535) {
        const unsigned gy = (unsigned)std::min(65535, naux - y0);
        if (df)
            k_ri_eri<true><<<dim3(ge, gy), kRiT, 0, stream>>>(lay.pd, lay.pf, n, aux + y0, nullptr,
                                                              lay.Xf + (int64_t)y0 * n);
        else
            k_ri_eri<false><<<dim3(ge, gy), kRiT, 0, stream>>>(lay.pd, lay.pf, n, aux + y0,
                                                               B + (int64_t)y0 * n, nullptr);
        CDS_LAUNCH_CHECK();
    }
    CDS_CUDA_TRY(cudaMemsetAsync(lay.status, 0, sizeof(int32_t), stream));
    for (int32_t k0 = 0; k0 < naux; k0 += kRiR) {
        const int32_t nr = std::min(kRiR, naux - k0);
        if (df) {
            k_ri_panel<true><<<1, kRiT, 0, stream>>>(B, lay.Xf, n, aux, k0, nr, lay, naux);
            k_ri_rows_df<<<gn, kRiT, 0, stream>>>(B, lay.Xf, n, k0, nr, lay.Lrowf, naux, lay.Lblkf);
        } else {
            k_ri_panel<false><<<1, kRiT, 0, stream>>>(B, nullptr, n, aux, k0, nr, lay, naux);
            k_ri_rows<<<gn, kRiT, 0, stream>>>(B, n, k0, nr, lay.Lrow, naux, lay.Lblk);
        }
    }
    count_launches(2ull * ((naux + kRiR - 1) / kRiR));
    CDS_CUDA_TRY(cudaGetLastError());
    int32_t h = 0;
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, lay.status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    return h ? CDS_ERR_NOT_PD : CDS_OK;
}
