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

namespace cds {
namespace {

struct AcdLayout {
    double* xyz;     // [na][3] zeros: the isolated atom at the origin
    double* alpha;   // [na]
    double* L;       // [npa][npa]
    int32_t* piv;    // [npa]
    double* D;       // [npa]
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
    l.bytes = c.off;
    return l;
}

// V[k][l] = cols[k][aux[l]] (the metric from the basis densities' columns);
// d0[k] = V[k][k].
__global__ void k_gather_metric(const double* __restrict__ cols, int64_t npair,
                                const int32_t* __restrict__ aux, int32_t naux,
                                double* __restrict__ V, double* __restrict__ d0) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)naux * naux) return;
    const int32_t k = (int32_t)(e / naux), l = (int32_t)(e - (int64_t)k * naux);
    const double v = cols[(int64_t)k * npair + aux[l]];
    V[e] = v;
    if (k == l) d0[k] = v;
}

// In-place lower Cholesky factor of the small metric (one block, right-
// looking).  status: 0, or 1 if a pivot is not finite or falls to
// kSingular x its original diagonal d0: the metric is then singular to
// working precision (e.g. a basis density listed twice) and B would carry
// errors of 1e6 x the rounding or more.
constexpr double kSingular = 1e-12;
__global__ void __launch_bounds__(256) k_chol_small(double* __restrict__ V, int32_t n,
                                                    const double* __restrict__ d0,
                                                    int32_t* __restrict__ status) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int32_t j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            const double d = V[(int64_t)j * n + j];
            if (!(d > kSingular * d0[j]) || !(d < INFINITY)) bad = 1;
            else V[(int64_t)j * n + j] = sqrt(d);
        }
        __syncthreads();
        if (bad) break;
        const double djj = V[(int64_t)j * n + j];
        for (int32_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) V[(int64_t)i * n + j] /= djj;
        __syncthreads();
        // trailing lower triangle: V[i][k] -= V[i][j] V[k][j], j < k <= i
        const int64_t m = n - 1 - j;
        for (int64_t e = threadIdx.x; e < m * (m + 1) / 2; e += blockDim.x) {
            int64_t r = (int64_t)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
            while (r * (r + 1) / 2 > e) --r;
            while ((r + 1) * (r + 2) / 2 <= e) ++r;
            const int32_t i = j + 1 + (int32_t)r, k = j + 1 + (int32_t)(e - r * (r + 1) / 2);
            V[(int64_t)i * n + k] -= V[(int64_t)i * n + j] * V[(int64_t)k * n + j];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *status = bad;
}

// Row k of the forward substitution, in place:
//   B[k][I] = (B[k][I] - sum_{j<k} Lm[k][j] B[j][I]) / Lm[k][k]
// (rows j < k are final).  The row of Lm is staged in shared memory.
constexpr int kRiRow = 4096;
__global__ void __launch_bounds__(256) k_ri_row(const double* __restrict__ Lm, int32_t naux,
                                                int32_t k, double* __restrict__ B, int64_t n) {
    __shared__ double lk[kRiRow];
    for (int j = threadIdx.x; j <= k; j += blockDim.x) lk[j] = Lm[(int64_t)k * naux + j];
    __syncthreads();
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= n) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    int j = 0;
    for (; j + 4 <= k; j += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = fma(lk[j + u], B[(int64_t)(j + u) * n + I], s[u]);
    }
    for (; j < k; ++j) s[0] = fma(lk[j], B[(int64_t)j * n + I], s[0]);
    double* b = B + (int64_t)k * n + I;
    *b = (*b - ((s[0] + s[1]) + (s[2] + s[3]))) / lk[k];
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
            // the isolated atom's decomposition (allocation-free entry point)
            const int64_t npa = npair_of(na);
            std::vector<double> zeros(3 * (size_t)na, 0.0);
            CDS_CUDA_TRY(cudaMemcpyAsync(lay.xyz, zeros.data(), sizeof(double) * 3 * na,
                                         cudaMemcpyHostToDevice, stream));
            CDS_CUDA_TRY(cudaMemcpyAsync(lay.alpha, key.data(), sizeof(double) * na,
                                         cudaMemcpyHostToDevice, stream));
            int32_t M = 0;
            double de = 0.0;
            int st = cds_cd_decompose_static(na, lay.xyz, lay.alpha, nullptr, delta,
                                             CDS_SCHEME_FULL, (int32_t)npa, lay.L, lay.piv, lay.D,
                                             &M, &de, stream);
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

extern "C" size_t cds_ri_workspace_bytes(int32_t naux) {
    if (naux < 0) return 0;
    Carver c(nullptr);
    c.take<double>((size_t)std::max<int64_t>((int64_t)naux * naux, 1));
    c.take<double>((size_t)std::max(naux, 1));
    c.take<int32_t>(4);
    return c.off;
}

extern "C" int cds_ri_factors(int32_t nbf, const double* xyz, const double* alpha,
                              const int32_t* aux, int32_t naux, double* B, void* workspace,
                              size_t workspace_bytes, cudaStream_t stream) {
    if (nbf <= 0 || naux < 0 || naux > 65535 || naux > kRiRow || !xyz || !alpha ||
        (naux > 0 && (!aux || !B)))
        return CDS_ERR_ARG;
    if (naux == 0) return CDS_OK;
    if (!workspace || workspace_bytes < cds_ri_workspace_bytes(naux)) return CDS_ERR_WORKSPACE;
    Carver c(workspace);
    double* V = c.take<double>((size_t)naux * naux);
    double* d0 = c.take<double>((size_t)naux);
    int32_t* status = c.take<int32_t>(4);
    const int64_t n = npair_of(nbf);
    {   // every basis density must be a pair of this basis
        std::vector<int32_t> h(naux);
        CDS_CUDA_TRY(cudaMemcpyAsync(h.data(), aux, sizeof(int32_t) * naux, cudaMemcpyDeviceToHost,
                                     stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
        for (int32_t P : h)
            if (P < 0 || P >= n) return CDS_ERR_ARG;
    }
    int st = cds_eri_columns(nbf, xyz, alpha, aux, naux, B, stream);   // (rho~_K|rho_I)
    if (st) return st;
    const int64_t nn = (int64_t)naux * naux;
    k_gather_metric<<<(unsigned)((nn + 255) / 256), 256, 0, stream>>>(B, n, aux, naux, V, d0);
    CDS_LAUNCH_CHECK();
    k_chol_small<<<1, 256, 0, stream>>>(V, naux, d0, status);
    CDS_LAUNCH_CHECK();
    int32_t h = 0;
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    if (h) return CDS_ERR_NOT_PD;
    const unsigned g = (unsigned)((n + 255) / 256);
    for (int32_t k = 0; k < naux; ++k) {
        k_ri_row<<<g, 256, 0, stream>>>(V, naux, k, B, n);
    }
    count_launches((unsigned long long)naux);
    CDS_CUDA_TRY(cudaGetLastError());
    return CDS_OK;
}
