// Diagonal second-order self-energy Sigma_qq(E) and dSigma/dE (paper Eq. SE,
// Eq. ps): FP64 path, the deterministic cross-tile reduction, and the entry
// point that dispatches on precision.
//
// MO integrals are formed tile by tile from the factors (paper Sec. III:
// recomputed from Eq. CD at every evaluation) and reduced with the energy
// denominators in the same kernel; no o^2 v^2 integral array exists.
#include "sigma.cuh"
#include "sigma_tc.cuh"

namespace cds {

constexpr int kTB64 = 32;   // pair-index block of the FP64 path
constexpr int kJK64 = 16;   // J depth per shared-memory stage
constexpr int kEChunk = 64; // energies reduced per pass over the tile
constexpr int64_t kCacheItem64 = kTB64 * kTB64;   // cached numerators per FP64 work item

// One work item per block: two 32x32 FP64 tiles over all J, then the fused
// denominator-weighted reduction for every energy.
__global__ void __launch_bounds__(256)
k_sigma_fp64(SigmaTerm tm, int32_t M, int32_t nE, const double* __restrict__ E,
             const int32_t* __restrict__ active, int64_t item0, double* __restrict__ part,
             double* __restrict__ cache) {
    __shared__ double sred[8][kEChunk][2];   // per-warp partial sums
    __shared__ double sA1[kTB64][kJK64 + 1], sB1[kTB64][kJK64 + 1];
    __shared__ double sA2[kTB64][kJK64 + 1], sB2[kTB64][kJK64 + 1];
    const int32_t nb = nblocks_of(tm.nx, kTB64);
    const int64_t npb = npairs_of(nb);
    const int64_t item = blockIdx.x;
    const int32_t t = (int32_t)(item / (tm.ns * npb));
    const int64_t r = item - (int64_t)t * tm.ns * npb;
    const int32_t s = (int32_t)(r / npb);
    int32_t A, B;
    block_pair(r - (int64_t)s * npb, nb, A, B);
    double* out = part + (item0 + item) * (int64_t)nE * 2;
    if (active && !active[t]) return;

    const double* aq = tm.Aq + t * tm.sAt;
    const double* bk = tm.Bk + s * tm.sBs;
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;
    double acc1[2][2] = {}, acc2[2][2] = {};
    for (int J0 = 0; J0 < M; J0 += kJK64) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            int idx = tid + 256 * rr;
            int row = idx / kJK64, c = idx % kJK64;
            int J = J0 + c;
            int xa = A * kTB64 + row, xb = B * kTB64 + row;
            bool okJ = J < M;
            bool oka = okJ && xa < tm.nx, okb = okJ && xb < tm.nx;
            sA1[row][c] = oka ? aq[xa * tm.sAx + J] : 0.0;
            sA2[row][c] = oka ? bk[xa * tm.sBy + J] : 0.0;
            sB1[row][c] = okb ? bk[xb * tm.sBy + J] : 0.0;
            sB2[row][c] = okb ? aq[xb * tm.sAx + J] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kJK64; ++c) {
            double a1[2], a2[2], b1[2], b2[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) { a1[i] = sA1[tr * 2 + i][c]; a2[i] = sA2[tr * 2 + i][c]; }
#pragma unroll
            for (int j = 0; j < 2; ++j) { b1[j] = sB1[tc * 2 + j][c]; b2[j] = sB2[tc * 2 + j][c]; }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    acc1[i][j] = fma(a1[i], b1[j], acc1[i][j]);
                    acc2[i][j] = fma(a2[i], b2[j], acc2[i][j]);
                }
        }
        __syncthreads();
    }
    // numerators and E-independent part of the denominators
    const double es = tm.eps_s[s];
    double num[4], base[4];
    bool ok[4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            int x = A * kTB64 + tr * 2 + i, y = B * kTB64 + tc * 2 + j;
            int e = i * 2 + j;
            ok[e] = x < tm.nx && y < tm.nx;
            double x1 = acc1[i][j], x2 = acc2[i][j];
            num[e] = (A == B) ? (2.0 * x1 - x2) * x1 : 2.0 * (x1 * x1 + x2 * x2 - x1 * x2);
            base[e] = ok[e] ? es - tm.eps_x[x] - tm.eps_x[y] : 0.0;
        }
    if (cache) {   // the numerators of this item, [element k][thread] (coalesced)
        double* c = cache + (item0 + item) * kCacheItem64;
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k * 256 + tid] = num[k];
    }
    const int lane = tid & 31, w = tid >> 5;
    for (int e0 = 0; e0 < nE; e0 += kEChunk) {
        const int ne = min(kEChunk, nE - e0);
        for (int e = 0; e < ne; ++e) {
            double Ee = E[(int64_t)t * nE + e0 + e];
            double sv = 0.0, dv = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!ok[k]) continue;
                double rcp = 1.0 / (Ee + base[k]);
                double nr = num[k] * rcp;
                sv += nr;
                dv -= nr * rcp;
            }
            for (int o = 16; o; o >>= 1) {
                sv += __shfl_xor_sync(0xffffffffu, sv, o);
                dv += __shfl_xor_sync(0xffffffffu, dv, o);
            }
            if (lane == 0) { sred[w][e][0] = sv; sred[w][e][1] = dv; }
        }
        __syncthreads();
        for (int e = tid; e < ne; e += blockDim.x) {
            double sv = 0.0, dv = 0.0;
            for (int ww = 0; ww < 8; ++ww) { sv += sred[ww][e][0]; dv += sred[ww][e][1]; }
            out[(e0 + e) * 2] = sv;
            out[(e0 + e) * 2 + 1] = dv;
        }
        __syncthreads();
    }
}

// sigma[t][e] = sum over both terms' items of orbital t, fixed order.
__global__ void k_sigma_reduce(const double* __restrict__ part, int64_t per_t0, int64_t off1,
                               int64_t per_t1, int32_t nE, const int32_t* __restrict__ active,
                               double* __restrict__ sigma, double* __restrict__ dsigma) {
    const int t = blockIdx.y, e = blockIdx.x;
    if (active && !active[t]) return;
    double sv = 0.0, dv = 0.0;
    for (int64_t i = threadIdx.x; i < per_t0 + per_t1; i += blockDim.x) {
        int64_t item = i < per_t0 ? (int64_t)t * per_t0 + i : off1 + (int64_t)t * per_t1 + (i - per_t0);
        sv += part[(item * nE + e) * 2];
        dv += part[(item * nE + e) * 2 + 1];
    }
    __shared__ double ss[32], sd[32];
    for (int o = 16; o; o >>= 1) {
        sv += __shfl_xor_sync(0xffffffffu, sv, o);
        dv += __shfl_xor_sync(0xffffffffu, dv, o);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { ss[w] = sv; sd[w] = dv; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += ss[i]; b += sd[i]; }
        sigma[(int64_t)t * nE + e] = a;
        if (dsigma) dsigma[(int64_t)t * nE + e] = b;
    }
}

// Sigma and dSigma/dE at one energy per orbital (E[t]) from the numerators a
// k_sigma_fp64 pass stored: per element the arithmetic of k_sigma_fp64's
// epilogue (same denominator, same order of sums), so the result equals the
// recomputing kernel's at the same energy bit for bit; streams 8 KB per item
// instead of recomputing the integrals.
__global__ void __launch_bounds__(256)
k_sigma_fp64_cached(SigmaTerm tm, const double* __restrict__ E, const int32_t* __restrict__ active,
                    int64_t item0, int64_t nitems, const double* __restrict__ cache,
                    double* __restrict__ part) {
    __shared__ double sred[8][2];
    const int32_t nb = nblocks_of(tm.nx, kTB64);
    const int64_t npb = npairs_of(nb);
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const int lane = tid & 31, w = tid >> 5;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int32_t t = (int32_t)(item / (tm.ns * npb));
        const int64_t r = item - (int64_t)t * tm.ns * npb;
        const int32_t s = (int32_t)(r / npb);
        int32_t A, B;
        block_pair(r - (int64_t)s * npb, nb, A, B);
        if (active && !active[t]) continue;   // the same for the whole block
        const double* c = cache + (item0 + item) * kCacheItem64;
        double num[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) num[k] = c[k * 256 + tid];
        const double Ee = E[t], es = tm.eps_s[s];
        double sv = 0.0, dv = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = A * kTB64 + tr * 2 + k / 2, y = B * kTB64 + tc * 2 + k % 2;
            if (x >= tm.nx || y >= tm.nx) continue;
            const double base = es - tm.eps_x[x] - tm.eps_x[y];
            const double rcp = 1.0 / (Ee + base);
            const double nr = num[k] * rcp;
            sv += nr;
            dv -= nr * rcp;
        }
        for (int o = 16; o; o >>= 1) {
            sv += __shfl_xor_sync(0xffffffffu, sv, o);
            dv += __shfl_xor_sync(0xffffffffu, dv, o);
        }
        if (lane == 0) { sred[w][0] = sv; sred[w][1] = dv; }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int ww = 0; ww < 8; ++ww) { a += sred[ww][0]; b += sred[ww][1]; }
            part[(item0 + item) * 2] = a;
            part[(item0 + item) * 2 + 1] = b;
        }
        __syncthreads();
    }
}

// The two terms of Eq. SE for the factor layout of cds_cd_to_mo.
void make_terms(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                const double* eps, SigmaTerm& t0, SigmaTerm& t1) {
    const int32_t nv = nmo - nocc;
    // first sum: s = a (virtual), x = i, y = j (occupied); L^J_{a j} = Lov[j][a][J]
    t0.Aq = Lp; t0.sAt = (int64_t)nmo * M; t0.sAx = M;
    t0.Bk = Lov; t0.sBs = M; t0.sBy = (int64_t)nv * M;
    t0.eps_s = eps + nocc; t0.eps_x = eps; t0.nx = nocc; t0.ns = nv;
    // second sum: s = i (occupied), x = a, y = b (virtual); L^J_{i b} = Lov[i][b][J]
    t1.Aq = Lp + (int64_t)nocc * M; t1.sAt = (int64_t)nmo * M; t1.sAx = M;
    t1.Bk = Lov; t1.sBs = (int64_t)nv * M; t1.sBy = M;
    t1.eps_s = eps; t1.eps_x = eps + nocc; t1.nx = nv; t1.ns = nocc;
}

int64_t items_of(const SigmaTerm& tm, int32_t np, int32_t tb) {
    if (tm.nx <= 0 || tm.ns <= 0) return 0;
    return (int64_t)np * tm.ns * npairs_of(nblocks_of(tm.nx, tb));
}

size_t fp64_part_bytes(int32_t nmo, int32_t nocc, int32_t np, int32_t nE) {
    SigmaTerm t0{}, t1{};
    make_terms(nmo, nocc, 1, nullptr, nullptr, nullptr, t0, t1);
    int64_t items = items_of(t0, np, kTB64) + items_of(t1, np, kTB64);
    return align_up((size_t)items * nE * 2 * sizeof(double));
}

size_t fp64_cache_bytes(int32_t nmo, int32_t nocc, int32_t np) {
    SigmaTerm t0{}, t1{};
    make_terms(nmo, nocc, 1, nullptr, nullptr, nullptr, t0, t1);
    const int64_t items = items_of(t0, np, kTB64) + items_of(t1, np, kTB64);
    return (size_t)items * kCacheItem64 * sizeof(double);
}

int sigma2_fp64(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                int32_t np, const double* eps, const double* E, int32_t nE,
                const int32_t* active, double* sigma, double* dsigma, double* part,
                cudaStream_t stream, double* cache) {
    SigmaTerm t0, t1;
    make_terms(nmo, nocc, M, Lov, Lp, eps, t0, t1);
    int64_t n0 = items_of(t0, np, kTB64), n1 = items_of(t1, np, kTB64);
    if (n0 > 0) {
        k_sigma_fp64<<<(unsigned)n0, 256, 0, stream>>>(t0, M, nE, E, active, 0, part, cache);
        CDS_LAUNCH_CHECK();
    }
    if (n1 > 0) {
        k_sigma_fp64<<<(unsigned)n1, 256, 0, stream>>>(t1, M, nE, E, active, n0, part, cache);
        CDS_LAUNCH_CHECK();
    }
    if (n0 + n1 == 0) {
        CDS_CUDA_TRY(cudaMemsetAsync(sigma, 0, sizeof(double) * np * nE, stream));
        if (dsigma) CDS_CUDA_TRY(cudaMemsetAsync(dsigma, 0, sizeof(double) * np * nE, stream));
        return CDS_OK;
    }
    dim3 grid(nE, np);
    k_sigma_reduce<<<grid, 256, 0, stream>>>(part, np ? n0 / np : 0, n0, np ? n1 / np : 0, nE,
                                            active, sigma, dsigma);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

size_t fp64_cached_workspace_bytes(int32_t nmo, int32_t nocc, int32_t np) {
    return fp64_part_bytes(nmo, nocc, np, 1);
}

int sigma2_cached_fp64(int32_t nmo, int32_t nocc, int32_t np, const double* eps, const double* E,
                       const int32_t* active, const double* cache, double* sigma, double* dsigma,
                       double* part, cudaStream_t stream) {
    SigmaTerm t0, t1;
    make_terms(nmo, nocc, 1, nullptr, nullptr, eps, t0, t1);
    const int64_t n0 = items_of(t0, np, kTB64), n1 = items_of(t1, np, kTB64);
    if (n0 + n1 == 0) {
        CDS_CUDA_TRY(cudaMemsetAsync(sigma, 0, sizeof(double) * np, stream));
        if (dsigma) CDS_CUDA_TRY(cudaMemsetAsync(dsigma, 0, sizeof(double) * np, stream));
        return CDS_OK;
    }
    int sms = 0, dev = 0;
    CDS_CUDA_TRY(cudaGetDevice(&dev));
    CDS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t gmax = (int64_t)std::max(sms, 1) * 8;
    if (n0 > 0) {
        k_sigma_fp64_cached<<<(unsigned)std::min(n0, gmax), 256, 0, stream>>>(t0, E, active, 0,
                                                                              n0, cache, part);
        CDS_LAUNCH_CHECK();
    }
    if (n1 > 0) {
        k_sigma_fp64_cached<<<(unsigned)std::min(n1, gmax), 256, 0, stream>>>(t1, E, active, n0,
                                                                              n1, cache, part);
        CDS_LAUNCH_CHECK();
    }
    k_sigma_reduce<<<dim3(1, np), 256, 0, stream>>>(part, np ? n0 / np : 0, n0, np ? n1 / np : 0, 1,
                                                    active, sigma, dsigma);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

__global__ void k_sum_fixed(const double* __restrict__ x, int32_t n, double* __restrict__ out) {
    __shared__ double sh[256];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += x[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

int sum_fixed(const double* x, int32_t n, double* out, cudaStream_t stream) {
    if (!out) return CDS_OK;
    k_sum_fixed<<<1, 256, 0, stream>>>(x, n, out);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

// Eq. MP2 as the second sum of Eq. SE with q := i, spectator j, E := e_i:
// both operands are rows of Lov, and the energies E of "orbital" i are eps.
static SigmaTerm mp2_term(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                          const double* eps) {
    const int32_t nv = nmo - nocc;
    SigmaTerm t;
    t.Aq = Lov; t.sAt = (int64_t)nv * M; t.sAx = M;
    t.Bk = Lov; t.sBs = (int64_t)nv * M; t.sBy = M;
    t.eps_s = eps; t.eps_x = eps ? eps + nocc : nullptr; t.nx = nv; t.ns = nocc;
    return t;
}

static size_t mp2_fp64_bytes(int32_t nmo, int32_t nocc) {
    const SigmaTerm t = mp2_term(nmo, nocc, 1, nullptr, nullptr);
    return align_up((size_t)std::max<int64_t>(items_of(t, nocc, kTB64), 1) * 2 * sizeof(double)) +
           align_up((size_t)std::max(nocc, 1) * sizeof(double));
}

static int mp2_fp64(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* eps,
                    double* e_pair, double* e_total, void* ws, cudaStream_t stream) {
    const SigmaTerm t = mp2_term(nmo, nocc, M, Lov, eps);
    const int64_t n = items_of(t, nocc, kTB64);
    Carver c(ws);
    double* part = c.take<double>((size_t)std::max<int64_t>(n, 1) * 2);
    double* ep = c.take<double>((size_t)std::max(nocc, 1));
    if (e_pair) ep = e_pair;
    if (n == 0 || M == 0) {
        CDS_CUDA_TRY(cudaMemsetAsync(ep, 0, sizeof(double) * std::max(nocc, 1), stream));
        return sum_fixed(ep, nocc, e_total, stream);
    }
    k_sigma_fp64<<<(unsigned)n, 256, 0, stream>>>(t, M, 1, eps, nullptr, 0, part, nullptr);
    CDS_LAUNCH_CHECK();
    k_sigma_reduce<<<dim3(1, nocc), 256, 0, stream>>>(part, 0, 0, n / nocc, 1, nullptr, ep,
                                                     nullptr);
    CDS_LAUNCH_CHECK();
    return sum_fixed(ep, nocc, e_total, stream);
}

size_t sigma_ws_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE,
                      int32_t precision) {
    if (precision == CDS_PREC_FP64) return fp64_part_bytes(nmo, nocc, np, nE);
    if (is_split_tc(precision))
        return tc_workspace_bytes(nmo, nocc, M, np, nE, precision == CDS_PREC_TF32X3);
    return 0;
}

int sigma2_dispatch(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                    int32_t np, const double* eps, const double* E, int32_t nE,
                    int32_t precision, const int32_t* active, double* sigma, double* dsigma,
                    void* ws, cudaStream_t stream, bool resplit) {
    if (precision == CDS_PREC_FP64)
        return sigma2_fp64(nmo, nocc, M, Lov, Lp, np, eps, E, nE, active, sigma, dsigma,
                           static_cast<double*>(ws), stream, nullptr);
    if (is_split_tc(precision))
        return sigma2_tc(nmo, nocc, M, Lov, Lp, np, eps, E, nE, active, precision, sigma, dsigma,
                         ws, stream, resplit);
    return CDS_ERR_UNSUPPORTED;
}

}  // namespace cds

using namespace cds;

static bool sigma_args_ok(int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE) {
    return nmo > 0 && nocc >= 0 && nocc <= nmo && M >= 0 && np >= 0 && nE >= 1 && nE <= 4096 &&
           np <= 65535;
}

extern "C" size_t cds_sigma2_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np,
                                             int32_t nE, int32_t precision) {
    if (!sigma_args_ok(nmo, nocc, M, np, nE)) return 0;
    return sigma_ws_bytes(nmo, nocc, M, np, nE, precision);
}

extern "C" int cds_sigma2_diag(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                               const double* Lp, int32_t np, const double* eps,
                               const double* E, int32_t nE, int32_t precision, double* sigma,
                               double* dsigma, void* workspace, size_t workspace_bytes,
                               cudaStream_t stream) {
    if (!sigma_args_ok(nmo, nocc, M, np, nE)) return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && !is_split_tc(precision)) return CDS_ERR_UNSUPPORTED;
    if (np == 0) return CDS_OK;
    if (!Lp || !eps || !E || !sigma || (nocc > 0 && nocc < nmo && !Lov)) return CDS_ERR_ARG;
    size_t need = sigma_ws_bytes(nmo, nocc, M, np, nE, precision);
    if (need && (!workspace || workspace_bytes < need)) return CDS_ERR_WORKSPACE;
    return sigma2_dispatch(nmo, nocc, M, Lov, Lp, np, eps, E, nE, precision, nullptr, sigma,
                           dsigma, workspace, stream);
}

extern "C" size_t cds_mp2_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t precision) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || M < 0) return 0;
    if (precision == CDS_PREC_FP64) return mp2_fp64_bytes(nmo, nocc);
    if (is_split16(precision)) return tc_mp2_workspace_bytes(nmo, nocc, M);
    return 0;
}

extern "C" int cds_mp2_energy(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                              const double* eps, int32_t precision, double* e_pair,
                              double* e_total, void* workspace, size_t workspace_bytes,
                              cudaStream_t stream) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || M < 0 || nocc > 65535) return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && !is_split16(precision)) return CDS_ERR_UNSUPPORTED;
    if (!eps || (!e_pair && !e_total) || (nocc > 0 && nocc < nmo && M > 0 && !Lov))
        return CDS_ERR_ARG;
    if (nocc == 0) {
        if (e_total) CDS_CUDA_TRY(cudaMemsetAsync(e_total, 0, sizeof(double), stream));
        return CDS_OK;
    }
    const size_t need = cds_mp2_workspace_bytes(nmo, nocc, M, precision);
    if (!workspace || workspace_bytes < need) return CDS_ERR_WORKSPACE;
    if (precision == CDS_PREC_FP64)
        return mp2_fp64(nmo, nocc, M, Lov, eps, e_pair, e_total, workspace, stream);
    return mp2_tc(nmo, nocc, M, Lov, eps, precision, e_pair, e_total, workspace, stream);
}

extern "C" size_t cds_sigma2_cache_bytes(int32_t nmo, int32_t nocc, int32_t np,
                                         int32_t precision) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || np < 0) return 0;
    if (precision == CDS_PREC_FP64) return fp64_cache_bytes(nmo, nocc, np);
    if (is_split_tc(precision)) return tc_cache_bytes(nmo, nocc, np);
    return 0;
}

extern "C" int cds_sigma2_diag_cache(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                                     const double* Lp, int32_t np, const double* eps,
                                     const double* E, int32_t nE, int32_t precision,
                                     double* sigma, double* dsigma, void* cache,
                                     size_t cache_bytes, void* workspace, size_t workspace_bytes,
                                     cudaStream_t stream) {
    if (!sigma_args_ok(nmo, nocc, M, np, nE)) return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && !is_split_tc(precision)) return CDS_ERR_UNSUPPORTED;
    if (np == 0) return CDS_OK;
    if (!Lp || !eps || !E || !sigma || !cache || (nocc > 0 && nocc < nmo && !Lov))
        return CDS_ERR_ARG;
    if (cache_bytes < cds_sigma2_cache_bytes(nmo, nocc, np, precision)) return CDS_ERR_ARG;
    size_t need = sigma_ws_bytes(nmo, nocc, M, np, nE, precision);
    if (need && (!workspace || workspace_bytes < need)) return CDS_ERR_WORKSPACE;
    if (precision == CDS_PREC_FP64)
        return sigma2_fp64(nmo, nocc, M, Lov, Lp, np, eps, E, nE, nullptr, sigma, dsigma,
                           static_cast<double*>(workspace), stream, static_cast<double*>(cache));
    return sigma2_tc(nmo, nocc, M, Lov, Lp, np, eps, E, nE, nullptr, precision, sigma, dsigma,
                     workspace, stream, true, static_cast<float*>(cache));
}
