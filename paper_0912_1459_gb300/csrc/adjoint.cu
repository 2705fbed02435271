// Hand-written adjoint of the quasiparticle energies (the paper does not
// differentiate; this is the derivative of Eq. SE and Eq. iter).
//
// For a loss l(w_1..w_np) with upstream gradients g_t = dl/dw_t at converged
// roots w_t = e_q + Sigma_qq(w_t):
//   dl/dtheta = sum_t W_t (de_qt/dtheta + dSigma_t/dtheta),
//   W_t = g_t P_t,  P_t = 1 / (1 - dSigma_t/dw)|w_t       (Eq. ps at the root).
// FP64 path, one orbital t at a time: per work item (spectator s, block pair
// A <= B) the kernel recomputes the two exchange-paired tiles X_xy, X_yx in
// FP64 (the MO integrals are recomputed, never stored across orbitals) and
// forms
//   G_xy = dSigma/dX_xy = (4 X_xy - 2 X_yx) / D_xy,
// writing the orbital's G (nx * ns * nx values per sum of Eq. SE) and the
// energy partials n / D^2.  Once the orbital's dSigma/dw is complete, G is
// scaled by W_t and the factor gradients are FP64 GEMMs:
//   dLq[t][x] = sum_(s,y) G[x][s][y] B[s][y],   dB[s][y] += sum_x G[x][s][y] Lq[t][x],
// so the workspace holds one orbital's G (o*v*o + v*o*v doubles), not all.
// The tensor-core form (adjoint_tc.cu) serves the split precisions.
#include "sigma.cuh"

namespace cds {

int launch_dgemm_strided(int m, int n, int k, int batch, const double* A, int64_t ars, int64_t acs,
                         int64_t abs_, const double* B, int64_t brs, int64_t bcs, int64_t bbs,
                         double* C, int64_t crs, int64_t ccs, int64_t cbs, cudaStream_t s,
                         bool accumulate = false);
void make_terms(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                const double* eps, SigmaTerm& t0, SigmaTerm& t1);

namespace {

constexpr int TB = 32, JK = 16;

struct AdjTerm {
    SigmaTerm tm;
    double* G;          // [nx][ns][nx] of the orbital in work
    int32_t s_eps_off;  // offsets of the spectator / pair orbitals in eps
    int32_t x_eps_off;
};

// One work item per block: FP64 tiles, then G and the energy partials.
__global__ void __launch_bounds__(256)
k_adj_g(AdjTerm at, int32_t t, int32_t M, int32_t nmo, const double* __restrict__ omega,
        double* __restrict__ deps_t /* [np][nmo] */, double* __restrict__ dsig_t /* [np] */) {
    __shared__ double sA1[TB][JK + 1], sB1[TB][JK + 1], sA2[TB][JK + 1], sB2[TB][JK + 1];
    __shared__ double srow[TB], scol[TB], sspec;
    const SigmaTerm& tm = at.tm;
    const int32_t nb = nblocks_of(tm.nx, TB);
    const int64_t npb = npairs_of(nb);
    const int64_t r = blockIdx.x;   // item of orbital t: (spectator, block pair)
    const int32_t s = (int32_t)(r / npb);
    int32_t A, B;
    block_pair(r - (int64_t)s * npb, nb, A, B);
    const double* aq = tm.Aq + t * tm.sAt;
    const double* bk = tm.Bk + s * tm.sBs;
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    if (tid < TB) { srow[tid] = 0.0; scol[tid] = 0.0; }
    if (tid == 0) sspec = 0.0;
    double acc1[2][2] = {}, acc2[2][2] = {};
    for (int J0 = 0; J0 < M; J0 += JK) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            int idx = tid + 256 * rr;
            int row = idx / JK, c = idx % JK;
            int J = J0 + c;
            int xa = A * TB + row, xb = B * TB + row;
            bool okJ = J < M;
            bool oka = okJ && xa < tm.nx, okb = okJ && xb < tm.nx;
            sA1[row][c] = oka ? aq[xa * tm.sAx + J] : 0.0;
            sA2[row][c] = oka ? bk[xa * tm.sBy + J] : 0.0;
            sB1[row][c] = okb ? bk[xb * tm.sBy + J] : 0.0;
            sB2[row][c] = okb ? aq[xb * tm.sAx + J] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < JK; ++c) {
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
    const double w = omega[t];
    const double es = tm.eps_s[s];
    double spec = 0.0;
    const int64_t gt = 0;   // G holds orbital t only
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int lx = tr * 2 + i, ly = tc * 2 + j;
            const int x = A * TB + lx, y = B * TB + ly;
            if (x >= tm.nx || y >= tm.nx) continue;
            const double x1 = acc1[i][j], x2 = acc2[i][j];
            const double D = w + es - tm.eps_x[x] - tm.eps_x[y];
            const double n = (A == B) ? (2.0 * x1 - x2) * x1 : 2.0 * (x1 * x1 + x2 * x2 - x1 * x2);
            const double rD = n / (D * D);
            at.G[gt + ((int64_t)x * tm.ns + s) * tm.nx + y] = (4.0 * x1 - 2.0 * x2) / D;
            if (A != B) at.G[gt + ((int64_t)y * tm.ns + s) * tm.nx + x] = (4.0 * x2 - 2.0 * x1) / D;
            spec += rD;
            atomicAdd(&srow[lx], rD);
            atomicAdd(&scol[ly], rD);
        }
    for (int o = 16; o; o >>= 1) spec += __shfl_xor_sync(0xffffffffu, spec, o);
    if ((tid & 31) == 0) atomicAdd(&sspec, spec);
    __syncthreads();
    double* de = deps_t + (int64_t)t * nmo;
    if (tid < TB) {
        const int x = A * TB + tid, y = B * TB + tid;
        if (x < tm.nx) atomicAdd(de + at.x_eps_off + x, srow[tid]);
        if (y < tm.nx) atomicAdd(de + at.x_eps_off + y, scol[tid]);
    }
    if (tid == 0) {
        atomicAdd(de + at.s_eps_off + s, -sspec);
        atomicAdd(dsig_t + t, -sspec);
    }
}

// W_t = g_t / (1 - dSigma_t/dw); d_eps = sum_t W_t (dSigma_t/de + e_qt).
__global__ void k_adj_weights(int32_t np, int32_t nmo, const int32_t* __restrict__ orb,
                              const double* __restrict__ g, const double* __restrict__ dsig_t,
                              const double* __restrict__ deps_t, double* __restrict__ W,
                              double* __restrict__ d_eps) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nmo; p += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < np; ++t) {
            const double wt = g[t] / (1.0 - dsig_t[t]);
            acc += wt * (deps_t[(int64_t)t * nmo + p] + (orb[t] == p ? 1.0 : 0.0));
            if (p == 0) W[t] = wt;
        }
        d_eps[p] = acc;
    }
}

// G *= g_t / (1 - dSigma_t/dw) for one orbital t
__global__ void k_scale_orbital(double* __restrict__ G, int64_t n, int32_t t,
                                const double* __restrict__ g, const double* __restrict__ dsig_t) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    G[i] *= g[t] / (1.0 - dsig_t[t]);
}

// dst[a][j][J] = src[j][a][J]  (or dst += ... with add)
__global__ void k_swap01(const double* __restrict__ src, int32_t d0, int32_t d1, int32_t M,
                         double* __restrict__ dst, int add) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)d0 * d1 * M;
    if (e >= tot) return;
    const int J = (int)(e % M);
    const int64_t r = e / M;
    const int i1 = (int)(r % d1), i0 = (int)(r / d1);   // e indexes src[i0][i1][J]
    const int64_t o = ((int64_t)i1 * d0 + i0) * M + J;
    dst[o] = add ? dst[o] + src[e] : src[e];
}

// dst[t][x][J] = Lp[t][off + x][J]
__global__ void k_gather_rows(const double* __restrict__ Lp, int32_t np, int32_t nmo, int32_t off,
                              int32_t nx, int32_t M, double* __restrict__ dst) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)np * nx * M) return;
    const int J = (int)(e % M);
    const int64_t r = e / M;
    const int x = (int)(r % nx), t = (int)(r / nx);
    dst[e] = Lp[((int64_t)t * nmo + off + x) * M + J];
}

struct AdjLayout {
    double* G0;        // first sum of orbital t   [o][v][o]
    double* G1;        // second sum of orbital t  [v][o][v]
    double* Lvo;       // [v][o][M]
    double* Aq;        // [max(o, v)][M] gathered rows of orbital t
    double* dB;        // [v][o][M] first-sum factor gradient, summed over orbitals
    double* deps_t;    // [np][nmo]
    double* dsig_t;    // [np]
    double* W;         // [np]
    size_t bytes;
};

AdjLayout adj_layout(void* ws, int32_t nmo, int32_t nocc, int32_t M, int32_t np) {
    const int64_t o = nocc, v = nmo - nocc;
    Carver c(ws);
    AdjLayout l;
    l.G0 = c.take<double>((size_t)std::max<int64_t>(o * v * o, 1));
    l.G1 = c.take<double>((size_t)std::max<int64_t>(v * o * v, 1));
    l.Lvo = c.take<double>((size_t)std::max<int64_t>(v * o * M, 1));
    l.Aq = c.take<double>((size_t)std::max<int64_t>(std::max(o, v) * M, 1));
    l.dB = c.take<double>((size_t)std::max<int64_t>(o * v * M, 1));
    l.deps_t = c.take<double>((size_t)std::max<int64_t>((int64_t)np * nmo, 1));
    l.dsig_t = c.take<double>((size_t)std::max(np, 1));
    l.W = c.take<double>((size_t)std::max(np, 1));
    l.bytes = c.off;
    return l;
}

}  // namespace

// d_eps = sum_t W_t (dSigma_t/de + e_qt) from the per-orbital energy partials
// and dSigma_t/dw (shared with the tensor-core form).
int adj_finish(int32_t np, int32_t nmo, const int32_t* orb, const double* g, const double* dsig_t,
               const double* deps_t, double* W, double* d_eps, cudaStream_t stream) {
    k_adj_weights<<<(nmo + 127) / 128, 128, 0, stream>>>(np, nmo, orb, g, dsig_t, deps_t, W, d_eps);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

}  // namespace cds

using namespace cds;

namespace cds {
size_t adj_tc_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np,
                              int32_t precision);
int adj_tc_gradient(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                    const int32_t* orb, int32_t np, const double* eps, const double* omega,
                    const double* g, int32_t precision, double* d_eps, double* d_Lov,
                    double* d_Lp, void* workspace, size_t workspace_bytes, cudaStream_t stream);
}  // namespace cds

extern "C" size_t cds_qp_gradient_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M,
                                                  int32_t np, int32_t precision) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || M < 0 || np < 0) return 0;
    if (precision == CDS_PREC_FP64) return adj_layout(nullptr, nmo, nocc, M, np).bytes;
    if (precision == CDS_PREC_BF16X3 || precision == CDS_PREC_TF32X3)
        return adj_tc_workspace_bytes(nmo, nocc, M, np, precision);
    return 0;
}

extern "C" int cds_qp_gradient(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                               const double* Lp, const int32_t* orb, int32_t np,
                               const double* eps, const double* omega, const double* g,
                               int32_t precision, double* d_eps, double* d_Lov, double* d_Lp,
                               void* workspace, size_t workspace_bytes, cudaStream_t stream) {
    if (nmo <= 0 || nocc <= 0 || nocc >= nmo || M <= 0 || np <= 0 || np > 65535) return CDS_ERR_ARG;
    if (!Lov || !Lp || !orb || !eps || !omega || !g || !d_eps || !d_Lov || !d_Lp) return CDS_ERR_ARG;
    if (precision == CDS_PREC_BF16X3 || precision == CDS_PREC_TF32X3)
        return adj_tc_gradient(nmo, nocc, M, Lov, Lp, orb, np, eps, omega, g, precision, d_eps,
                               d_Lov, d_Lp, workspace, workspace_bytes, stream);
    if (precision != CDS_PREC_FP64) return CDS_ERR_UNSUPPORTED;
    AdjLayout lay = adj_layout(workspace, nmo, nocc, M, np);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    const int32_t o = nocc, v = nmo - nocc;
    SigmaTerm t0, t1;
    make_terms(nmo, nocc, M, Lov, Lp, eps, t0, t1);
    CDS_CUDA_TRY(cudaMemsetAsync(lay.deps_t, 0, sizeof(double) * np * nmo, stream));
    CDS_CUDA_TRY(cudaMemsetAsync(lay.dsig_t, 0, sizeof(double) * np, stream));
    CDS_CUDA_TRY(cudaMemsetAsync(d_Lov, 0, sizeof(double) * (size_t)o * v * M, stream));
    AdjTerm a0{t0, lay.G0, nocc, 0}, a1{t1, lay.G1, 0, nocc};
    const int64_t n0 = (int64_t)t0.ns * npairs_of(nblocks_of(t0.nx, TB));
    const int64_t n1 = (int64_t)t1.ns * npairs_of(nblocks_of(t1.nx, TB));
    const int64_t per0 = (int64_t)o * v * o, per1 = (int64_t)v * o * v;
    // first sum: x = i (occupied rows of Lp), B[s=a][y=j] = Lov[j][a] -> Lvo[a][j]
    k_swap01<<<(unsigned)(((int64_t)o * v * M + 255) / 256), 256, 0, stream>>>(Lov, o, v, M, lay.Lvo, 0);
    CDS_LAUNCH_CHECK();
    for (int32_t t = 0; t < np; ++t) {
        // the orbital's G (every (x, s, y) written by exactly one item) and
        // energy partials
        k_adj_g<<<(unsigned)n0, 256, 0, stream>>>(a0, t, M, nmo, omega, lay.deps_t, lay.dsig_t);
        CDS_LAUNCH_CHECK();
        k_adj_g<<<(unsigned)n1, 256, 0, stream>>>(a1, t, M, nmo, omega, lay.deps_t, lay.dsig_t);
        CDS_LAUNCH_CHECK();
        k_scale_orbital<<<(unsigned)((per0 + 255) / 256), 256, 0, stream>>>(lay.G0, per0, t, g,
                                                                            lay.dsig_t);
        CDS_LAUNCH_CHECK();
        k_scale_orbital<<<(unsigned)((per1 + 255) / 256), 256, 0, stream>>>(lay.G1, per1, t, g,
                                                                            lay.dsig_t);
        CDS_LAUNCH_CHECK();
        double* dLq = d_Lp + (int64_t)t * nmo * M;
        // first sum: dLq[i] = sum_(a,j) G0[i][a][j] Lvo[a][j];  dB[a][j] += sum_i G0[i][a][j] Lq[i]
        int st = launch_dgemm_strided(o, M, v * o, 1, lay.G0, (int64_t)v * o, 1, 0, lay.Lvo, M, 1,
                                      0, dLq, M, 1, 0, stream);
        if (st) return st;
        k_gather_rows<<<(unsigned)(((int64_t)o * M + 255) / 256), 256, 0, stream>>>(
            Lp + (int64_t)t * nmo * M, 1, nmo, 0, o, M, lay.Aq);
        CDS_LAUNCH_CHECK();
        st = launch_dgemm_strided(v * o, M, o, 1, lay.G0, 1, (int64_t)v * o, 0, lay.Aq, M, 1, 0,
                                  lay.dB, M, 1, 0, stream, t > 0);
        if (st) return st;
        // second sum: x = a (virtual rows of Lp), B[s=i][y=b] = Lov[i][b]
        st = launch_dgemm_strided(v, M, o * v, 1, lay.G1, (int64_t)o * v, 1, 0, Lov, M, 1, 0,
                                  dLq + (int64_t)nocc * M, M, 1, 0, stream);
        if (st) return st;
        k_gather_rows<<<(unsigned)(((int64_t)v * M + 255) / 256), 256, 0, stream>>>(
            Lp + (int64_t)t * nmo * M, 1, nmo, nocc, v, M, lay.Aq);
        CDS_LAUNCH_CHECK();
        st = launch_dgemm_strided(o * v, M, v, 1, lay.G1, 1, (int64_t)o * v, 0, lay.Aq, M, 1, 0,
                                  d_Lov, M, 1, 0, stream, true);
        if (st) return st;
    }
    // d_Lov += dB  ([a][j] -> [j][a])
    k_swap01<<<(unsigned)(((int64_t)o * v * M + 255) / 256), 256, 0, stream>>>(lay.dB, v, o, M, d_Lov, 1);
    CDS_LAUNCH_CHECK();
    return adj_finish(np, nmo, orb, g, lay.dsig_t, lay.deps_t, lay.W, d_eps, stream);
}
