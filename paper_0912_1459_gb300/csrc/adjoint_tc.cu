// Adjoint of the quasiparticle energies on the tensor cores (split precisions
// BF16X3 / TF32X3; the paper does not differentiate -- this is the derivative
// of Eq. SE and Eq. iter, as in adjoint.cu).
//
// Per orbital t (row q of the factors, Lq = Lp[t]) and per sum of Eq. SE the
// MO integrals are recomputed as one tcgen05 GEMM over the Cholesky index,
//   first sum   X[i][(j, a)] = sum_J Lq[i][J] Lov[j][a][J]       = (qi|aj),
//   second sum  X[a][(i, b)] = sum_J Lq[o + a][J] Lov[i][b][J]   = (qa|ib),
// i.e. X[x][(c1, c2)] with c1 occupied, c2 virtual, in Lov's row order.  Its
// exchange partner swaps x with c1 (first sum) or with c2 (second sum).  With
// D = w + e_spec - e_x - e_other (first sum: spec = c2, other = c1; second:
// spec = c1, other = c2), n = (2 X - X_partner) X and r = n / D^2:
//   G = dSigma/dX = (4 X - 2 X_partner) / D,   dSigma/dw = -sum r,
//   dSigma/de_x = dSigma/de_other = +r,  dSigma/de_spec = -r  (summed).
// k_adj_gx forms G in one pass over X and writes it split (hi + lo) in the
// two layouts the factor-gradient GEMMs read as K-major operands:
//   GA[(t, x)][(c1, c2)]   ->  dLq[t][x][J]  = W_t sum_c GA[(t,x)][c] Lov[c][J]
//   GB[(c1, c2)][(t, x)]   ->  dLov[c][J]   += sum_(t,x) GB[c][(t,x)] W_t Lq[t][x][J]
// with W_t = g_t / (1 - dSigma_t/dw) (the pole strength at the root times the
// upstream gradient), folded into the Lq operand and into the dLq rows once
// both sums of the orbital are complete.  Orbitals go in chunks of kChunk so
// the workspace holds one chunk's G, not all orbitals'.  X itself is FP64 for
// one orbital and one sum at a time.  Every GEMM accumulates in FP32.
#include <algorithm>

#include "ao2mo_tc.cuh"
#include "split.cuh"

namespace cds {

int adj_finish(int32_t np, int32_t nmo, const int32_t* orb, const double* g, const double* dsig_t,
               const double* deps_t, double* W, double* d_eps, cudaStream_t stream);

namespace {

constexpr int32_t kChunk = 8;   // orbitals whose G is held at once
constexpr int kT = 32;          // tile edge of the G pass

inline int32_t ld8(int64_t n) { return (int32_t)((n + 7) / 8 * 8); }   // 16-byte operand rows

template <bool TF32>
using E = trc::SplitE<TF32>;

template <bool TF32>
__device__ __forceinline__ void split_d(double x, E<TF32>* hi, E<TF32>* lo, int64_t e) {
    float f, r;
    trc::pair_of_double(x, f, r);
    trc::split_store<TF32>(f, r, hi, lo, e);
}

// dst[r][k] = src[r][k] for k < K (rows of ld elements), split.
template <bool TF32>
__global__ void k_split_rows(const double* __restrict__ src, int64_t rows, int32_t K, int32_t ld,
                             E<TF32>* __restrict__ hi, E<TF32>* __restrict__ lo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * K) return;
    const int64_t r = e / K;
    const int32_t k = (int32_t)(e % K);
    split_d<TF32>(src[e], hi, lo, r * ld + k);
}

// dst[k][r] = scale[r / per] * src[r][k] (src rows of K elements, src row r at
// src + (r / per) * grp + (r % per) * K), split, dst rows of ld elements.
template <bool TF32>
__global__ void k_split_transpose(const double* __restrict__ src, int64_t nrows, int32_t K,
                                  int64_t per, int64_t grp, const double* __restrict__ scale,
                                  int32_t ld, E<TF32>* __restrict__ hi, E<TF32>* __restrict__ lo) {
    __shared__ double tile[kT][kT + 1];
    const int64_t r0 = (int64_t)blockIdx.y * kT;
    const int32_t k0 = blockIdx.x * kT;
    for (int i = threadIdx.y; i < kT; i += blockDim.y) {
        const int64_t r = r0 + i;
        const int32_t k = k0 + threadIdx.x;
        double v = 0.0;
        if (r < nrows && k < K) {
            v = src[(r / per) * grp + (r % per) * K + k];
            if (scale) v *= scale[r / per];
        }
        tile[i][threadIdx.x] = v;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < kT; i += blockDim.y) {
        const int32_t k = k0 + i;
        const int64_t r = r0 + threadIdx.x;
        if (k < K && r < nrows) split_d<TF32>(tile[threadIdx.x][i], hi, lo, (int64_t)k * ld + r);
    }
}

struct GxArgs {
    const double* X;    // [nx][ldc], column c = c1 * n2 + c2
    int32_t nx, n1, n2, ldc;
    int32_t swap_c1;    // 1: partner X[c1][(x, c2)] (first sum), 0: X[c2][(c1, x)] (second)
    int32_t xoff;       // eps offset of x (0 occupied, nocc virtual)
    int32_t nocc;
    int32_t tl;         // orbital's position in the chunk
    int32_t ldk;        // row stride of GB
    void *ga_hi, *ga_lo, *gb_hi, *gb_lo;
};

// One 32 x 32 tile (x, c2) at fixed c1 per block: G in both layouts, the
// energy partials and dSigma/dw of orbital t.
template <bool TF32>
__global__ void __launch_bounds__(256)
k_adj_gx(GxArgs a, int32_t t, int32_t nmo, const double* __restrict__ eps,
         const double* __restrict__ omega, double* __restrict__ deps_t,
         double* __restrict__ dsig_t) {
    __shared__ double sY[kT][kT + 1], sP[kT][kT + 1], sG[kT][kT + 1];
    __shared__ double rx[kT], rc2[kT], rc1;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int32_t c2_0 = blockIdx.x * kT, x0 = blockIdx.y * kT, c1 = blockIdx.z;
    const int64_t col0 = (int64_t)c1 * a.n2;
    if (ty == 0) { rx[tx] = 0.0; rc2[tx] = 0.0; }
    if (tx == 0 && ty == 0) rc1 = 0.0;
    for (int i = ty; i < kT; i += 8) {
        const int32_t x = x0 + i, c2 = c2_0 + tx;
        const bool ok = x < a.nx && c2 < a.n2;
        sY[i][tx] = ok ? a.X[(int64_t)x * a.ldc + col0 + c2] : 0.0;
        if (a.swap_c1) {
            sP[i][tx] = ok ? a.X[(int64_t)c1 * a.ldc + (int64_t)x * a.n2 + c2] : 0.0;
        } else {   // partner X[c2][c1 n2 + x]: rows c2, read along x, stored transposed
            const int32_t cr = c2_0 + i, xr = x0 + tx;
            sP[tx][i] = (cr < a.n2 && xr < a.nx) ? a.X[(int64_t)cr * a.ldc + col0 + xr] : 0.0;
        }
    }
    __syncthreads();
    const double w = omega[t];
    const double sgn = a.swap_c1 ? 1.0 : -1.0;   // D = w - e_x + sgn (e_c2 - e_c1)
    const double ec1 = eps[c1];
    E<TF32>* gah = (E<TF32>*)a.ga_hi;
    E<TF32>* gal = (E<TF32>*)a.ga_lo;
    double rsum = 0.0, rcol = 0.0;
    for (int i = ty; i < kT; i += 8) {   // one warp per row x of the tile
        const int32_t x = x0 + i, c2 = c2_0 + tx;
        double G = 0.0, r = 0.0;
        if (x < a.nx && c2 < a.n2) {
            const double y = sY[i][tx], yx = sP[i][tx];
            const double D = w - eps[a.xoff + x] + sgn * (eps[a.nocc + c2] - ec1);
            G = (4.0 * y - 2.0 * yx) / D;
            r = (2.0 * y - yx) * y / (D * D);
            split_d<TF32>(G, gah, gal, ((int64_t)a.tl * a.nx + x) * a.ldc + col0 + c2);
        }
        sG[i][tx] = G;
        rcol += r;
        double rrow = r;
        for (int o = 16; o; o >>= 1) rrow += __shfl_xor_sync(0xffffffffu, rrow, o);
        if (tx == 0) rx[i] = rrow;
        rsum += rrow;
    }
    atomicAdd(&rc2[tx], rcol);
    if (tx == 0) atomicAdd(&rc1, rsum);
    __syncthreads();
    // GB[(c1, c2)][(tl, x)]: 32 consecutive x per warp store
    E<TF32>* gbh = (E<TF32>*)a.gb_hi;
    E<TF32>* gbl = (E<TF32>*)a.gb_lo;
    for (int i = ty; i < kT; i += 8) {
        const int32_t c2 = c2_0 + i, x = x0 + tx;
        if (c2 < a.n2 && x < a.nx)
            split_d<TF32>(sG[tx][i], gbh, gbl,
                          (col0 + c2) * a.ldk + (int64_t)a.tl * a.nx + x);
    }
    double* de = deps_t + (int64_t)t * nmo;
    if (ty == 0) {
        if (x0 + tx < a.nx) atomicAdd(de + a.xoff + x0 + tx, rx[tx]);
        if (c2_0 + tx < a.n2) atomicAdd(de + a.nocc + c2_0 + tx, -sgn * rc2[tx]);
    }
    if (tx == 0 && ty == 1) {
        atomicAdd(de + c1, sgn * rc1);
        atomicAdd(dsig_t + t, -rc1);
    }
}

// W[t] = g[t] / (1 - dSigma_t/dw) for the orbitals of a chunk
__global__ void k_chunk_weights(int32_t t0, int32_t nc, const double* __restrict__ g,
                                const double* __restrict__ dsig_t, double* __restrict__ W) {
    const int t = t0 + threadIdx.x;
    if (threadIdx.x < nc) W[t] = g[t] / (1.0 - dsig_t[t]);
}

// rows of dLq of a chunk *= W[t]
__global__ void k_scale_chunk(double* __restrict__ dLp, int64_t per, int32_t nc, int32_t t0,
                              const double* __restrict__ W) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= per * nc) return;
    dLp[e] *= W[t0 + e / per];
}

struct TcLayout {
    int32_t* err;
    double *deps_t, *dsig_t, *W, *X;
    void *lov_hi, *lov_lo;     // [o v][ldM]       Lov rows, K = J
    void *lovt_hi, *lovt_lo;   // [M][ldc]         Lov^T, K = (c1, c2)
    void *lq_hi, *lq_lo;       // [kChunk nmo][ldM] rows of the chunk's Lp
    void *lqt_hi, *lqt_lo;     // [M][ldk_max]     W-scaled Lq^T of one sum, K = (t, x)
    void *ga1_hi, *ga1_lo, *gb1_hi, *gb1_lo;   // first sum
    void *ga2_hi, *ga2_lo, *gb2_hi, *gb2_lo;   // second sum
    int32_t ldM, ldc, ldk1, ldk2;
    size_t bytes;
};

TcLayout tc_layout(void* ws, int32_t nmo, int32_t nocc, int32_t M, int32_t np, bool tf32) {
    const int64_t o = nocc, v = nmo - nocc, ov = o * v;
    const int64_t ch = std::max(1, std::min(np, kChunk));
    const size_t es = tf32 ? 4 : 2;
    TcLayout l;
    l.ldM = ld8(M);
    l.ldc = ld8(ov);
    l.ldk1 = ld8(ch * o);
    l.ldk2 = ld8(ch * v);
    Carver c(ws);
    auto take = [&](int64_t elems) { return (void*)c.take<char>((size_t)std::max<int64_t>(elems, 1) * es); };
    l.err = c.take<int32_t>(4);
    l.deps_t = c.take<double>((size_t)std::max<int64_t>((int64_t)np * nmo, 1));
    l.dsig_t = c.take<double>((size_t)std::max(np, 1));
    l.W = c.take<double>((size_t)std::max(np, 1));
    l.X = c.take<double>((size_t)std::max<int64_t>(std::max(o, v) * l.ldc, 1));
    l.lov_hi = take(ov * l.ldM);
    l.lov_lo = take(ov * l.ldM);
    l.lovt_hi = take((int64_t)M * l.ldc);
    l.lovt_lo = take((int64_t)M * l.ldc);
    l.lq_hi = take(ch * nmo * l.ldM);
    l.lq_lo = take(ch * nmo * l.ldM);
    l.lqt_hi = take((int64_t)M * std::max(l.ldk1, l.ldk2));
    l.lqt_lo = take((int64_t)M * std::max(l.ldk1, l.ldk2));
    l.ga1_hi = take(ch * o * l.ldc);
    l.ga1_lo = take(ch * o * l.ldc);
    l.gb1_hi = take(ov * l.ldk1);
    l.gb1_lo = take(ov * l.ldk1);
    l.ga2_hi = take(ch * v * l.ldc);
    l.ga2_lo = take(ch * v * l.ldc);
    l.gb2_hi = take(ov * l.ldk2);
    l.gb2_lo = take(ov * l.ldk2);
    l.bytes = c.off;
    return l;
}

inline unsigned blocks(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

template <bool TF32>
int gradient(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
             const int32_t* orb, int32_t np, const double* eps, const double* omega,
             const double* g, int32_t precision, double* d_eps, double* d_Lov, double* d_Lp,
             const TcLayout& l, cudaStream_t stream) {
    const int32_t o = nocc, v = nmo - nocc;
    const int64_t ov = (int64_t)o * v;
    using T = E<TF32>;
    CDS_CUDA_TRY(cudaMemsetAsync(l.err, 0, sizeof(int32_t), stream));
    CDS_CUDA_TRY(cudaMemsetAsync(l.deps_t, 0, sizeof(double) * np * nmo, stream));
    CDS_CUDA_TRY(cudaMemsetAsync(l.dsig_t, 0, sizeof(double) * np, stream));
    CDS_CUDA_TRY(cudaMemsetAsync(d_Lov, 0, sizeof(double) * ov * M, stream));
    // the factors, split once: Lov rows (K = J) and Lov^T (K = (c1, c2))
    k_split_rows<TF32><<<blocks(ov * M), 256, 0, stream>>>(Lov, ov, M, l.ldM, (T*)l.lov_hi,
                                                            (T*)l.lov_lo);
    CDS_LAUNCH_CHECK();
    {
        dim3 grid((unsigned)((M + kT - 1) / kT), (unsigned)((ov + kT - 1) / kT));
        k_split_transpose<TF32><<<grid, dim3(kT, 8), 0, stream>>>(
            Lov, ov, M, ov, 0, nullptr, l.ldc, (T*)l.lovt_hi, (T*)l.lovt_lo);
        CDS_LAUNCH_CHECK();
    }
    for (int32_t t0 = 0; t0 < np; t0 += kChunk) {
        const int32_t nc = std::min(kChunk, np - t0);
        const double* lp0 = Lp + (int64_t)t0 * nmo * M;
        k_split_rows<TF32><<<blocks((int64_t)nc * nmo * M), 256, 0, stream>>>(
            lp0, (int64_t)nc * nmo, M, l.ldM, (T*)l.lq_hi, (T*)l.lq_lo);
        CDS_LAUNCH_CHECK();
        for (int32_t tl = 0; tl < nc; ++tl) {
            const int32_t t = t0 + tl;
            for (int sum = 0; sum < 2; ++sum) {
                const int32_t nx = sum == 0 ? o : v, xoff = sum == 0 ? 0 : o;
                const size_t arow = ((size_t)tl * nmo + xoff) * l.ldM * sizeof(T);
                // X[x][c] = sum_J Lq[x][J] Lov[c][J]
                int st = tr_split_gemm(precision, (char*)l.lq_hi + arow, (char*)l.lq_lo + arow, nx,
                                       l.lov_hi, l.lov_lo, ov, M, l.ldM, nx, 0, l.ldc, 1, l.X,
                                       false, l.err, stream);
                if (st) return st;
                GxArgs a;
                a.X = l.X;
                a.nx = nx;
                a.n1 = o;
                a.n2 = v;
                a.ldc = l.ldc;
                a.swap_c1 = sum == 0;
                a.xoff = xoff;
                a.nocc = o;
                a.tl = tl;
                a.ldk = sum == 0 ? l.ldk1 : l.ldk2;
                a.ga_hi = sum == 0 ? l.ga1_hi : l.ga2_hi;
                a.ga_lo = sum == 0 ? l.ga1_lo : l.ga2_lo;
                a.gb_hi = sum == 0 ? l.gb1_hi : l.gb2_hi;
                a.gb_lo = sum == 0 ? l.gb1_lo : l.gb2_lo;
                dim3 grid((unsigned)((v + kT - 1) / kT), (unsigned)((nx + kT - 1) / kT), (unsigned)o);
                k_adj_gx<TF32><<<grid, dim3(kT, 8), 0, stream>>>(a, t, nmo, eps, omega, l.deps_t,
                                                                  l.dsig_t);
                CDS_LAUNCH_CHECK();
            }
        }
        k_chunk_weights<<<1, kChunk, 0, stream>>>(t0, nc, g, l.dsig_t, l.W);
        CDS_LAUNCH_CHECK();
        for (int sum = 0; sum < 2; ++sum) {
            const int32_t nx = sum == 0 ? o : v, xoff = sum == 0 ? 0 : o;
            const int32_t ldk = sum == 0 ? l.ldk1 : l.ldk2;
            // dLq[t][x][J] (unscaled) = sum_c GA[(t, x)][c] Lov^T[J][c]
            int st = tr_split_gemm(precision, sum == 0 ? l.ga1_hi : l.ga2_hi,
                                   sum == 0 ? l.ga1_lo : l.ga2_lo, (int64_t)nc * nx, l.lovt_hi,
                                   l.lovt_lo, M, (int32_t)ov, l.ldc, nx, (int64_t)nmo * M, M, 1,
                                   d_Lp + ((int64_t)t0 * nmo + xoff) * M, false, l.err, stream);
            if (st) return st;
            // W_t Lq[t][x][J] as K-major rows J over (t, x)
            dim3 grid((unsigned)((M + kT - 1) / kT), (unsigned)(((int64_t)nc * nx + kT - 1) / kT));
            k_split_transpose<TF32><<<grid, dim3(kT, 8), 0, stream>>>(
                lp0 + (int64_t)xoff * M, (int64_t)nc * nx, M, nx, (int64_t)nmo * M, l.W + t0, ldk,
                (T*)l.lqt_hi, (T*)l.lqt_lo);
            CDS_LAUNCH_CHECK();
            // dLov[c][J] += sum_(t, x) GB[c][(t, x)] W_t Lq[t][x][J]
            st = tr_split_gemm(precision, sum == 0 ? l.gb1_hi : l.gb2_hi,
                               sum == 0 ? l.gb1_lo : l.gb2_lo, ov, l.lqt_hi, l.lqt_lo, M,
                               nc * nx, ldk, ov, 0, M, 1, d_Lov, true, l.err, stream);
            if (st) return st;
        }
        const int64_t per = (int64_t)nmo * M;
        k_scale_chunk<<<blocks(per * nc), 256, 0, stream>>>(d_Lp + (int64_t)t0 * per, per, nc, t0,
                                                            l.W);
        CDS_LAUNCH_CHECK();
    }
    int st = adj_finish(np, nmo, orb, g, l.dsig_t, l.deps_t, l.W, d_eps, stream);
    if (st) return st;
    int32_t h = 0;
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, l.err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    return h ? CDS_ERR_TIMEOUT : CDS_OK;
}

}  // namespace

size_t adj_tc_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np,
                              int32_t precision) {
    return tc_layout(nullptr, nmo, nocc, M, np, precision == CDS_PREC_TF32X3).bytes;
}

int adj_tc_gradient(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                    const int32_t* orb, int32_t np, const double* eps, const double* omega,
                    const double* g, int32_t precision, double* d_eps, double* d_Lov,
                    double* d_Lp, void* workspace, size_t workspace_bytes, cudaStream_t stream) {
    const bool tf32 = precision == CDS_PREC_TF32X3;
    // grid limits of the G pass (z = occupied index) and of the transposes
    const int64_t ov = (int64_t)nocc * (nmo - nocc);
    if (nocc > 65535 || (ov + kT - 1) / kT > 65535 || ov > INT32_MAX) return CDS_ERR_ARG;
    const TcLayout l = tc_layout(workspace, nmo, nocc, M, np, tf32);
    if (!workspace || workspace_bytes < l.bytes) return CDS_ERR_WORKSPACE;
    return tf32 ? gradient<true>(nmo, nocc, M, Lov, Lp, orb, np, eps, omega, g, precision, d_eps,
                                 d_Lov, d_Lp, l, stream)
                : gradient<false>(nmo, nocc, M, Lov, Lp, orb, np, eps, omega, g, precision, d_eps,
                                  d_Lov, d_Lp, l, stream);
}

}  // namespace cds
