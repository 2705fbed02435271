// AO -> MO transform of the Cholesky vectors (paper Eq. transformation),
// binary64:  B^K = C^T A^K C  with A^K the symmetric unpacked L^K.
//
// Per batch of kb vectors: unpack A^K (N x N), then two strided-batched FP64
// GEMMs per output block,  T = C_occ^T A^K  (o x N)  and  Bov = T C_vir
// (o x v), and the same for the requested orbital rows with C_P.  The second
// GEMM writes straight into the K-innermost layouts Lov[i][a][K], Lp[t][r][K].
// On this part FP64 issue rate, not HBM, bounds the transform.
//
// F32X2 (double-FP32) form for the split-precision pipeline: every operand is
// held as an (hi, lo) pair of floats (hi = fl32(x), lo = fl32(x - hi)) and
// every multiply-add keeps the exact product error (FMA) and the exact sum
// error (two-sum), ~2^-44 relative per operation on the 78 TFLOP/s FP32
// units instead of the 1.25 TFLOP/s FP64 ones.  Tensor-core splits cannot
// serve here: C = S^-1/2 Q has |C| up to ~1e3, the transform cancels ~1e6
// relative, and the tensor-core FP32 accumulation truncates.
#include <mutex>

#include "common.cuh"
#include "ao2mo_tc.cuh"

namespace cds {

constexpr int kGB = 64;   // output tile (rows and cols)
constexpr int kGK = 16;   // depth of a shared-memory stage
constexpr int kAoBatch = 32;

// Vectors per batch of the tensor-core forms in cds_cd_to_mo (all M vectors
// known up front): enough that the first GEMM has about 64 k rows (kb x N),
// so small bases do not run as many tiny launches; at least kAoBatch, at most
// M.  Each vector's results do not depend on the batch it is in.
static int32_t tr_batch(int32_t nbf, int32_t M) {
    const int32_t want = ((65536 / std::max(nbf, 1) + kAoBatch - 1) / kAoBatch) * kAoBatch;
    return std::max(1, std::min(M, std::max(kAoBatch, want)));
}

struct StridedMat {
    const double* p;
    int64_t rs, cs, bs;   // element strides: row, column, batch
};
struct StridedOut {
    double* p;
    int64_t rs, cs, bs;
};

// C[b] (m x n) = A[b] (m x k) * B[b] (k x n), all operands by strides.
// A_M_CONTIG: A's unit stride is along m; B_N_CONTIG: B's unit stride is along n.
template <bool A_M_CONTIG, bool B_N_CONTIG, bool ACC = false>
__global__ void __launch_bounds__(256)
k_dgemm(int m, int n, int k, StridedMat A, StridedMat B, StridedOut C) {
    __shared__ double As[kGK][kGB + 1];
    __shared__ double Bs[kGK][kGB + 1];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;
    const int m0 = blockIdx.y * kGB, n0 = blockIdx.x * kGB;
    const int64_t b = blockIdx.z;
    const double* Ab = A.p + b * A.bs;
    const double* Bb = B.p + b * B.bs;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < k; k0 += kGK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = tid + 256 * r;
            int mm, kk;
            if (A_M_CONTIG) { mm = idx % kGB; kk = idx / kGB; }
            else { kk = idx % kGK; mm = idx / kGK; }
            int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < m && gk < k) ? Ab[gm * A.rs + gk * A.cs] : 0.0;
            int nn;
            if (B_N_CONTIG) { nn = idx % kGB; kk = idx / kGB; }
            else { kk = idx % kGK; nn = idx / kGK; }
            int gn = n0 + nn;
            gk = k0 + kk;
            Bs[kk][nn] = (gn < n && gk < k) ? Bb[gk * B.rs + gn * B.cs] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    double* Cb = C.p + b * C.bs;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + tr + 16 * i;
        if (gm >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tc + 16 * j;
            if (gn < n) {
                double* dst = Cb + gm * C.rs + gn * C.cs;
                *dst = ACC ? *dst + acc[i][j] : acc[i][j];
            }
        }
    }
}

struct PairMat {
    const float2* p;
    int64_t rs, cs, bs;
};
template <typename T>
struct OutMat {
    T* p;
    int64_t rs, cs, bs;
};

// acc += a * b in (hi, lo) float-pair arithmetic.
__device__ __forceinline__ void df_fma(float2& acc, float2 a, float2 b) {
    const float p = a.x * b.x;
    float pe = fmaf(a.x, b.x, -p);        // exact error of the leading product
    pe = fmaf(a.x, b.y, pe);
    pe = fmaf(a.y, b.x, pe);
    const float s = acc.x + p;            // two-sum of the leading parts
    const float bp = s - acc.x;
    const float err = (acc.x - (s - bp)) + (p - bp);
    acc.x = s;
    acc.y += err + pe;
}

__device__ __forceinline__ void store_out(double* p, float2 v) { p[0] = (double)v.x + (double)v.y; }
__device__ __forceinline__ void store_out(float2* p, float2 v) {
    const float h = v.x + v.y;
    p[0] = make_float2(h, v.y - (h - v.x));
}

// C[b] = A[b] * B[b] in float-pair arithmetic.  Tile: 16*RM rows starting
// at row m_off + 16*RM*blockIdx.y, 64 columns; each of the 256 threads owns
// RM x 4 outputs.  The next K stage is fetched into registers while the
// current one is consumed from shared memory.  RM < 4 serves the last rows of
// a short m (the 20 orbital rows, the tail of o) without padding to 64.
#ifndef CDS_DFGEMM_PF
#define CDS_DFGEMM_PF 1
#endif
// PF: fetch the next K stage into registers during the current one (more
// registers: 2 instead of 3 blocks per SM for RM = 4).
constexpr bool kDfPrefetch = CDS_DFGEMM_PF != 0;

template <int RM, bool A_M_CONTIG, bool B_N_CONTIG, typename TOut>
__global__ void __launch_bounds__(256, (kDfPrefetch && RM == 4) ? 2 : 3)
k_dfgemm(int m, int n, int k, int m_off, PairMat A, PairMat B, OutMat<TOut> C) {
    constexpr int BM = 16 * RM;
    constexpr int NA = BM * kGK / 256;
    constexpr int NB = kGB * kGK / 256;
    __shared__ float2 As[kGK][BM + 1];
    __shared__ float2 Bs[kGK][kGB + 1];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;
    const int m0 = m_off + blockIdx.y * BM, n0 = blockIdx.x * kGB;
    const int64_t b = blockIdx.z;
    const float2* Ab = A.p + b * A.bs;
    const float2* Bb = B.p + b * B.bs;
    const float2 zero = make_float2(0.f, 0.f);
    float2 acc[RM][4];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = zero;
    float2 ra[NA], rb[NB];
    auto a_pos = [&](int r, int& mm, int& kk) {
        const int idx = tid + 256 * r;
        if (A_M_CONTIG) { mm = idx % BM; kk = idx / BM; }
        else { kk = idx % kGK; mm = idx / kGK; }
    };
    auto b_pos = [&](int r, int& nn, int& kk) {
        const int idx = tid + 256 * r;
        if (B_N_CONTIG) { nn = idx % kGB; kk = idx / kGB; }
        else { kk = idx % kGK; nn = idx / kGK; }
    };
    auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            int mm, kk;
            a_pos(r, mm, kk);
            const int gm = m0 + mm, gk = k0 + kk;
            ra[r] = (gm < m && gk < k) ? Ab[gm * A.rs + gk * A.cs] : zero;
        }
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            int nn, kk;
            b_pos(r, nn, kk);
            const int gn = n0 + nn, gk = k0 + kk;
            rb[r] = (gn < n && gk < k) ? Bb[gk * B.rs + gn * B.cs] : zero;
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            int mm, kk;
            a_pos(r, mm, kk);
            As[kk][mm] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            int nn, kk;
            b_pos(r, nn, kk);
            Bs[kk][nn] = rb[r];
        }
    };
    if (kDfPrefetch) {
        fetch(0);
        stash();
        __syncthreads();
    }
    for (int k0 = 0; k0 < k; k0 += kGK) {
        const bool more = k0 + kGK < k;
        if (!kDfPrefetch) {
            fetch(k0);
            stash();
            __syncthreads();
        } else if (more) {
            fetch(k0 + kGK);
        }
#pragma unroll 4
        for (int kk = 0; kk < kGK; ++kk) {
            float2 a[RM], bb[4];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) df_fma(acc[i][j], a[i], bb[j]);
        }
        __syncthreads();
        if (kDfPrefetch && more) {
            stash();
            __syncthreads();
        }
    }
    TOut* Cb = C.p + b * C.bs;
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        const int gm = m0 + tr + 16 * i;
        if (gm >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tc + 16 * j;
            if (gn < n) store_out(Cb + gm * C.rs + gn * C.cs, acc[i][j]);
        }
    }
}

__device__ __forceinline__ float2 to_pair(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// U[b][mu][nu] = pair(L[K0+b][pair(mu,nu)])
__global__ void k_unpack_pairs(const double* __restrict__ L, int64_t npair, int32_t K0,
                               int32_t kb, int32_t N, float2* __restrict__ U) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t per = (int64_t)N * N;
    if (e >= per * kb) return;
    int b = (int)(e / per);
    int64_t r = e - b * per;
    int mu = (int)(r / N), nu = (int)(r - (int64_t)mu * N);
    int lo = min(mu, nu), hi = max(mu, nu);
    U[e] = to_pair(L[(int64_t)(K0 + b) * npair + (int64_t)hi * (hi + 1) / 2 + lo]);
}

// The same from vectors already held as float pairs.
__global__ void k_unpack_f2(const float2* __restrict__ Lf, int64_t npair, int32_t K0, int32_t kb,
                            int32_t N, float2* __restrict__ U) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t per = (int64_t)N * N;
    if (e >= per * kb) return;
    int b = (int)(e / per);
    int64_t r = e - b * per;
    int mu = (int)(r / N), nu = (int)(r - (int64_t)mu * N);
    int lo = min(mu, nu), hi = max(mu, nu);
    U[e] = Lf[(int64_t)(K0 + b) * npair + (int64_t)hi * (hi + 1) / 2 + lo];
}

// Cq[mu][j] = pair(C[mu][col(j)]) with col(j) = j (all MOs) or orb[j].
__global__ void k_pair_cols(const double* __restrict__ C, int32_t N, int32_t nmo,
                            const int32_t* __restrict__ orb, int32_t ncol, float2* __restrict__ Cq) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * ncol) return;
    int mu = e / ncol, j = e % ncol;
    int p = orb ? orb[j] : j;
    Cq[e] = (p >= 0 && p < nmo) ? to_pair(C[(int64_t)mu * nmo + p])
                                : make_float2(__int_as_float(0x7fc00000), 0.f);
}

// Cj[mu][j] = pair(C[mu][j]) for j < nocc, pair(C[mu][orb[j - nocc]]) after.
__global__ void k_pair_cols_joint(const double* __restrict__ C, int32_t N, int32_t nmo,
                                  int32_t nocc, const int32_t* __restrict__ orb, int32_t np,
                                  float2* __restrict__ Cj) {
    const int nc = nocc + np;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * nc) return;
    int mu = e / nc, j = e % nc;
    int p = j < nocc ? j : orb[j - nocc];
    Cj[e] = (p >= 0 && p < nmo) ? to_pair(C[(int64_t)mu * nmo + p])
                                : make_float2(__int_as_float(0x7fc00000), 0.f);
}

// U[b][mu][nu] = L[K0+b][pair(mu,nu)]
__global__ void k_unpack(const double* __restrict__ L, int64_t npair, int32_t K0, int32_t kb,
                         int32_t N, double* __restrict__ U) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t per = (int64_t)N * N;
    if (e >= per * kb) return;
    int b = (int)(e / per);
    int64_t r = e - b * per;
    int mu = (int)(r / N), nu = (int)(r - (int64_t)mu * N);
    int lo = min(mu, nu), hi = max(mu, nu);
    U[e] = L[(int64_t)(K0 + b) * npair + (int64_t)hi * (hi + 1) / 2 + lo];
}

// Cp[mu][t] = C[mu][orb[t]]
__global__ void k_gather_cols(const double* __restrict__ C, int32_t N, int32_t nmo,
                              const int32_t* __restrict__ orb, int32_t np, double* __restrict__ Cp) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * np) return;
    int mu = e / np, t = e % np;
    int p = orb[t];
    Cp[e] = (p >= 0 && p < nmo) ? C[(int64_t)mu * nmo + p] : __longlong_as_double(0x7ff8000000000000LL);
}

template <bool AM, bool BN, bool ACC = false>
static int launch_dgemm(int m, int n, int k, int batch, StridedMat A, StridedMat B, StridedOut C,
                        cudaStream_t s) {
    if (m <= 0 || n <= 0 || batch <= 0) return CDS_OK;
    dim3 grid((n + kGB - 1) / kGB, (m + kGB - 1) / kGB, batch);
    k_dgemm<AM, BN, ACC><<<grid, 256, 0, s>>>(m, n, k, A, B, C);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

// Strided-batched FP64 GEMM for other translation units; picks the load
// pattern from the unit strides.  accumulate: C += A B (batch entries must
// then write disjoint C).
int launch_dgemm_strided(int m, int n, int k, int batch, const double* A, int64_t ars, int64_t acs,
                         int64_t abs_, const double* B, int64_t brs, int64_t bcs, int64_t bbs,
                         double* C, int64_t crs, int64_t ccs, int64_t cbs, cudaStream_t s,
                         bool accumulate = false) {
    StridedMat Am{A, ars, acs, abs_}, Bm{B, brs, bcs, bbs};
    StridedOut Cm{C, crs, ccs, cbs};
    const bool am = ars == 1, bn = bcs == 1;
    if (accumulate) {
        if (am && bn) return launch_dgemm<true, true, true>(m, n, k, batch, Am, Bm, Cm, s);
        if (am) return launch_dgemm<true, false, true>(m, n, k, batch, Am, Bm, Cm, s);
        if (bn) return launch_dgemm<false, true, true>(m, n, k, batch, Am, Bm, Cm, s);
        return launch_dgemm<false, false, true>(m, n, k, batch, Am, Bm, Cm, s);
    }
    if (am && bn) return launch_dgemm<true, true>(m, n, k, batch, Am, Bm, Cm, s);
    if (am) return launch_dgemm<true, false>(m, n, k, batch, Am, Bm, Cm, s);
    if (bn) return launch_dgemm<false, true>(m, n, k, batch, Am, Bm, Cm, s);
    return launch_dgemm<false, false>(m, n, k, batch, Am, Bm, Cm, s);
}

// U2[mu][b][nu] = L[K0+b][pair(mu,nu)] (vector index inside the row, so the
// contraction over (vector, nu) is one GEMM dimension).
__global__ void k_unpack_t(const double* __restrict__ L, int64_t npair, int32_t K0, int32_t kb,
                           int32_t N, double* __restrict__ U2) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * kb * N) return;
    const int nu = (int)(e % N);
    const int64_t r = e / N;
    const int b = (int)(r % kb), mu = (int)(r / kb);
    const int lo = min(mu, nu), hi = max(mu, nu);
    U2[e] = L[(int64_t)(K0 + b) * npair + (int64_t)hi * (hi + 1) / 2 + lo];
}

// dC[mu][orb[t]] += dCp[mu][t]
__global__ void k_scatter_cols(const double* __restrict__ dCp, int32_t N, int32_t np,
                               const int32_t* __restrict__ orb, int32_t nmo, double* __restrict__ dC) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    for (int t = 0; t < np; ++t) dC[(int64_t)e * nmo + orb[t]] += dCp[(int64_t)e * np + t];
}

// 64-row tiles for the bulk of m, then one narrower tile for the rest.
template <bool AM, bool BN, typename TOut>
static int launch_dfgemm(int m, int n, int k, int batch, PairMat A, PairMat B, OutMat<TOut> C,
                         cudaStream_t s) {
    if (m <= 0 || n <= 0 || batch <= 0) return CDS_OK;
    const unsigned gx = (unsigned)((n + kGB - 1) / kGB);
    const int full = m / 64 * 64, rest = m - full;
    if (full > 0) {
        k_dfgemm<4, AM, BN, TOut><<<dim3(gx, full / 64, batch), 256, 0, s>>>(m, n, k, 0, A, B, C);
        CDS_LAUNCH_CHECK();
    }
    if (rest > 32) {
        k_dfgemm<4, AM, BN, TOut><<<dim3(gx, 1, batch), 256, 0, s>>>(m, n, k, full, A, B, C);
        CDS_LAUNCH_CHECK();
    } else if (rest > 16) {
        k_dfgemm<2, AM, BN, TOut><<<dim3(gx, 1, batch), 256, 0, s>>>(m, n, k, full, A, B, C);
        CDS_LAUNCH_CHECK();
    } else if (rest > 0) {
        k_dfgemm<1, AM, BN, TOut><<<dim3(gx, 1, batch), 256, 0, s>>>(m, n, k, full, A, B, C);
        CDS_LAUNCH_CHECK();
    }
    return CDS_OK;
}

struct AoLayout {
    double* U;    // [kb][N][N]             (float pairs in the F32X2 form)
    double* T;    // [kb][o + np][N]
    double* Cp;   // [N][np]
    double* Cq;   // [N][nmo] float pairs of C (F32X2 form)
    double* Cj;   // [N][o + np] float pairs of C_occ and C_P (F32X2 form)
    size_t bytes;
};

static AoLayout ao_layout(void* ws, int32_t nbf, int32_t nmo, int32_t nocc, int32_t np) {
    Carver c(ws);
    AoLayout l;
    l.U = c.take<double>((size_t)kAoBatch * nbf * nbf);
    l.T = c.take<double>((size_t)kAoBatch * std::max(nocc + np, 1) * nbf);
    l.Cp = c.take<double>((size_t)nbf * std::max(np, 1));
    l.Cq = c.take<double>((size_t)nbf * nmo);
    l.Cj = c.take<double>((size_t)nbf * std::max(nocc + np, 1));
    l.bytes = c.off;
    return l;
}

// The float-pair transform.  Per batch of vectors one GEMM forms the
// occupied and the requested orbital rows together, T = [C_occ | C_P]^T A^K
// ((o + np) x N), then Lov = T_occ C_vir and Lp = T_P C.
static int f32x2_columns(int32_t N, int32_t nmo, int32_t nocc, const double* C, const int32_t* orb,
                         int32_t np, const AoLayout& lay, cudaStream_t stream) {
    const int32_t nc = nocc + np;
    k_pair_cols<<<(N * nmo + 255) / 256, 256, 0, stream>>>(C, N, nmo, nullptr, nmo,
                                                           reinterpret_cast<float2*>(lay.Cq));
    CDS_LAUNCH_CHECK();
    k_pair_cols_joint<<<(N * nc + 255) / 256, 256, 0, stream>>>(C, N, nmo, nocc, orb, np,
                                                                reinterpret_cast<float2*>(lay.Cj));
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

// Vectors [K0, K0 + kb) (FP64 rows of L, or float-pair rows when Lf is given)
// into Lov[i][a][K] and Lp[t][r][K], K stride ldK.
static int f32x2_batch(int32_t N, int32_t nmo, int32_t nocc, int32_t np, const double* L,
                       const float2* Lf, int32_t K0, int32_t kb, int64_t ldK, double* Lov,
                       double* Lp, const AoLayout& lay, cudaStream_t stream) {
    const int64_t npair = npair_of(N);
    const int32_t nv = nmo - nocc, nc = nocc + np;
    const float2* Cq = reinterpret_cast<const float2*>(lay.Cq);
    const float2* Cj = reinterpret_cast<const float2*>(lay.Cj);
    float2* U = reinterpret_cast<float2*>(lay.U);
    float2* T = reinterpret_cast<float2*>(lay.T);
    const bool ov = nocc > 0 && nv > 0;
    if ((!ov && np == 0) || kb <= 0) return CDS_OK;
    const int64_t tot = (int64_t)kb * N * N;
    if (Lf)
        k_unpack_f2<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(Lf, npair, K0, kb, N, U);
    else
        k_unpack_pairs<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(L, npair, K0, kb, N, U);
    CDS_LAUNCH_CHECK();
    PairMat Um{U, N, 1, (int64_t)N * N};
    // rows of the occupied block only when Lov is wanted
    const int32_t r0 = ov ? 0 : nocc, rows = nc - r0;
    int st = launch_dfgemm<true, true, float2>(rows, N, N, kb, PairMat{Cj + r0, 1, nc, 0}, Um,
                                               OutMat<float2>{T + (int64_t)r0 * N, N, 1,
                                                              (int64_t)nc * N},
                                               stream);
    if (st) return st;
    if (ov) {
        st = launch_dfgemm<false, true, double>(
            nocc, nv, N, kb, PairMat{T, N, 1, (int64_t)nc * N}, PairMat{Cq + nocc, nmo, 1, 0},
            OutMat<double>{Lov + K0, (int64_t)nv * ldK, ldK, 1}, stream);
        if (st) return st;
    }
    if (np > 0) {
        st = launch_dfgemm<false, true, double>(
            np, nmo, N, kb, PairMat{T + (int64_t)nocc * N, N, 1, (int64_t)nc * N},
            PairMat{Cq, nmo, 1, 0}, OutMat<double>{Lp + K0, (int64_t)nmo * ldK, ldK, 1}, stream);
        if (st) return st;
    }
    return CDS_OK;
}

static int cd_to_mo_f32x2(int32_t N, int32_t nmo, int32_t nocc, int32_t M, const double* L,
                          const double* C, const int32_t* orb, int32_t np, double* Lov,
                          double* Lp, const AoLayout& lay, cudaStream_t stream) {
    int st = f32x2_columns(N, nmo, nocc, C, orb, np, lay, stream);
    if (st) return st;
    for (int32_t K0 = 0; K0 < M; K0 += kAoBatch) {
        st = f32x2_batch(N, nmo, nocc, np, L, nullptr, K0, std::min(kAoBatch, M - K0), M, Lov, Lp,
                         lay, stream);
        if (st) return st;
    }
    return CDS_OK;
}

}  // namespace cds

using namespace cds;

extern "C" size_t cds_cd_to_mo_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc, int32_t M,
                                            int32_t np) {
    if (nbf <= 0 || nocc < 0 || np < 0) return 0;
    return std::max(ao_layout(nullptr, nbf, nmo, nocc, np).bytes,
                    tr_any_workspace_bytes(nbf, nmo, nocc, np, tr_batch(nbf, std::max(M, 1))));
}

extern "C" int cds_cd_to_mo(int32_t nbf, int32_t nmo, int32_t nocc, int32_t M, const double* L,
                         const double* C, const int32_t* orb, int32_t np, int32_t precision,
                         double* Lov, double* Lp, void* workspace, size_t workspace_bytes,
                         cudaStream_t stream) {
    if (nbf <= 0 || nmo <= 0 || nmo > nbf || nocc < 0 || nocc > nmo || M < 0 || np < 0)
        return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && precision != CDS_PREC_F32X2 && !is_tr_tc(precision))
        return CDS_ERR_UNSUPPORTED;
    if (M == 0) return CDS_OK;
    if (!L || !C || !Lov || (np > 0 && (!orb || !Lp))) return CDS_ERR_ARG;
    if (!workspace || workspace_bytes < cds_cd_to_mo_workspace_bytes(nbf, nmo, nocc, M, np))
        return CDS_ERR_WORKSPACE;
    if (is_tr_tc(precision)) {
        const int32_t kb = tr_batch(nbf, M);
        int st = tr_any_columns(precision, nbf, nmo, nocc, C, orb, np, kb, workspace, stream);
        for (int32_t K0 = 0; st == CDS_OK && K0 < M; K0 += kb)
            st = tr_any_batch(precision, nbf, nmo, nocc, np, L, nullptr, K0, std::min(kb, M - K0),
                              M, Lov, Lp, kb, workspace, stream);
        if (st) return st;
        return tr_any_status(precision, nbf, nmo, nocc, np, kb, workspace, stream);
    }
    AoLayout lay = ao_layout(workspace, nbf, nmo, nocc, np);
    if (precision == CDS_PREC_F32X2)
        return cd_to_mo_f32x2(nbf, nmo, nocc, M, L, C, orb, np, Lov, Lp, lay, stream);
    const int64_t npair = npair_of(nbf);
    const int32_t N = nbf, nv = nmo - nocc;
    if (np > 0) {
        k_gather_cols<<<(N * np + 255) / 256, 256, 0, stream>>>(C, N, nmo, orb, np, lay.Cp);
        CDS_LAUNCH_CHECK();
    }
    for (int32_t K0 = 0; K0 < M; K0 += kAoBatch) {
        int32_t kb = std::min(kAoBatch, M - K0);
        int64_t tot = (int64_t)kb * N * N;
        k_unpack<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(L, npair, K0, kb, N, lay.U);
        CDS_LAUNCH_CHECK();
        StridedMat U{lay.U, N, 1, (int64_t)N * N};
        if (nocc > 0 && nv > 0) {
            // T[b][i][nu] = sum_mu C[mu][i] U[b][mu][nu]
            StridedMat Aop{C, 1, nmo, 0};
            StridedOut Tout{lay.T, N, 1, (int64_t)nocc * N};
            int st = launch_dgemm<true, true>(nocc, N, N, kb, Aop, U, Tout, stream);
            if (st) return st;
            // Lov[i][a][K0+b] = sum_nu T[b][i][nu] C[nu][nocc+a]
            StridedMat Top{lay.T, N, 1, (int64_t)nocc * N};
            StridedMat Cv{C + nocc, nmo, 1, 0};
            StridedOut Out{Lov + K0, (int64_t)nv * M, M, 1};
            st = launch_dgemm<false, true>(nocc, nv, N, kb, Top, Cv, Out, stream);
            if (st) return st;
        }
        if (np > 0) {
            StridedMat Aop{lay.Cp, 1, np, 0};
            StridedOut Tout{lay.T, N, 1, (int64_t)np * N};
            int st = launch_dgemm<true, true>(np, N, N, kb, Aop, U, Tout, stream);
            if (st) return st;
            StridedMat Top{lay.T, N, 1, (int64_t)np * N};
            StridedMat Call{C, nmo, 1, 0};
            StridedOut Out{Lp + K0, (int64_t)nmo * M, M, 1};
            st = launch_dgemm<false, true>(np, nmo, N, kb, Top, Call, Out, stream);
            if (st) return st;
        }
    }
    return CDS_OK;
}

// Adjoint of the transform: given dl/dLov and dl/dLp, dl/dC through
//   Lov^K = C_occ^T A^K C_vir,   Lp^K[t] = C_{.,q_t}^T A^K C   (Eq. transformation):
//   dC_occ += A^K C_vir dLov^K^T,  dC_vir += A^K C_occ dLov^K,
//   dC_{.,q_t} += A^K C dLp^K[t]^T,  dC += A^K C_P dLp^K.
extern "C" size_t cds_cd_to_mo_backward_workspace_bytes(int32_t nbf, int32_t nmo, int32_t np) {
    if (nbf <= 0 || nmo <= 0 || np < 0) return 0;
    Carver c(nullptr);
    c.take<double>((size_t)nbf * kAoBatch * nbf);                       // U2
    c.take<double>((size_t)kAoBatch * nbf * std::max(nmo, np));          // T
    c.take<double>((size_t)nbf * std::max(np, 1));                       // C_P, dCp
    c.take<double>((size_t)nbf * std::max(np, 1));
    return c.off;
}

extern "C" int cds_cd_to_mo_backward(int32_t nbf, int32_t nmo, int32_t nocc, int32_t M,
                                     const double* L, const double* C, const int32_t* orb,
                                     int32_t np, const double* dLov, const double* dLp,
                                     double* dC, void* workspace, size_t workspace_bytes,
                                     cudaStream_t stream) {
    if (nbf <= 0 || nmo <= 0 || nmo > nbf || nocc <= 0 || nocc >= nmo || M < 0 || np < 0)
        return CDS_ERR_ARG;
    if (!L || !C || !dLov || !dC || (np > 0 && (!orb || !dLp))) return CDS_ERR_ARG;
    if (!workspace || workspace_bytes < cds_cd_to_mo_backward_workspace_bytes(nbf, nmo, np))
        return CDS_ERR_WORKSPACE;
    const int32_t N = nbf, nv = nmo - nocc;
    const int64_t npair = npair_of(nbf);
    Carver cv(workspace);
    double* U2 = cv.take<double>((size_t)N * kAoBatch * N);
    double* T = cv.take<double>((size_t)kAoBatch * N * std::max(nmo, np));
    double* Cp = cv.take<double>((size_t)N * std::max(np, 1));
    double* dCp = cv.take<double>((size_t)N * std::max(np, 1));
    CDS_CUDA_TRY(cudaMemsetAsync(dC, 0, sizeof(double) * (size_t)N * nmo, stream));
    if (np > 0) {
        k_gather_cols<<<(N * np + 255) / 256, 256, 0, stream>>>(C, N, nmo, orb, np, Cp);
        CDS_LAUNCH_CHECK();
        CDS_CUDA_TRY(cudaMemsetAsync(dCp, 0, sizeof(double) * (size_t)N * np, stream));
    }
    for (int32_t K0 = 0; K0 < M; K0 += kAoBatch) {
        const int32_t kb = std::min(kAoBatch, M - K0);
        const int64_t tot = (int64_t)N * kb * N;
        k_unpack_t<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(L, npair, K0, kb, N, U2);
        CDS_LAUNCH_CHECK();
        // T[b] = C_vir dLov^K^T   (N x o);  dLov^K[i][a] = dLov[(i v + a) M + K]
        int st = launch_dgemm_strided(N, nocc, nv, kb, C + nocc, nmo, 1, 0, dLov + K0, M,
                                      (int64_t)nv * M, 1, T, nocc, 1, (int64_t)N * nocc, stream);
        if (st) return st;
        st = launch_dgemm_strided(N, nocc, kb * N, 1, U2, (int64_t)kb * N, 1, 0, T, nocc, 1, 0, dC,
                                  nmo, 1, 0, stream, true);
        if (st) return st;
        // T[b] = C_occ dLov^K   (N x v)
        st = launch_dgemm_strided(N, nv, nocc, kb, C, nmo, 1, 0, dLov + K0, (int64_t)nv * M, M, 1, T,
                                  nv, 1, (int64_t)N * nv, stream);
        if (st) return st;
        st = launch_dgemm_strided(N, nv, kb * N, 1, U2, (int64_t)kb * N, 1, 0, T, nv, 1, 0,
                                  dC + nocc, nmo, 1, 0, stream, true);
        if (st) return st;
        if (np > 0) {
            // T[b] = C dLp^K^T   (N x np);  dLp^K[t][r] = dLp[(t nmo + r) M + K]
            st = launch_dgemm_strided(N, np, nmo, kb, C, nmo, 1, 0, dLp + K0, M, (int64_t)nmo * M, 1,
                                      T, np, 1, (int64_t)N * np, stream);
            if (st) return st;
            st = launch_dgemm_strided(N, np, kb * N, 1, U2, (int64_t)kb * N, 1, 0, T, np, 1, 0, dCp,
                                      np, 1, 0, stream, true);
            if (st) return st;
            // T[b] = C_P dLp^K   (N x nmo)
            st = launch_dgemm_strided(N, nmo, np, kb, Cp, np, 1, 0, dLp + K0, (int64_t)nmo * M, M, 1,
                                      T, nmo, 1, (int64_t)N * nmo, stream);
            if (st) return st;
            st = launch_dgemm_strided(N, nmo, kb * N, 1, U2, (int64_t)kb * N, 1, 0, T, nmo, 1, 0, dC,
                                      nmo, 1, 0, stream, true);
            if (st) return st;
        }
    }
    if (np > 0) {
        k_scatter_cols<<<(N + 255) / 256, 256, 0, stream>>>(dCp, N, np, orb, nmo, dC);
        CDS_LAUNCH_CHECK();
    }
    return CDS_OK;
}

// ===========================================================================
// Decomposition and transform as one pipelined call (float-pair form).  The
// transform of a batch of vectors needs only those vectors, so batch j is
// transformed on a second stream while the decomposition computes the next
// ones: the steps that stream nothing leave most of the GPU idle, and the
// transform GEMMs fill it.  The transform reads the float-pair rows directly
// and writes Lov / Lp with a K stride of max_rank (the rank is unknown until
// the end); two strided copies compact them at the end.
// ===========================================================================
namespace cds {
int& pipe_tr_ctas() {
    static thread_local int v = 0;
    return v;
}
namespace tc {
int tune_pipe_split();
}

namespace {

struct PipeStreams {
    cudaStream_t cd = nullptr, tr = nullptr;
};

int pipeline_streams(PipeStreams* out) {
    static std::mutex lock;
    static PipeStreams per_dev[64];
    int dev = 0;
    CDS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CDS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(lock);
    PipeStreams& p = per_dev[dev];
    if (!p.cd) {
        int lo = 0, hi = 0;
        CDS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CDS_CUDA_TRY(cudaStreamCreateWithPriority(&p.cd, cudaStreamNonBlocking, hi));
        CDS_CUDA_TRY(cudaStreamCreateWithPriority(&p.tr, cudaStreamNonBlocking, lo));
    }
    *out = p;
    return CDS_OK;
}

// stream `waiter` waits for the work enqueued so far on `on`
int stream_wait(cudaStream_t waiter, cudaStream_t on) {
    cudaEvent_t ev;
    CDS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CDS_CUDA_TRY(cudaEventRecord(ev, on));
    CDS_CUDA_TRY(cudaStreamWaitEvent(waiter, ev, 0));
    CDS_CUDA_TRY(cudaEventDestroy(ev));
    return CDS_OK;
}

struct FusedLayout {
    void* cd;
    size_t cd_bytes;
    AoLayout ao;       // float-pair transform
    void* tr;          // tensor-core transform (the same bytes as ao)
    double* lov_cap;   // [nocc][nv][max_rank]
    double* lp_cap;    // [np][nmo][max_rank]
    size_t bytes;
};

FusedLayout fused_layout(void* ws, int32_t nbf, int32_t nmo, int32_t nocc, int32_t max_rank,
                         int32_t np, int32_t cd_precision) {
    FusedLayout l;
    l.cd_bytes = cd_workspace_bytes_prec(nbf, max_rank, cd_precision);
    Carver c(ws);
    l.cd = c.take<char>(l.cd_bytes);
    const size_t ao_bytes = std::max(ao_layout(nullptr, nbf, nmo, nocc, np).bytes,
                                     tr_any_workspace_bytes(nbf, nmo, nocc, np, kAoBatch));
    char* ao = c.take<char>(ao_bytes);
    l.ao = ao_layout(ao, nbf, nmo, nocc, np);
    l.tr = ao;
    l.lov_cap = c.take<double>((size_t)std::max<int64_t>((int64_t)nocc * (nmo - nocc) * max_rank, 1));
    l.lp_cap = c.take<double>((size_t)std::max<int64_t>((int64_t)np * nmo * max_rank, 1));
    l.bytes = c.off;
    return l;
}

}  // namespace
}  // namespace cds

extern "C" size_t cds_cd_decompose_to_mo_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc,
                                                         int32_t max_rank, int32_t np,
                                                         int32_t cd_precision) {
    if (nbf <= 0 || nmo <= 0 || nmo > nbf || nocc < 0 || nocc > nmo || max_rank < 0 || np < 0)
        return 0;
    if (cd_precision != CDS_PREC_F32X2 && cd_precision != CDS_PREC_OZAKI) return 0;
    return fused_layout(nullptr, nbf, nmo, nocc, max_rank, np, cd_precision).bytes;
}

extern "C" int cds_cd_decompose_to_mo(int32_t nbf, const double* xyz, const double* alpha,
                                      const int32_t* atom, double delta, int32_t scheme,
                                      int32_t max_rank, const double* C, int32_t nmo,
                                      int32_t nocc, const int32_t* orb, int32_t np,
                                      int32_t tr_precision, int32_t cd_precision, double* L,
                                      int32_t* piv, double* D, int32_t* M_out,
                                      double* delta_eff_out, double* Lov, double* Lp,
                                      void* workspace, size_t workspace_bytes,
                                      cudaStream_t stream) {
    if (nbf <= 0 || nmo <= 0 || nmo > nbf || nocc < 0 || nocc > nmo || np < 0 || max_rank < 0)
        return CDS_ERR_ARG;
    if (!C || !Lov || !M_out || (np > 0 && (!orb || !Lp))) return CDS_ERR_ARG;
    if (tr_precision != CDS_PREC_F32X2 && !is_tr_tc(tr_precision)) return CDS_ERR_UNSUPPORTED;
    if (cd_precision != CDS_PREC_F32X2 && cd_precision != CDS_PREC_OZAKI) return CDS_ERR_UNSUPPORTED;
    const bool tcx = is_tr_tc(tr_precision);
    FusedLayout lay = fused_layout(workspace, nbf, nmo, nocc, max_rank, np, cd_precision);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    PipeStreams ps;
    int st = pipeline_streams(&ps);
    if (st) return st;
    if ((st = stream_wait(ps.cd, stream)) || (st = stream_wait(ps.tr, stream))) return st;
    st = tcx ? tr_any_columns(tr_precision, nbf, nmo, nocc, C, orb, np, kAoBatch, lay.tr, ps.tr)
             : f32x2_columns(nbf, nmo, nocc, C, orb, np, lay.ao, ps.tr);
    if (st) return st;
    const float2* Lf = reinterpret_cast<const float2*>(L);
    // vectors [K0, K0 + kb) from float-pair rows (Lf) or FP64 rows (L)
    auto transform = [&](const double* Ld, const float2* Lq, int32_t K0, int32_t kb) -> int {
        return tcx ? tr_any_batch(tr_precision, nbf, nmo, nocc, np, Ld, Lq, K0, kb, max_rank,
                                  lay.lov_cap, lay.lp_cap, kAoBatch, lay.tr, ps.tr)
                   : f32x2_batch(nbf, nmo, nocc, np, Ld, Lq, K0, kb, max_rank, lay.lov_cap,
                                 lay.lp_cap, lay.ao, ps.tr);
    };
    // the SM split while this thread runs the pipeline
    struct SplitGuard {
        SplitGuard(int v) { pipe_tr_ctas() = v; }
        ~SplitGuard() { pipe_tr_ctas() = 0; }
    } split_guard(tcx ? tc::tune_pipe_split() : 0);
    // The tensor-core decomposition never reads L's rows once they are
    // written (it works on its compact copy), so each batch's rows go to FP64
    // right after their transform, on the transform's stream, instead of all
    // rows at the end; the float-pair decomposition keeps reading them, so
    // it converts at the end.
    const bool convert_by_batch = cd_precision == CDS_PREC_OZAKI;
    const int64_t npr = npair_of(nbf);
    int32_t next = 0;   // first vector not yet handed to the transform
    CdChunkHook hook = [&](int32_t rows, bool done) -> int {
        while (next < rows && (done || next + kAoBatch <= rows)) {
            const int32_t kb = std::min(kAoBatch, rows - next);
            int s2 = transform(nullptr, Lf, next, kb);
            if (!s2 && convert_by_batch) s2 = pairs_to_fp64(L + (int64_t)next * npr, kb * npr, ps.tr);
            if (s2) return s2;
            next += kb;
        }
        return CDS_OK;
    };
    int32_t M = 0;
    const int cd_st = cd_decompose_run(nbf, xyz, alpha, atom, delta, scheme, max_rank,
                                       cd_precision, L, piv, D, &M, delta_eff_out, lay.cd,
                                       lay.cd_bytes, ps.cd, &hook, ps.tr, true, !convert_by_batch);
    *M_out = M;
    const int32_t nv = nmo - nocc;
    if (convert_by_batch && next < M) {   // rows no batch took (a stop before the last check)
        if ((st = stream_wait(ps.tr, ps.cd))) return st;
        if ((st = pairs_to_fp64(L + (int64_t)next * npr, (int64_t)(M - next) * npr, ps.tr)))
            return st;
    }
    if (M > 0 && (cd_st == CDS_OK || cd_st == CDS_ERR_RANK_CAP)) {
        // the last host check reports the stop, so every vector has been
        // handed over; should any remain, take them from the converted rows
        if (next < M) {
            if ((st = stream_wait(ps.tr, ps.cd))) return st;
            for (; next < M; next += kAoBatch)
                if ((st = transform(L, nullptr, next, std::min(kAoBatch, M - next)))) return st;
        }
        if (nocc > 0 && nv > 0)
            CDS_CUDA_TRY(cudaMemcpy2DAsync(Lov, (size_t)M * sizeof(double), lay.lov_cap,
                                           (size_t)max_rank * sizeof(double),
                                           (size_t)M * sizeof(double), (size_t)nocc * nv,
                                           cudaMemcpyDeviceToDevice, ps.tr));
        if (np > 0)
            CDS_CUDA_TRY(cudaMemcpy2DAsync(Lp, (size_t)M * sizeof(double), lay.lp_cap,
                                           (size_t)max_rank * sizeof(double),
                                           (size_t)M * sizeof(double), (size_t)np * nmo,
                                           cudaMemcpyDeviceToDevice, ps.tr));
    }
    if ((st = stream_wait(stream, ps.cd)) || (st = stream_wait(stream, ps.tr))) return st;
    if (tcx && M > 0 &&
        (st = tr_any_status(tr_precision, nbf, nmo, nocc, np, kAoBatch, lay.tr, stream)))
        return st;
    return cd_st;
}
