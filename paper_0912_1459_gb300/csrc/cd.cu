// Threshold-delta diagonal-pivoted Cholesky decomposition of the ERI
// supermatrix, columns generated on the fly (paper Sec. II.A, Eq. gs_coulomb,
// Eq. CD, Eq. stricterr).
//
// Left-looking form of the Gram-Schmidt steps: at step k with pivot P,
//   L^k_I = [ (rho_I|rho_P) - sum_{K<k} L^K_I L^K_P ] / sqrt(D_P),
//   D_I  -= (L^k_I)^2,  D_P := 0,
// then the next pivot is the largest candidate residual (lowest index among
// values within 1e-12 * max initial diagonal).  A step is two launches:
// k_cd_project makes the integral column (FP64, on a few blocks) while its
// other blocks stream L[0:k][*] once for the projections (coalesced along I);
// k_cd_update forms L^k and the residuals, and the last of its blocks to
// arrive finishes the grid-wide extrema and picks the next pivot (no spin
// waits).  k_cd_select picks the first pivot only.
// The float-pair form streams L only at the first step of a batch, forming
// the projections of four candidate pivots at once (k_cd_project_spec);
// steps whose pivot is among them reuse those (cd_spec_dot_body).  Its
// integral column is in float pairs as well (eri_column_df).
// All kernels read a device control block and return at once after the
// decomposition has stopped, so the host enqueues steps ahead and checks the
// control block only every few steps.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "cd.cuh"
#include "eri_col.cuh"
#include "sigma_tc.cuh"

namespace cds {

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ long long warp_min_ll(long long v) {
    for (int o = 16; o; o >>= 1) {
        long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Block-wide max / min of two doubles; result valid in thread 0.
__device__ void block_maxmin(double& mx, double& mn) {
    __shared__ double smx[32], smn[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    mx = warp_max(mx);
    mn = warp_min(mn);
    if (lane == 0) { smx[w] = mx; smn[w] = mn; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        mx = lane < nw ? smx[lane] : -INFINITY;
        mn = lane < nw ? smn[lane] : INFINITY;
        mx = warp_max(mx);
        mn = warp_min(mn);
    }
    __syncthreads();
}

// True (in every thread) for the last of nblk blocks to finish, after the
// partials of all of them are visible.
__device__ bool last_block(unsigned int* counter, int nblk) {
    __shared__ bool am_last;
    __threadfence();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == (unsigned int)nblk - 1);
    }
    __syncthreads();
    return am_last;
}

// D = initial diagonal, candidate mask, scale = max D, G = max candidate D.
// bid / nblk: this block's index and the number of blocks working on the
// molecule (the grid of the single-molecule kernel, a slice of a batch grid).
__device__ void cd_init_body(PairSoA pd, const int32_t* __restrict__ atom, int32_t scheme,
                             int64_t n, double delta, double* __restrict__ D,
                             uint8_t* __restrict__ cand, double* __restrict__ blk_a,
                             double* __restrict__ blk_b, CdCtrl* ctrl, int bid, int nblk,
                             bool given = false) {
    double mx_all = -INFINITY, mx_cand = -INFINITY;
    for (int64_t I = bid * (int64_t)blockDim.x + threadIdx.x; I < n;
         I += (int64_t)nblk * blockDim.x) {
        double d;
        if (given) {   // the diagonal was made by another integral kernel (contracted shells)
            d = D[I];
        } else {
            double p = pd.p[I], px = pd.Px[I], py = pd.Py[I], pz = pd.Pz[I], k = pd.Kp[I];
            d = eri_pair(p, px, py, pz, k, p, px, py, pz, k);
            D[I] = d;
        }
        uint8_t c = 1;
        if (scheme == CDS_SCHEME_ATOMIC) {
            int32_t mu, nu;
            unpack_pair(I, mu, nu);
            c = atom[mu] == atom[nu];
        }
        cand[I] = c;
        mx_all = fmax(mx_all, d);
        if (c) mx_cand = fmax(mx_cand, fmax(d, 0.0));
    }
    double a = mx_all, b = -mx_cand;   // reuse max/min: min(-x) = -max(x)
    block_maxmin(a, b);
    if (threadIdx.x == 0) { blk_a[bid] = a; blk_b[bid] = b; }
    if (last_block(&ctrl->counter, nblk)) {
        double A = -INFINITY, B = INFINITY;
        for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
            A = fmax(A, __ldcg(blk_a + i));
            B = fmin(B, __ldcg(blk_b + i));
        }
        block_maxmin(A, B);
        if (threadIdx.x == 0) {
            ctrl->scale = A;
            ctrl->delta_eff = fmax(delta, (double)n * 2.220446049250313e-16 * A);
            ctrl->G = -B;
            ctrl->Dmin = 0.0;
            ctrl->done = 0;
            ctrl->status = CDS_OK;
            ctrl->M = 0;
            ctrl->counter = 0;
        }
    }
}

__global__ void k_cd_init(PairSoA pd, const int32_t* __restrict__ atom, int32_t scheme, int64_t n,
                          double delta, double* __restrict__ D, uint8_t* __restrict__ cand,
                          double* __restrict__ blk_a, double* __restrict__ blk_b, CdCtrl* ctrl,
                          int given = 0) {
    cd_init_body(pd, atom, scheme, n, delta, D, cand, blk_a, blk_b, ctrl, blockIdx.x, gridDim.x,
                 given != 0);
}

// Pivot for vector k (k vectors already made): stop test, rank cap, then the
// lowest candidate index with max(D,0) >= G - 1e-12*scale and D > delta_eff.
__device__ void cd_select_body(int64_t n, int32_t k, int32_t max_rank,
                               const double* __restrict__ D, const uint8_t* __restrict__ cand,
                               long long* __restrict__ blk_i, int32_t* __restrict__ piv,
                               CdCtrl* ctrl, int bid, int nblk) {
    if (ctrl->done) return;
    double G = ctrl->G, de = ctrl->delta_eff, scale = ctrl->scale;
    if (ctrl->Dmin < -kNotPdRel * scale || !(G == G)) {
        if (bid == 0 && threadIdx.x == 0) {
            ctrl->status = CDS_ERR_NOT_PD; ctrl->done = 1; ctrl->M = k;
        }
        return;
    }
    if (G <= de) {
        if (bid == 0 && threadIdx.x == 0) { ctrl->done = 1; ctrl->M = k; }
        return;
    }
    if (k >= max_rank) {
        if (bid == 0 && threadIdx.x == 0) {
            ctrl->status = CDS_ERR_RANK_CAP; ctrl->done = 1; ctrl->M = k;
        }
        return;
    }
    double thr = G - kTieRel * scale;
    long long best = LLONG_MAX;
    for (int64_t I = bid * (int64_t)blockDim.x + threadIdx.x; I < n;
         I += (int64_t)nblk * blockDim.x) {
        double d = D[I];
        if (cand[I] && fmax(d, 0.0) >= thr && d > de) { best = (long long)I; break; }
    }
    __shared__ long long sb[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    best = warp_min_ll(best);
    if (lane == 0) sb[w] = best;
    __syncthreads();
    if (w == 0) {
        best = lane < (int)(blockDim.x >> 5) ? sb[lane] : LLONG_MAX;
        best = warp_min_ll(best);
        if (lane == 0) blk_i[bid] = best;
    }
    if (last_block(&ctrl->counter, nblk)) {
        long long b = LLONG_MAX;
        for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
            long long v = __ldcg(blk_i + i);
            b = v < b ? v : b;
        }
        b = warp_min_ll(b);
        if (lane == 0) sb[w] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long m = LLONG_MAX;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = sb[i] < m ? sb[i] : m;
            if (m < 0 || m >= n) {
                // no candidate passed the test although G > delta_eff: the
                // residual diagonal holds NaN or is otherwise inconsistent
                ctrl->status = CDS_ERR_NOT_PD; ctrl->done = 1; ctrl->M = k;
            } else {
                ctrl->P = m;
                ctrl->DP = __ldcg(D + m);
                ctrl->rDP = 1.0 / sqrt(ctrl->DP);
                {
                    const float h = (float)ctrl->rDP;
                    ctrl->rDPf = make_float2(h, (float)(ctrl->rDP - (double)h));
                }
                piv[k] = (int32_t)m;
                ctrl->S[0] = m;
                for (int i = 1; i < kSpec; ++i) ctrl->S[i] = -1;
                ctrl->STc[0] = m;
                for (int i = 1; i < kSpecTC; ++i) ctrl->STc[i] = -1;
                ctrl->k0 = k;
                ctrl->slot = 0;
                ctrl->pass = 1;
                ctrl->passes = 1;
                ctrl->streamed = k;
                ctrl->extra = 0;
            }
            ctrl->counter = 0;
        }
    }
}

__global__ void k_cd_select(int64_t n, int32_t k, int32_t max_rank, const double* __restrict__ D,
                            const uint8_t* __restrict__ cand, long long* __restrict__ blk_i,
                            int32_t* __restrict__ piv, CdCtrl* ctrl) {
    cd_select_body(n, k, max_rank, D, cand, blk_i, piv, ctrl, blockIdx.x, gridDim.x);
}

// Integral column of step k (pivot ctrl->P) into ecol, FP64 or float pairs.
__device__ __forceinline__ void cd_eri_body_df(PairSoA pd, PairF2 pf, int64_t n,
                                               const CdCtrl* ctrl, float2* __restrict__ ecol,
                                               int bid, int nblk) {
    eri_column_df<kUpdThreads>(pd, pf, n, ctrl->P, ecol, bid, nblk);
}

__device__ __forceinline__ void cd_eri_body(PairSoA pd, int64_t n, const CdCtrl* ctrl,
                                            double* __restrict__ ecol, int bid, int nblk) {
    eri_column_fp64<kUpdThreads>(pd, n, ctrl->P, ecol, bid, nblk);
}

// Projection sum_{K<k} L^K_I L^K_P for one tile of kUpdPairs pairs, stored in
// row k of L (the slot vector k will occupy).  Lane l of every warp holds
// pairs l and l + 32 of the tile; the kUpdWarps warps split the K sum (warp w
// takes the staged rows j = w mod kUpdWarps, four rows per iteration: 8 loads
// of L in flight per thread), and their partial sums are added in a fixed
// order, so the result does not depend on scheduling.
//
// DF: the stored vectors are (hi, lo) float pairs in the 8 bytes of each L
// element, and the projection runs and is stored in float-pair arithmetic on
// the FP32 units.
template <bool DF>
__device__ __forceinline__ void cd_dot_body(int64_t n, int32_t k, double* __restrict__ L,
                                            const CdCtrl* ctrl, int tile) {
    __shared__ double lp_raw[kCdChunk];
    __shared__ double red[kUpdWarps][kUpdPairs];
    const int64_t P = ctrl->P;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)tile * kUpdPairs;
    int64_t Ic[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int64_t I = base + lane + 32 * r;
        Ic[r] = I < n ? I : 0;   // dead lanes read pair 0
    }
    double dot[2][4] = {};
    float2 dfd[2][4];
    if constexpr (DF) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int u = 0; u < 4; ++u) dfd[r][u] = make_float2(0.f, 0.f);
    }
    for (int K0 = 0; K0 < k; K0 += kCdChunk) {
        const int kc = min(kCdChunk, k - K0);
        __syncthreads();
        for (int j = threadIdx.x; j < kc; j += blockDim.x) lp_raw[j] = L[(int64_t)(K0 + j) * n + P];
        __syncthreads();
        int j = w;
        constexpr int S = kUpdWarps;
        if constexpr (DF) {
            const float2* lp = reinterpret_cast<const float2*>(lp_raw);
            const float2* src = reinterpret_cast<const float2*>(L) + (int64_t)K0 * n;
            for (; j + 3 * S < kc; j += 4 * S) {
                float2 v[4][2];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int r = 0; r < 2; ++r) v[u][r] = src[(int64_t)(j + u * S) * n + Ic[r]];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 lu = lp[j + u * S];
#pragma unroll
                    for (int r = 0; r < 2; ++r) df_fma(dfd[r][u], v[u][r], lu);
                }
            }
            for (; j < kc; j += S) {
#pragma unroll
                for (int r = 0; r < 2; ++r) df_fma(dfd[r][0], src[(int64_t)j * n + Ic[r]], lp[j]);
            }
        } else {
            const double* lp = lp_raw;
            const double* src = L + (int64_t)K0 * n;
            for (; j + 3 * S < kc; j += 4 * S) {
                double v[4][2];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int r = 0; r < 2; ++r) v[u][r] = src[(int64_t)(j + u * S) * n + Ic[r]];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const double lu = lp[j + u * S];
#pragma unroll
                    for (int r = 0; r < 2; ++r) dot[r][u] = fma(v[u][r], lu, dot[r][u]);
                }
            }
            for (; j < kc; j += S) {
#pragma unroll
                for (int r = 0; r < 2; ++r) dot[r][0] = fma(src[(int64_t)j * n + Ic[r]], lp[j], dot[r][0]);
            }
        }
    }
    float2(*red2)[kUpdPairs] = reinterpret_cast<float2(*)[kUpdPairs]>(red);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if constexpr (DF)
            red2[w][lane + 32 * r] = df_add(df_add(dfd[r][0], dfd[r][1]), df_add(dfd[r][2], dfd[r][3]));
        else
            red[w][lane + 32 * r] = (dot[r][0] + dot[r][1]) + (dot[r][2] + dot[r][3]);
    }
    __syncthreads();
    const int64_t I = base + threadIdx.x;
    if (threadIdx.x < kUpdPairs && I < n) {
        if constexpr (DF) {
            float2 sum = red2[0][threadIdx.x];
#pragma unroll
            for (int v = 1; v < kUpdWarps; ++v) sum = df_add(sum, red2[v][threadIdx.x]);
            reinterpret_cast<float2*>(L)[(int64_t)k * n + I] = sum;
        } else {
            double sum = red[0][threadIdx.x];
#pragma unroll
            for (int v = 1; v < kUpdWarps; ++v) sum += red[v][threadIdx.x];
            L[(int64_t)k * n + I] = sum;
        }
    }
}

// Speculative projections (float-pair mode).  At the first step k0 of a
// batch one pass over L[0:k0] forms, for the batch's kSpec candidate pivots
// S_s (S_0 is the step's own pivot),
//   G_s[I] = sum_{K<k0} L^K_I L^K_{S_s}      (float pairs, [kSpec][npair]).
// A later step k of the batch whose pivot is S_s takes its projection as
// G_s[I] + sum_{k0<=K<k} L^K_I L^K_{S_s} and streams nothing; a pivot outside
// the set, or a full batch, starts the next batch.  The sums are the same as
// the plain left-looking ones, grouped differently.  Tile layout as
// cd_dot_body, with kSpec accumulators per pair instead of four partial sums.
static_assert(kUpdWarps * kUpdPairs <= kSpecChunk, "warp partials fit the staging buffer");
__device__ __forceinline__ void cd_spec_dot_body(int64_t n, int32_t k,
                                                 const double* __restrict__ L,
                                                 float2* __restrict__ G, const CdCtrl* ctrl,
                                                 int tile) {
    __shared__ float2 lp[kSpec][kSpecChunk];   // pivot columns; then the warp partials
    __shared__ long long S[kSpec];
    if (threadIdx.x < kSpec) S[threadIdx.x] = ctrl->S[threadIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)tile * kUpdPairs;
    int64_t Ic[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int64_t I = base + lane + 32 * r;
        Ic[r] = I < n ? I : 0;   // dead lanes read pair 0
    }
    float2 acc[2][kSpec];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < kSpec; ++c) acc[r][c] = make_float2(0.f, 0.f);
    const float2* Lf = reinterpret_cast<const float2*>(L);
    constexpr int SW = kUpdWarps;
    for (int K0 = 0; K0 < k; K0 += kSpecChunk) {
        const int kc = min(kSpecChunk, k - K0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kSpec * kc; idx += blockDim.x) {
            const int c = idx / kc, j = idx - c * kc;
            lp[c][j] = S[c] >= 0 ? Lf[(int64_t)(K0 + j) * n + S[c]] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2* src = Lf + (int64_t)K0 * n;
        int j = w;
        for (; j + (kSpecRows - 1) * SW < kc; j += kSpecRows * SW) {
            float2 v[kSpecRows][2];
#pragma unroll
            for (int u = 0; u < kSpecRows; ++u)
#pragma unroll
                for (int r = 0; r < 2; ++r) v[u][r] = src[(int64_t)(j + u * SW) * n + Ic[r]];
#pragma unroll
            for (int u = 0; u < kSpecRows; ++u)
#pragma unroll
                for (int c = 0; c < kSpec; ++c) {
                    const float2 lu = lp[c][j + u * SW];
#pragma unroll
                    for (int r = 0; r < 2; ++r) df_fma(acc[r][c], v[u][r], lu);
                }
        }
        for (; j < kc; j += SW) {
            float2 v[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) v[r] = src[(int64_t)j * n + Ic[r]];
#pragma unroll
            for (int c = 0; c < kSpec; ++c)
#pragma unroll
                for (int r = 0; r < 2; ++r) df_fma(acc[r][c], v[r], lp[c][j]);
        }
    }
    __syncthreads();
    float2(*red)[kSpec][kUpdPairs] = reinterpret_cast<float2(*)[kSpec][kUpdPairs]>(&lp[0][0]);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < kSpec; ++c) red[w][c][lane + 32 * r] = acc[r][c];
    __syncthreads();
    for (int idx = threadIdx.x; idx < kSpec * kUpdPairs; idx += blockDim.x) {
        const int c = idx / kUpdPairs, pp = idx - c * kUpdPairs;
        const int64_t I = base + pp;
        if (I < n) {
            float2 sum = red[0][c][pp];
#pragma unroll
            for (int v = 1; v < kUpdWarps; ++v) sum = df_add(sum, red[v][c][pp]);
            G[(int64_t)c * n + I] = sum;
        }
    }
    __syncthreads();   // red aliases lp, which the next tile restages
}

// ---------------------------------------------------------------------------
// Exact-slice tensor-core form (CDS_PREC_OZAKI).  Every stored element L^K_I
// is kept, besides its float pair in L, as a 56-bit fixed-point number below
// the pair's scale sigma_I = 2^e_I > sqrt(D0_I) >= |L^K_I| (the residual
// matrix stays positive semidefinite, so sum_K (L^K_I)^2 <= D0_I), cut into
// eight 7-bit digits held as exact BF16 slices in a store blocked by
// 32-column groups, [group][slice][pair][32] (one group's tile of 128 pairs
// is 8 KB of contiguous memory per slice); a streaming pass multiplies the
// store with the candidates' rows on the tensor cores (cd_tc.cu).
// ---------------------------------------------------------------------------
__global__ void k_cd_tc_scales(const double* __restrict__ D, int64_t n, float* __restrict__ sig) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= n) return;
    const double r = sqrt(fmax(D[I], 0.0));
    int e = 0;
    if (r > 0.0) frexp(r, &e);   // r = f 2^e, f in [0.5, 1): r < 2^e
    sig[I] = ldexpf(1.f, e);
}

// The digit slices of x / sigma (sigma = 2^e > |x|), x a float pair:
// q = trunc(x 2^(Q-e)) (|q| < 2^Q, Q = 56 bits), digit s = bits
// [Q-7(s+1), Q-7s) of |q|, slice s = sign(x) digit 2^(-7(s+1)) (exact in BF16).
__device__ __forceinline__ void tc_slices(float2 x, int e, uint16_t (&out)[kSlicesTC]) {
    constexpr int QB = kSlicesTC * kBitsTC;
    long long q = __float2ll_rz(ldexpf(x.x, QB - e)) + __float2ll_rz(ldexpf(x.y, QB - e));
    const long long qmax = (1LL << QB) - 1;
    q = q > qmax ? qmax : (q < -qmax ? -qmax : q);
    const bool neg = q < 0;
    const unsigned long long aq = (unsigned long long)(neg ? -q : q);
#pragma unroll
    for (int s = 0; s < kSlicesTC; ++s) {
        const int d = (int)((aq >> (QB - kBitsTC * (s + 1))) & ((1ull << kBitsTC) - 1));
        out[s] = __bfloat16_as_ushort(__float2bfloat16_rn(ldexpf((float)(neg ? -d : d),
                                                                 -kBitsTC * (s + 1))));
    }
}

// Eight consecutive columns K0.. K0+7 (zero at K >= k) of one row of L, sliced
// with exponent e, stored as one 16-byte segment per slice: row `row` of a
// group-blocked store [group][slice][rows][kGroupTC].
__device__ __forceinline__ void tc_store8(const float2* __restrict__ Lf, int64_t n, int64_t I,
                                          int32_t K0, int32_t k, int e,
                                          __nv_bfloat16* __restrict__ store, int64_t rows,
                                          int64_t row) {
    const int64_t plane = rows * kGroupTC;
    const int64_t off = ((int64_t)(K0 / kGroupTC) * kSlicesTC * rows + row) * kGroupTC +
                        K0 % kGroupTC;
    uint32_t w[kSlicesTC][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        uint16_t d0[kSlicesTC], d1[kSlicesTC];
        const float2 v0 = (I >= 0 && K0 + j < k) ? Lf[(int64_t)(K0 + j) * n + I] : make_float2(0.f, 0.f);
        const float2 v1 = (I >= 0 && K0 + j + 1 < k) ? Lf[(int64_t)(K0 + j + 1) * n + I]
                                                     : make_float2(0.f, 0.f);
        tc_slices(v0, e, d0);
        tc_slices(v1, e, d1);
#pragma unroll
        for (int s = 0; s < kSlicesTC; ++s) w[s][j / 2] = (uint32_t)d0[s] | ((uint32_t)d1[s] << 16);
    }
#pragma unroll
    for (int s = 0; s < kSlicesTC; ++s)
        *reinterpret_cast<uint4*>(store + s * plane + off) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// Order-preserving map of binary64 values to int64 (its own inverse), so the
// residual extrema reduce on the integer units instead of the narrow FP64 pipe.
__device__ __forceinline__ long long key_of(double d) {
    const long long b = __double_as_longlong(d);
    return b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
}
__device__ __forceinline__ double value_of(long long s) {
    return __longlong_as_double(s < 0 ? (s ^ 0x7fffffffffffffffLL) : s);
}
__device__ __forceinline__ long long warp_max_ll(long long v) {
    for (int o = 16; o; o >>= 1) {
        long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}
// Block-wide max / min of two int64 values, returned in every thread.
__device__ void block_maxmin_ll(long long& mx, long long& mn) {
    __shared__ long long smx[32], smn[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    mx = warp_max_ll(mx);
    mn = warp_min_ll(mn);
    if (lane == 0) { smx[w] = mx; smn[w] = mn; }
    __syncthreads();
    if (w == 0) {
        long long a = lane < nw ? smx[lane] : LLONG_MIN;
        long long b = lane < nw ? smn[lane] : LLONG_MAX;
        a = warp_max_ll(a);
        b = warp_min_ll(b);
        if (lane == 0) { smx[0] = a; smn[0] = b; }
    }
    __syncthreads();
    mx = smx[0];
    mn = smn[0];
    __syncthreads();
}
__device__ long long block_min_ll(long long v) {
    long long dummy = LLONG_MIN;
    block_maxmin_ll(dummy, v);
    return v;
}

// Vector k, the residual update and the pivot of step k+1, one launch:
//   L^k_I = (ecol_I - proj_I) / sqrt(D_P),  D_I -= (L^k_I)^2,  D_P := 0.
// Block b owns the contiguous pairs [b*kStepChunk, (b+1)*kStepChunk) and
// records the largest candidate max(D,0) and the smallest D of its range.
// The last block to arrive finishes both extrema, applies the stop tests and,
// if the decomposition goes on, picks the next pivot: the lowest candidate
// index with max(D,0) >= G - 1e-12*scale and D > delta_eff.  That index lies
// in the lowest block whose own maximum passes the test (a block maximum that
// passes without any entry passing, possible only when the band reaches below
// delta_eff, moves the search to the next such block).  DF: proj and L^k are
// (hi, lo) float pairs.
template <bool DF, bool SPEC, bool TC = false>
__device__ __forceinline__ void cd_step_body(int64_t n, int32_t k, int32_t max_rank,
                                             double* __restrict__ L, double* __restrict__ D,
                                             const uint8_t* __restrict__ cand,
                                             const double* __restrict__ ecol,
                                             const float2* __restrict__ Gp,
                                             long long* __restrict__ blk_a,
                                             long long* __restrict__ blk_b,
                                             long long* __restrict__ blk_i,
                                             int32_t* __restrict__ piv, CdCtrl* ctrl, int bid,
                                             int nblk, PairF2 pf = PairF2{}) {
    static_assert(!SPEC || DF, "speculative projections are a float-pair mode");
    static_assert(!TC || SPEC, "the tensor-core form is a speculative form");
    const int64_t P = ctrl->P;
    const double rDP = ctrl->rDP;
    const float2 rDPf = ctrl->rDPf;
    long long mx = -1, mn = LLONG_MAX;   // bits of max(D,0) over candidates (-1: none), key of min D
    const int64_t base = (int64_t)bid * kStepChunk;
    // SPEC: projection = G_slot + the vectors made since the batch began
    int32_t k0 = 0, extra = 0;
    const float2* Gs = Gp;
    float2 lpP[kSpec - 1];
    __shared__ float2 s_lp[TC ? kBatchTC : 1];   // TC: pivot values of the vectors since the pass
    if constexpr (SPEC) {
        k0 = ctrl->k0;
        extra = k - k0;
        Gs = Gp + (int64_t)ctrl->slot * n;
        const float2* Lf = reinterpret_cast<const float2*>(L);
        if constexpr (TC) {
            for (int i = threadIdx.x; i < extra; i += blockDim.x) s_lp[i] = Lf[(int64_t)(k0 + i) * n + P];
            __syncthreads();
        } else {
#pragma unroll
            for (int i = 0; i < kSpec - 1; ++i)
                lpP[i] = i < extra ? Lf[(int64_t)(k0 + i) * n + P] : make_float2(0.f, 0.f);
        }
    }
    long long mx_i = LLONG_MAX;   // SPEC: lowest index holding the block's candidate maximum
    // TC: the integral column is formed here, element by element, from the
    // pivot's pair data
    PivotF2 pv;
    if constexpr (TC) pv = pivot_f2(pf, P);
    // TC: the pass's projection plus the vectors made since, for this thread's
    // pairs, with four rows of L in flight per pair (the rows are a batch's
    // worth of recent vectors, up to 63 of them)
    float2 accTC[kStepPer];
    if constexpr (TC) {
        const float2* Lf = reinterpret_cast<const float2*>(L);
#pragma unroll
        for (int r = 0; r < kStepPer; ++r) {
            const int64_t I = base + r * kUpdThreads + threadIdx.x;
            accTC[r] = (k0 > 0 && I < n) ? Gs[I] : make_float2(0.f, 0.f);   // nothing precedes step 0
        }
        constexpr int kDepth = 4;
        for (int i0 = 0; i0 < extra; i0 += kDepth) {
            float2 v[kStepPer][kDepth];
#pragma unroll
            for (int r = 0; r < kStepPer; ++r) {
                const int64_t I = base + r * kUpdThreads + threadIdx.x;
#pragma unroll
                for (int j = 0; j < kDepth; ++j)
                    v[r][j] = (I < n && i0 + j < extra) ? Lf[(int64_t)(k0 + i0 + j) * n + I]
                                                        : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < kDepth; ++j)
                if (i0 + j < extra) {
                    const float2 lp = s_lp[i0 + j];
#pragma unroll
                    for (int r = 0; r < kStepPer; ++r) df_fma(accTC[r], v[r][j], lp);
                }
        }
    }
#pragma unroll
    for (int r = 0; r < kStepPer; ++r) {
        const int64_t I = base + r * kUpdThreads + threadIdx.x;
        if (I < n) {
            double* slot = L + (int64_t)k * n + I;
            double d;
            if constexpr (SPEC) {
                // everything but the residual in float pairs (column, projection, L^k)
                const float2* Lf = reinterpret_cast<const float2*>(L);
                float2 acc;
                if constexpr (TC) {
                    acc = accTC[r];
                } else {
                    acc = Gs[I];
#pragma unroll
                    for (int i = 0; i < kSpec - 1; ++i)
                        if (i < extra) df_fma(acc, Lf[(int64_t)(k0 + i) * n + I], lpP[i]);
                }
                float2 e;
                if constexpr (TC) e = eri_elem_df(pf, I, pv);
                else e = reinterpret_cast<const float2*>(ecol)[I];
                const float2 lf = df_mul(df_add(e, df_neg(acc)), rDPf);
                *reinterpret_cast<float2*>(slot) = lf;
                const float2 l2 = df_mul(lf, lf);
                d = D[I] - ((double)l2.x + (double)l2.y);
            } else {
                double proj = 0.0;
                if (k > 0) {
                    if constexpr (DF) {
                        const float2 f = *reinterpret_cast<const float2*>(slot);
                        proj = (double)f.x + (double)f.y;
                    } else {
                        proj = *slot;
                    }
                }
                const double l = (ecol[I] - proj) * rDP;
                if constexpr (DF) {
                    const float h = (float)l;
                    *reinterpret_cast<float2*>(slot) = make_float2(h, (float)(l - (double)h));
                } else {
                    *slot = l;
                }
                d = D[I] - l * l;
            }
            if (I == P) d = 0.0;
            D[I] = d;
            const long long bits = __double_as_longlong(d);
            if (cand[I]) {
                const long long key = bits > 0 ? bits : 0LL;
                if (key > mx) { mx = key; mx_i = I; }   // I increases with r: lowest index kept
            }
            mn = min(mn, key_of(d));
        }
    }
    long long mine = mx;
    block_maxmin_ll(mx, mn);
    if constexpr (SPEC) mx_i = block_min_ll(mine == mx && mx >= 0 ? mx_i : LLONG_MAX);
    if (threadIdx.x == 0) {
        blk_a[bid] = mx;
        blk_b[bid] = mn;
        if constexpr (SPEC) blk_i[bid] = mx >= 0 ? mx_i : -1;
    }
    if (!last_block(&ctrl->counter, nblk)) return;

    __shared__ double s_dp;   // the residual of the next pivot
    long long A = -1, B = LLONG_MAX;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        A = max(A, __ldcg(blk_a + i));
        B = min(B, __ldcg(blk_b + i));
    }
    block_maxmin_ll(A, B);
    const double G = A < 0 ? -INFINITY : __longlong_as_double(A);
    const double Dmin = value_of(B);
    const double scale = ctrl->scale, de = ctrl->delta_eff;
    const int32_t made = k + 1;
    int32_t status = CDS_OK;
    bool stop = true;
    long long pick = -1;
    if (Dmin < -kNotPdRel * scale || !(G == G)) {
        status = CDS_ERR_NOT_PD;
    } else if (G <= de) {
        status = CDS_OK;
    } else if (made >= max_rank) {
        status = CDS_ERR_RANK_CAP;
    } else {
        const double thr = G - kTieRel * scale;
        int from = 0;
        for (;;) {
            long long bl = LLONG_MAX;
            for (int i = from + threadIdx.x; i < nblk; i += blockDim.x) {
                const double m = __longlong_as_double(__ldcg(blk_a + i));   // -1: NaN, fails
                if (m >= thr && m > de) { bl = i; break; }
            }
            bl = block_min_ll(bl);
            if (bl == LLONG_MAX) break;
            long long best = LLONG_MAX;
            double dbest = 0.0;
#pragma unroll
            for (int r = 0; r < kStepPer; ++r) {
                const int64_t I = bl * kStepChunk + r * kUpdThreads + threadIdx.x;
                if (I < n) {
                    const double d = __ldcg(D + I);
                    if (cand[I] && fmax(d, 0.0) >= thr && d > de && I < best) {
                        best = (long long)I;
                        dbest = d;
                    }
                }
            }
            const long long mine_best = best;
            best = block_min_ll(best);
            if (best != LLONG_MAX) {
                if (mine_best == best) s_dp = dbest;   // the pivot's residual, for DP
                __syncthreads();
                pick = best;
                break;
            }
            from = (int)bl + 1;
        }
        if (pick >= 0) stop = false;
        else status = CDS_ERR_NOT_PD;   // G > delta_eff but no entry passes: D is inconsistent
    }
    // SPEC: does step k+1 continue the batch (its pivot is in the candidate
    // set and the batch is not full), or start a new one?  A new set holds the
    // pivot and the maxima of the blocks with the largest residuals.
    // TC: 32 candidates, a batch of up to 64 steps; the block maxima are held
    // in shared memory while the candidates are taken in order.
    constexpr int NS = TC ? kSpecTC : kSpec;
    constexpr int NB = TC ? kBatchTC : kSpec;
    __shared__ long long s_spec[NS];
    __shared__ int s_hit;
    if constexpr (SPEC) {
        if (!stop) {
            const long long* Sset = TC ? ctrl->STc : ctrl->S;
            if (threadIdx.x == 0) {
                s_hit = -1;
                if (made - ctrl->k0 < NB)
                    for (int c = 0; c < NS; ++c)
                        if (Sset[c] == pick) s_hit = c;
                s_spec[0] = pick;
            }
            __syncthreads();
            if (s_hit < 0 && TC) {
                // the blocks by (maximum descending, block index ascending), a
                // bitonic sort in shared memory; the first NS - 1 eligible ones
                // are the candidates after the pivot
                __shared__ long long s_key[TC ? kMaxBlocksTC : 1];
                __shared__ int32_t s_blk[TC ? kMaxBlocksTC : 1];
                const long long de_key = __double_as_longlong(de);
                int P = 1;
                while (P < nblk) P <<= 1;
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    long long key = LLONG_MIN;
                    if (i < nblk) {
                        const long long a = __ldcg(blk_a + i), idx = __ldcg(blk_i + i);
                        key = (idx >= 0 && idx != pick && a > de_key) ? a : -1;
                    }
                    s_key[i] = key;
                    s_blk[i] = i;
                }
                __syncthreads();
                for (int size = 2; size <= P; size <<= 1)
                    for (int stride = size >> 1; stride > 0; stride >>= 1) {
                        for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                            const int lo = 2 * stride * (t / stride) + t % stride, hi = lo + stride;
                            const long long ka = s_key[lo], kb = s_key[hi];
                            const int ia = s_blk[lo], ib = s_blk[hi];
                            const bool hi_first = kb > ka || (kb == ka && ib < ia);
                            if (hi_first == ((lo & size) == 0)) {   // out of order for this run
                                s_key[lo] = kb; s_key[hi] = ka;
                                s_blk[lo] = ib; s_blk[hi] = ia;
                            }
                        }
                        __syncthreads();
                    }
                if (threadIdx.x > 0 && threadIdx.x < NS)
                    s_spec[threadIdx.x] = (threadIdx.x - 1 < P && s_key[threadIdx.x - 1] >= 0)
                                              ? __ldcg(blk_i + s_blk[threadIdx.x - 1])
                                              : -1;
                __syncthreads();
            } else if (s_hit < 0) {
                const long long de_key = __double_as_longlong(de);
                for (int c = 1; c < kSpec; ++c) {
                    long long best = -1, dummy = LLONG_MAX;
                    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
                        const long long key = __ldcg(blk_a + i), idx = __ldcg(blk_i + i);
                        bool taken = idx == pick;
                        for (int e = 1; e < c; ++e) taken = taken || idx == s_spec[e];
                        if (!taken && idx >= 0 && key > de_key && key > best) best = key;
                    }
                    block_maxmin_ll(best, dummy);
                    long long first = LLONG_MAX;
                    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
                        const long long key = __ldcg(blk_a + i), idx = __ldcg(blk_i + i);
                        bool taken = idx == pick;
                        for (int e = 1; e < c; ++e) taken = taken || idx == s_spec[e];
                        if (!taken && idx >= 0 && best >= 0 && key == best && i < first) first = i;
                    }
                    first = block_min_ll(first);
                    if (threadIdx.x == 0) s_spec[c] = first == LLONG_MAX ? -1 : __ldcg(blk_i + first);
                    __syncthreads();
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        ctrl->G = G;
        ctrl->Dmin = Dmin;
        if (stop) {
            ctrl->status = status;
            ctrl->done = 1;
            ctrl->M = made;
        } else {
            ctrl->P = pick;
            const double DP = s_dp, rDP = 1.0 / sqrt(DP);
            ctrl->DP = DP;
            ctrl->rDP = rDP;
            {
                const float h = (float)rDP;
                ctrl->rDPf = make_float2(h, (float)(rDP - (double)h));
            }
            piv[made] = (int32_t)pick;
            if constexpr (SPEC) {
                if (s_hit >= 0) {
                    ctrl->slot = s_hit;
                    ctrl->pass = 0;
                    ctrl->extra += made - ctrl->k0;
                } else {
                    if constexpr (TC) {
                        // the store holds the rows before the last pass's step
                        ctrl->kdone = ctrl->k0;
                        for (int c = 0; c < kSpecTC; ++c) ctrl->STc[c] = s_spec[c];
                    } else {
                        for (int c = 0; c < kSpec; ++c) ctrl->S[c] = s_spec[c];
                    }
                    ctrl->k0 = made;
                    ctrl->slot = 0;
                    ctrl->pass = 1;
                    ctrl->passes += 1;
                    ctrl->streamed += made;
                }
            }
        }
        if constexpr (TC) ctrl->kstep = made;   // every block of this step has read it
        ctrl->counter = 0;
    }
}

// Step k, part 1: blocks [0, neri) make the integral column, the rest the
// projections, one tile each.  The two have no dependence on each other; the
// integral blocks come first in the grid, so their FP64 work overlaps the
// streaming of L by the projection blocks.
template <bool DF>
__global__ void __launch_bounds__(kUpdThreads, 4)
k_cd_project(PairSoA pd, int64_t n, int32_t k, double* __restrict__ L,
             double* __restrict__ ecol, int neri, const CdCtrl* ctrl) {
    if (ctrl->done) return;
    if ((int)blockIdx.x < neri) cd_eri_body(pd, n, ctrl, ecol, blockIdx.x, neri);
    else if (k > 0) cd_dot_body<DF>(n, k, L, ctrl, blockIdx.x - neri);
}

// Step k, part 1 of the speculative float-pair form, on a resident grid:
// every block takes its share of the integral column, then, when step k
// starts a batch, projection tiles in turn.
__global__ void __launch_bounds__(kUpdThreads, 4)
k_cd_project_spec(PairSoA pd, PairF2 pf, int64_t n, int32_t k, const double* __restrict__ L,
                  float2* __restrict__ G, float2* __restrict__ ecol, int ntiles,
                  const CdCtrl* ctrl) {
    if (ctrl->done) return;
    cd_eri_body_df(pd, pf, n, ctrl, ecol, blockIdx.x, gridDim.x);
    if (ctrl->pass == 0) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) cd_spec_dot_body(n, k, L, G, ctrl, t);
}

// Item `it` of the slicing that precedes a pass at step k.  Items
// [0, itemsA) bring the slice store up to date: the 8-column segments
// [s0, s0 + nseg) of every pair, the segment fastest (rows below k sliced,
// the rest zero); the rest slice the candidates' rows [0, k) into the B
// planes.
__device__ __forceinline__ void tc_slice_item(int64_t it, int64_t itemsA, int64_t n,
                                              const float2* __restrict__ Lf,
                                              const float* __restrict__ sigA,
                                              __nv_bfloat16* __restrict__ A,
                                              __nv_bfloat16* __restrict__ B,
                                              float* __restrict__ sigB, const CdCtrl* ctrl,
                                              int32_t k, int32_t s0, int32_t nseg) {
    if (it < itemsA) {
        const int64_t I = it / nseg;
        const int32_t K0 = (s0 + (int32_t)(it - I * nseg)) * 8;
        if (K0 >= k) {   // zero columns above the last vector
            const int64_t plane = n * kGroupTC;
            const int64_t off = ((int64_t)(K0 / kGroupTC) * kSlicesTC * n + I) * kGroupTC +
                                K0 % kGroupTC;
#pragma unroll
            for (int q = 0; q < kSlicesTC; ++q)
                *reinterpret_cast<uint4*>(A + q * plane + off) = make_uint4(0, 0, 0, 0);
            return;
        }
        int e = 0;
        frexpf(sigA[I], &e);   // sigma = 2^(e-1)
        tc_store8(Lf, n, I, K0, k, e - 1, A, n, I);
    } else {
        const int64_t r = it - itemsA;
        const int c = (int)(r % kSpecTC);
        const int32_t K0 = (int32_t)(r / kSpecTC) * 8;
        const long long Sc = ctrl->STc[c];
        const float sg = Sc >= 0 ? sigA[Sc] : 1.f;
        int e = 0;
        frexpf(sg, &e);
        tc_store8(Lf, n, Sc >= 0 ? Sc : -1, K0, k, e - 1, B, kSpecTC, c);
        if (K0 == 0) sigB[c] = sg;
    }
}

// The slicing of step k (no items unless the step starts a pass after the
// first step).  Segments below the previous pass's step kd hold final rows;
// those from its segment on are sliced again up to k, and the segments
// above k up to the group boundary must read zero: the previous pass zeroed
// its own group's, so only a new group's are written.
__device__ __forceinline__ void tc_slice_counts(const CdCtrl* ctrl, int64_t n, int32_t& k,
                                                int32_t& s0, int32_t& nseg, int64_t& itemsA,
                                                int64_t& itemsB) {
    itemsA = itemsB = 0;
    k = s0 = nseg = 0;
    if (ctrl->done || ctrl->pass == 0) return;
    k = ctrl->kstep;   // the step number lives on the device (graph replays)
    if (k == 0) return;
    const int32_t kd = ctrl->kdone;
    const int32_t kend = (k + kGroupTC - 1) / kGroupTC * kGroupTC;
    const int32_t kend_prev = (kd + kGroupTC - 1) / kGroupTC * kGroupTC;
    const int32_t s1 = (kend > kend_prev ? kend : (k + 7) / 8 * 8) / 8;
    s0 = kd / 8;
    nseg = s1 - s0;
    itemsA = (int64_t)nseg * n;
    itemsB = (int64_t)kSpecTC * (kend / 8);
}

// Step k, part 1 of the exact-slice tensor-core form (the integral column is
// formed in the update): when step k starts a pass, the blocks bring the
// slice store up to date (the rows made since the previous pass, zero above
// k to the group boundary) and slice the candidates' rows [0, k) into the B
// planes, for the projection GEMM that follows; otherwise the kernel returns
// at once.
__global__ void __launch_bounds__(kUpdThreads, 4)
k_cd_project_tc(int64_t n, const double* __restrict__ L, const float* __restrict__ sigA,
                __nv_bfloat16* __restrict__ A, __nv_bfloat16* __restrict__ B,
                float* __restrict__ sigB, const CdCtrl* ctrl) {
    pdl_trigger();
    pdl_wait();
    int32_t k, s0, nseg;
    int64_t itemsA, itemsB;
    tc_slice_counts(ctrl, n, k, s0, nseg, itemsA, itemsB);
    const float2* Lf = reinterpret_cast<const float2*>(L);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < itemsA + itemsB;
         it += stride)
        tc_slice_item(it, itemsA, n, Lf, sigA, A, B, sigB, ctrl, k, s0, nseg);
}

// Step k, part 2: vector k, residuals, next pivot.  Five blocks per SM keep
// the C60-shaped grid (690 blocks of 512 pairs) in one wave; the tensor-core
// form runs on the screened pairs (425 blocks at C60), where four blocks per
// SM do, and takes the registers (64) that its column and projection need.
template <bool DF, bool SPEC, bool TC = false>
__global__ void __launch_bounds__(kUpdThreads, TC ? 4 : 5)
k_cd_update(int64_t n, int32_t k, int32_t max_rank, double* __restrict__ L,
            double* __restrict__ D, const uint8_t* __restrict__ cand,
            const double* __restrict__ ecol, const float2* __restrict__ G,
            double* __restrict__ blk_a, double* __restrict__ blk_b,
            long long* __restrict__ blk_i, int32_t* __restrict__ piv, CdCtrl* ctrl,
            PairF2 pf = PairF2{}) {
    if constexpr (TC) {
        pdl_trigger();
        pdl_wait();
    }
    if (ctrl->done) return;
    if constexpr (TC) k = ctrl->kstep;   // the step number lives on the device (graph replays)
    cd_step_body<DF, SPEC, TC>(n, k, max_rank, L, D, cand, ecol, G,
                           reinterpret_cast<long long*>(blk_a),
                           reinterpret_cast<long long*>(blk_b), blk_i, piv, ctrl, blockIdx.x,
                           gridDim.x, pf);
}

// ---- screening of the tensor-core form (kScreenRel) ----
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;   // inclusive over warps
    }
    __syncthreads();
    const int before = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before;
}

// Live pairs per compaction block.
__global__ void __launch_bounds__(kScanThreads)
k_screen_count(const double* __restrict__ D, int64_t n, const CdCtrl* ctrl, int32_t* cnt) {
    const double thr = kScreenRel * ctrl->scale;
    const int64_t I0 = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int v = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) v += (I0 + i < n && D[I0 + i] >= thr) ? 1 : 0;
    int total = 0;
    block_excl_scan(v, &total);
    if (threadIdx.x == 0) cnt[blockIdx.x] = total;
}

// Exclusive prefix over the block counts (one block), the total into ctrl.
__global__ void __launch_bounds__(1024) k_screen_scan(int32_t* cnt, int nb, CdCtrl* ctrl) {
    int run = 0;
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const int v = b < nb ? cnt[b] : 0;
        int total = 0;
        const int before = block_excl_scan(v, &total);
        if (b < nb) cnt[b] = run + before;
        run += total;
    }
    if (threadIdx.x == 0) ctrl->nlive = run;
}

// The live pairs in packed order: live[j] = I, and their data gathered (pair
// data as float pairs, candidate flag, initial diagonal).
__global__ void __launch_bounds__(kScanThreads)
k_screen_gather(PairSoA pd, const double* __restrict__ D, const uint8_t* __restrict__ cand,
                int64_t n, const CdCtrl* ctrl, const int32_t* __restrict__ cnt,
                int32_t* __restrict__ live, PairF2 pf, double* __restrict__ Dc,
                uint8_t* __restrict__ candc) {
    const double thr = kScreenRel * ctrl->scale;
    const int64_t I0 = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    bool f[kScanPer];
    int v = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        f[i] = I0 + i < n && D[I0 + i] >= thr;
        v += f[i] ? 1 : 0;
    }
    int total = 0;
    int pos = cnt[blockIdx.x] + block_excl_scan(v, &total);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (!f[i]) continue;
        const int64_t I = I0 + i;
        live[pos] = (int32_t)I;
        Dc[pos] = D[I];
        candc[pos] = cand[I];
        pf.p[pos] = to_f2(pd.p[I]);
        pf.Px[pos] = to_f2(pd.Px[I]);
        pf.Py[pos] = to_f2(pd.Py[I]);
        pf.Pz[pos] = to_f2(pd.Pz[I]);
        pf.Kp[pos] = to_f2(pd.Kp[I]);
        ++pos;
    }
}

// Rows [r0, r0 + nrows) of the compact vectors into the full rows of L (whose
// screened entries were zeroed), as float pairs.
__global__ void k_screen_scatter(const double* __restrict__ Lc, int64_t nc,
                                 const int32_t* __restrict__ live, double* __restrict__ L,
                                 int64_t n, int32_t r0, int32_t nrows) {
    const int64_t total = (int64_t)nrows * nc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = r0 + i / nc, j = i % nc;
        L[r * n + live[j]] = Lc[r * nc + j];
    }
}

// Pivots back to packed indices; the live pairs' residuals into D (the
// screened ones keep D0).
__global__ void k_screen_finish(const int32_t* __restrict__ pivc, int32_t M,
                                const int32_t* __restrict__ live, int32_t* __restrict__ piv,
                                const double* __restrict__ Dc, int64_t nc, double* __restrict__ D) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < M) piv[i] = live[pivc[i]];
    if (i < nc) D[live[i]] = Dc[i];
}

// Float pairs (hi, lo) of the first count elements of L back to FP64, in place.
__global__ void k_pairs_to_fp64(double* __restrict__ L, int64_t count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float2 v = reinterpret_cast<const float2*>(L)[i];
    L[i] = (double)v.x + (double)v.y;
}

int pairs_to_fp64(double* L, int64_t count, cudaStream_t stream) {
    if (count <= 0) return CDS_OK;
    k_pairs_to_fp64<<<(unsigned)((count + 255) / 256), 256, 0, stream>>>(L, count);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

struct CdLayout {
    PairSoA pd;
    uint8_t* cand;
    double* ecol;     // integral column of the current step
    float2* G;        // [kSpec][npair] candidate projections (float-pair mode; [kSpecTC] in TC)
    // exact-slice tensor-core form
    __nv_bfloat16* A; // slice store [kcap / kGroupTC][kSlicesTC][npair][kGroupTC]
    __nv_bfloat16* B; // candidate rows [kcap / kGroupTC][kSlicesTC][kSpecTC][kGroupTC]
    float* sigA;      // [npair] pair scales
    float* sigB;      // [kSpecTC] candidate scales
    int32_t* err;     // the GEMM's bounded-wait error word
    int32_t kcap;
    // screening (tensor-core form): the live pairs and the compact problem
    int32_t* live;    // [npair] packed index of live pair j
    int32_t* scan;    // [npair / kScanChunk + 1] block counts / offsets
    double* Dc;       // [npair] compact residual diagonal
    uint8_t* candc;   // [npair] compact candidate flags
    int32_t* pivc;    // [max_rank] compact pivots
    double* Lc;       // [max_rank][npair] compact vectors (float pairs)
    PairF2 pf;        // pair data as float pairs (float-pair mode)
    double* blk_a;
    double* blk_b;
    long long* blk_i;
    CdCtrl* ctrl;
    size_t bytes;
};

static int cd_blocks(int64_t n) { return (int)((n + kCdThreads - 1) / kCdThreads); }
static int dot_tiles(int64_t n) { return (int)((n + kUpdPairs - 1) / kUpdPairs); }
// integral-column blocks of k_cd_project: two per SM at most (grid-stride)
static int eri_blocks(int64_t n, int nsm) {
    return (int)std::min<int64_t>(2 * nsm, (n + kUpdThreads - 1) / kUpdThreads);
}
static int step_blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + kStepChunk - 1) / kStepChunk); }
// block partials are shared by the init, update and select grids (each at
// most cd_blocks blocks)
static int part_blocks(int64_t n) { return std::max(cd_blocks(n), 1); }
static int sm_count() {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return 152;
    return nsm;
}
static int sel_blocks(int64_t n) { return (int)std::min<int64_t>(4 * 152, (n + kCdThreads - 1) / kCdThreads); }

// Column capacity of the slice store for max_rank vectors.
static int32_t tc_kcap(int32_t max_rank) {
    return std::max(1, (max_rank + kGroupTC - 1) / kGroupTC) * kGroupTC;
}

// spec: room for the candidate projections of the float-pair mode; tc (with
// max_rank): also the tensor-core form's slice store and candidate rows
static CdLayout cd_layout(void* ws, int32_t nbf, bool spec = true, bool tc = false,
                          int32_t max_rank = 0) {
    int64_t n = npair_of(nbf);
    int nb = part_blocks(n);
    spec = spec || tc;
    Carver c(ws);
    CdLayout l;
    l.kcap = tc ? tc_kcap(max_rank) : 0;
    l.ctrl = c.take<CdCtrl>(1);   // first: at the same offset in every form (cds_cd_stats)
    l.pd.p = c.take<double>(n);
    l.pd.Px = c.take<double>(n);
    l.pd.Py = c.take<double>(n);
    l.pd.Pz = c.take<double>(n);
    l.pd.Kp = c.take<double>(n);
    l.cand = c.take<uint8_t>(n);
    l.ecol = c.take<double>(n);
    l.G = spec ? c.take<float2>((size_t)(tc ? kSpecTC : kSpec) * n) : nullptr;
    l.A = tc ? c.take<__nv_bfloat16>((size_t)kSlicesTC * n * l.kcap) : nullptr;
    l.B = tc ? c.take<__nv_bfloat16>((size_t)kSlicesTC * kSpecTC * l.kcap) : nullptr;
    l.sigA = tc ? c.take<float>(n) : nullptr;
    l.sigB = tc ? c.take<float>(kSpecTC) : nullptr;
    l.err = tc ? c.take<int32_t>(4) : nullptr;
    l.live = tc ? c.take<int32_t>(n) : nullptr;
    l.scan = tc ? c.take<int32_t>(n / kScanChunk + 2) : nullptr;
    l.Dc = tc ? c.take<double>(n) : nullptr;
    l.candc = tc ? c.take<uint8_t>(n) : nullptr;
    l.pivc = tc ? c.take<int32_t>(std::max(max_rank, 1)) : nullptr;
    l.Lc = tc ? c.take<double>((size_t)std::max(max_rank, 1) * n) : nullptr;
    l.pf.p = spec ? c.take<float2>(n) : nullptr;
    l.pf.Px = spec ? c.take<float2>(n) : nullptr;
    l.pf.Py = spec ? c.take<float2>(n) : nullptr;
    l.pf.Pz = spec ? c.take<float2>(n) : nullptr;
    l.pf.Kp = spec ? c.take<float2>(n) : nullptr;
    l.blk_a = c.take<double>(nb);
    l.blk_b = c.take<double>(nb);
    l.blk_i = c.take<long long>(nb);
    l.bytes = c.off;
    return l;
}

size_t cd_workspace_bytes_for(int32_t nbf, bool f32x2) {
    if (nbf < 0) return 0;
    return cd_layout(nullptr, nbf, f32x2).bytes;
}

size_t cd_workspace_bytes_prec(int32_t nbf, int32_t max_rank, int32_t precision) {
    if (nbf < 0 || max_rank < 0) return 0;
    if (precision == CDS_PREC_OZAKI) return cd_layout(nullptr, nbf, true, true, max_rank).bytes;
    if (precision == CDS_PREC_F32X2) return cd_layout(nullptr, nbf, true).bytes;
    if (precision == CDS_PREC_FP64) return cd_layout(nullptr, nbf, false).bytes;
    return 0;
}

}  // namespace cds

using namespace cds;

// Enough for either precision.
extern "C" size_t cds_cd_workspace_bytes(int32_t nbf) { return cd_workspace_bytes_for(nbf, true); }

extern "C" int cds_cd_candidates(int32_t precision) {
    return precision == CDS_PREC_OZAKI ? kSpecTC : precision == CDS_PREC_F32X2 ? kSpec : 1;
}

extern "C" size_t cds_cd_workspace_bytes_prec(int32_t nbf, int32_t max_rank, int32_t precision) {
    return cd_workspace_bytes_prec(nbf, max_rank, precision);
}

extern "C" int cds_cd_stats(int32_t nbf, const void* workspace, int32_t precision,
                            int32_t* passes, int64_t* streamed, int64_t* extra,
                            cudaStream_t stream) {
    if (nbf <= 0 || !workspace || !passes || !streamed || !extra) return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && precision != CDS_PREC_F32X2 && precision != CDS_PREC_OZAKI)
        return CDS_ERR_UNSUPPORTED;
    CdLayout lay = cd_layout(const_cast<void*>(workspace), nbf, precision != CDS_PREC_FP64);
    CdCtrl h{};
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, lay.ctrl, sizeof(CdCtrl), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    if (precision != CDS_PREC_FP64) {
        *passes = h.passes;
        *streamed = h.streamed;
        *extra = h.extra;
    } else {   // the FP64 form streams L at every step
        *passes = h.M;
        *streamed = (int64_t)h.M * (h.M - 1) / 2;
        *extra = 0;
    }
    return CDS_OK;
}

extern "C" int cds_cd_live_pairs(int32_t nbf, const void* workspace, int32_t precision,
                                 int64_t* nlive, cudaStream_t stream) {
    if (nbf <= 0 || !workspace || !nlive) return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && precision != CDS_PREC_F32X2 && precision != CDS_PREC_OZAKI)
        return CDS_ERR_UNSUPPORTED;
    if (precision != CDS_PREC_OZAKI) {   // the other forms do not screen
        *nlive = npair_of(nbf);
        return CDS_OK;
    }
    CdLayout lay = cd_layout(const_cast<void*>(workspace), nbf, true);
    CdCtrl h{};
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, lay.ctrl, sizeof(CdCtrl), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    *nlive = h.nlive;
    return CDS_OK;
}

namespace cds {

// Timing of the tensor-core projection GEMM (cds_cd_gemm_timing): process-wide
// totals over the launches made while it is on.
struct GemmTiming {
    bool on = false;
    double ms = 0.0;
    long long launches = 0;
};
static GemmTiming g_gemm_timing;

// The tensor-core form after the initial diagonal: screening, then the steps
// on the compact problem of the live pairs (vectors in lay.Lc, scattered into
// L's full rows after each host check, so the hook sees float-pair rows as
// in the float-pair form).
static int cd_run_tc(int64_t n, int32_t max_rank, double* L, int32_t* piv, double* D,
                     int32_t* M_out, double* delta_eff_out, const CdLayout& lay,
                     cudaStream_t stream, const CdChunkHook* on_chunk,
                     cudaStream_t convert_after, bool chunk_graph, bool convert) {
    const int nsb = (int)((n + kScanChunk - 1) / kScanChunk);
    k_screen_count<<<nsb, kScanThreads, 0, stream>>>(D, n, lay.ctrl, lay.scan);
    CDS_LAUNCH_CHECK();
    k_screen_scan<<<1, 1024, 0, stream>>>(lay.scan, nsb, lay.ctrl);
    CDS_LAUNCH_CHECK();
    k_screen_gather<<<nsb, kScanThreads, 0, stream>>>(lay.pd, D, lay.cand, n, lay.ctrl, lay.scan,
                                                      lay.live, lay.pf, lay.Dc, lay.candc);
    CDS_LAUNCH_CHECK();
    int32_t nlive = 0;
    CDS_CUDA_TRY(cudaMemcpyAsync(&nlive, &lay.ctrl->nlive, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    if (nlive <= 0) return CDS_ERR_NOT_PD;   // no diagonal passed the test: NaN or a zero scale
    const int64_t nc = nlive;
    if (step_blocks(nc) > kMaxBlocksTC) return CDS_ERR_UNSUPPORTED;
    const int nsm = sm_count();
    const int ns = sel_blocks(nc), nu = step_blocks(nc);
    const int nres = (int)std::min<int64_t>(4 * nsm, dot_tiles(nc));   // resident grid
    k_cd_select<<<ns, kCdThreads, 0, stream>>>(nc, 0, max_rank, lay.Dc, lay.candc, lay.blk_i,
                                              lay.pivc, lay.ctrl);
    CDS_LAUNCH_CHECK();
    // pair scales from the initial diagonal, the GEMM's tensor maps (fixed for
    // the whole decomposition) and error word
    k_cd_tc_scales<<<(unsigned)((nc + 255) / 256), 256, 0, stream>>>(lay.Dc, nc, lay.sigA);
    CDS_LAUNCH_CHECK();
    CDS_CUDA_TRY(cudaMemsetAsync(lay.err, 0, sizeof(int32_t), stream));
    CdTcGemm* gemm = nullptr;
    struct GemmGuard {
        CdTcGemm*& g;
        ~GemmGuard() { if (g) cd_tc_gemm_free(g); }
    } guard{gemm};
    int st = cd_tc_gemm_setup(&gemm, nc, lay.kcap, lay.A, lay.B, lay.sigA, lay.sigB, lay.G,
                              lay.ctrl, lay.err);
    if (st) return st;
    // CUDA events around every GEMM launch of the steps that run (one pair per
    // step of a host-check chunk, reused), summed after each check
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CDS_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
    const bool timing = g_gemm_timing.on && cap == cudaStreamCaptureStatusNone;
    std::vector<cudaEvent_t> tev;
    struct EventGuard {
        std::vector<cudaEvent_t>& v;
        ~EventGuard() { for (cudaEvent_t e : v) cudaEventDestroy(e); }
    } tev_guard{tev};
    if (timing)
        for (int i = 0; i < 2 * kHostCheckEvery; ++i) {
            cudaEvent_t e;
            CDS_CUDA_TRY(cudaEventCreate(&e));
            tev.push_back(e);
        }
    // the kernels of steps [k0, k1) (each reads its step number from ctrl)
    auto enqueue = [&](int32_t k0, int32_t k1) -> int {
        for (int32_t k = k0; k < k1; ++k) {
            CDS_CUDA_TRY(launch_pdl(k_cd_project_tc, (unsigned)nres, kUpdThreads, 0, stream, nc,
                                    (const double*)lay.Lc, (const float*)lay.sigA, lay.A, lay.B,
                                    lay.sigB, (const CdCtrl*)lay.ctrl));
            if (timing) CDS_CUDA_TRY(cudaEventRecord(tev[2 * (k - k0)], stream));
            const int s2 = cd_tc_gemm_launch(gemm, stream);
            if (s2) return s2;
            if (timing) CDS_CUDA_TRY(cudaEventRecord(tev[2 * (k - k0) + 1], stream));
            CDS_CUDA_TRY(launch_pdl(k_cd_update<true, true, true>, (unsigned)nu, kUpdThreads, 0,
                                    stream, nc, k, max_rank, lay.Lc, lay.Dc,
                                    (const uint8_t*)lay.candc, (const double*)lay.ecol,
                                    (const float2*)lay.G, lay.blk_a, lay.blk_b, lay.blk_i,
                                    lay.pivc, lay.ctrl, lay.pf));
        }
        return CDS_OK;
    };
    // a full chunk of steps as one CUDA graph, replayed at every host check
    // (one launch instead of 3 x kHostCheckEvery): not under capture or
    // timing, not on a default stream (no capture there), and only for
    // decompositions long enough to repay the instantiation
    cudaGraphExec_t chunk = nullptr;
    struct ExecGuard {
        cudaGraphExec_t& e;
        ~ExecGuard() { if (e) cudaGraphExecDestroy(e); }
    } chunk_guard{chunk};
    const int graph_min = tc::tune_cd_graph();
    const bool default_stream =
        stream == nullptr || stream == cudaStreamLegacy || stream == cudaStreamPerThread;
    if (chunk_graph && !timing && cap == cudaStreamCaptureStatusNone && !default_stream &&
        graph_min > 0 && max_rank >= std::max(graph_min, kHostCheckEvery)) {
        cudaGraph_t g = nullptr;
        CDS_CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        const int s2 = enqueue(0, kHostCheckEvery);
        const cudaError_t ce = cudaStreamEndCapture(stream, &g);
        if (s2) {
            if (g) cudaGraphDestroy(g);
            return s2;
        }
        CDS_CUDA_TRY(ce);
        const cudaError_t ie = cudaGraphInstantiate(&chunk, g, 0);
        cudaGraphDestroy(g);
        CDS_CUDA_TRY(ie);
    }
    CdCtrl h{};
    for (int32_t k0 = 0; k0 <= max_rank; k0 += kHostCheckEvery) {
        const int32_t k1 = std::min(max_rank, k0 + kHostCheckEvery);
        if (chunk && k1 - k0 == kHostCheckEvery) {
            CDS_CUDA_TRY(cudaGraphLaunch(chunk, stream));
        } else if ((st = enqueue(k0, k1))) {
            return st;
        }
        count_launches(3ull * (unsigned long long)(k1 - k0));
        if (k1 > k0) {   // this chunk's rows into L's full rows (screened entries 0)
            CDS_CUDA_TRY(cudaMemsetAsync(L + (int64_t)k0 * n, 0,
                                         (size_t)(k1 - k0) * n * sizeof(double), stream));
            const int64_t items = (int64_t)(k1 - k0) * nc;
            k_screen_scatter<<<(unsigned)std::min<int64_t>((items + 255) / 256, 8 * nsm), 256, 0,
                               stream>>>(lay.Lc, nc, lay.live, L, n, k0, k1 - k0);
            CDS_LAUNCH_CHECK();
        }
        CDS_CUDA_TRY(cudaGetLastError());
        CDS_CUDA_TRY(cudaMemcpyAsync(&h, lay.ctrl, sizeof(CdCtrl), cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
        if (timing) {   // the steps that ran (k < M once the decomposition has stopped)
            const int32_t kr = h.done ? std::min(k1, h.M) : k1;
            for (int32_t k = k0; k < kr; ++k) {
                float ms = 0.f;
                CDS_CUDA_TRY(cudaEventElapsedTime(&ms, tev[2 * (k - k0)], tev[2 * (k - k0) + 1]));
                g_gemm_timing.ms += ms;
                ++g_gemm_timing.launches;
            }
        }
        if (on_chunk && *on_chunk) {
            st = (*on_chunk)(h.done ? h.M : k1, h.done != 0);
            if (st) return st;
        }
        if (h.done) break;
    }
    *M_out = h.M;
    if (delta_eff_out) *delta_eff_out = h.delta_eff;
    const int64_t fin = std::max<int64_t>(h.M, nc);
    k_screen_finish<<<(unsigned)((fin + 255) / 256), 256, 0, stream>>>(lay.pivc, h.M, lay.live,
                                                                       piv, lay.Dc, nc, D);
    CDS_LAUNCH_CHECK();
    if (h.M > 0 && convert) {
        if (convert_after) {
            cudaEvent_t ev;
            CDS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            CDS_CUDA_TRY(cudaEventRecord(ev, convert_after));
            CDS_CUDA_TRY(cudaStreamWaitEvent(stream, ev, 0));
            CDS_CUDA_TRY(cudaEventDestroy(ev));
        }
        const int64_t cnt = (int64_t)h.M * n;
        k_pairs_to_fp64<<<(unsigned)((cnt + 255) / 256), 256, 0, stream>>>(L, cnt);
        CDS_LAUNCH_CHECK();
    }
    int32_t e = 0;   // a bounded wait of the projection GEMM gave up
    CDS_CUDA_TRY(cudaMemcpyAsync(&e, lay.err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    if (e) return CDS_ERR_TIMEOUT;
    if (!h.done) return CDS_ERR_RANK_CAP;
    return h.status;
}

// The decomposition of cds_cd_decompose.  on_chunk (may be null) runs after
// every host check with the number of rows of L that are final and whether
// the decomposition has stopped; before the float-pair rows are converted to
// FP64 at the end, stream waits for convert_after (may be null), so work that
// reads the float-pair rows can run on another stream meanwhile.  With
// convert false the float-pair rows are left to the caller (pairs_to_fp64).
int cd_decompose_run(int32_t nbf, const double* xyz, const double* alpha, const int32_t* atom,
                     double delta, int32_t scheme, int32_t max_rank, int32_t precision, double* L,
                     int32_t* piv, double* D, int32_t* M_out, double* delta_eff_out,
                     void* workspace, size_t workspace_bytes, cudaStream_t stream,
                     const CdChunkHook* on_chunk, cudaStream_t convert_after, bool chunk_graph,
                     bool convert) {
    if (nbf <= 0 || !xyz || !alpha || !L || !piv || !D || !M_out || max_rank < 0)
        return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && precision != CDS_PREC_F32X2 && precision != CDS_PREC_OZAKI)
        return CDS_ERR_UNSUPPORTED;
    const bool tcm = precision == CDS_PREC_OZAKI;
    const bool df = precision == CDS_PREC_F32X2;
    if (!(delta >= 0.0)) return CDS_ERR_ARG;
    if (scheme != CDS_SCHEME_FULL && scheme != CDS_SCHEME_ATOMIC) return CDS_ERR_ARG;
    if (scheme == CDS_SCHEME_ATOMIC && !atom) return CDS_ERR_ARG;
    int64_t n = npair_of(nbf);
    CdLayout lay = cd_layout(workspace, nbf, df || tcm, tcm, max_rank);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    int st = build_pairs(nbf, xyz, alpha, lay.pd, stream);
    if (st) return st;
    if (df) {
        k_pairs_to_f2<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(lay.pd, lay.pf, n);
        CDS_LAUNCH_CHECK();
    }
    CDS_CUDA_TRY(cudaMemsetAsync(lay.ctrl, 0, sizeof(CdCtrl), stream));
    const int nsm = sm_count();
    const int nb = cd_blocks(n), ns = sel_blocks(n);
    const int ne = eri_blocks(n, nsm), np_ = ne + dot_tiles(n), nu = step_blocks(n);
    const int nres = (int)std::min<int64_t>(4 * nsm, dot_tiles(n));   // resident grid
    k_cd_init<<<nb, kCdThreads, 0, stream>>>(lay.pd, atom, scheme, n, delta, D, lay.cand,
                                            lay.blk_a, lay.blk_b, lay.ctrl);
    CDS_LAUNCH_CHECK();
    if (tcm)
        return cd_run_tc(n, max_rank, L, piv, D, M_out, delta_eff_out, lay, stream, on_chunk,
                         convert_after, chunk_graph, convert);
    k_cd_select<<<ns, kCdThreads, 0, stream>>>(n, 0, max_rank, D, lay.cand, lay.blk_i, piv,
                                              lay.ctrl);
    CDS_LAUNCH_CHECK();
    CdCtrl h{};
    for (int32_t k0 = 0; k0 <= max_rank; k0 += kHostCheckEvery) {
        int32_t k1 = std::min(max_rank, k0 + kHostCheckEvery);
        for (int32_t k = k0; k < k1; ++k) {
            if (df) {
                k_cd_project_spec<<<nres, kUpdThreads, 0, stream>>>(
                    lay.pd, lay.pf, n, k, L, lay.G, reinterpret_cast<float2*>(lay.ecol),
                    dot_tiles(n), lay.ctrl);
                k_cd_update<true, true><<<nu, kUpdThreads, 0, stream>>>(
                    n, k, max_rank, L, D, lay.cand, lay.ecol, lay.G, lay.blk_a, lay.blk_b,
                    lay.blk_i, piv, lay.ctrl);
            } else {
                k_cd_project<false><<<np_, kUpdThreads, 0, stream>>>(lay.pd, n, k, L, lay.ecol, ne,
                                                                     lay.ctrl);
                k_cd_update<false, false><<<nu, kUpdThreads, 0, stream>>>(
                    n, k, max_rank, L, D, lay.cand, lay.ecol, nullptr, lay.blk_a, lay.blk_b,
                    lay.blk_i, piv, lay.ctrl);
            }
        }
        count_launches(2ull * (unsigned long long)(k1 - k0));
        CDS_CUDA_TRY(cudaGetLastError());
        CDS_CUDA_TRY(cudaMemcpyAsync(&h, lay.ctrl, sizeof(CdCtrl), cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
        if (on_chunk && *on_chunk) {
            st = (*on_chunk)(h.done ? h.M : k1, h.done != 0);
            if (st) return st;
        }
        if (h.done) break;
    }
    *M_out = h.M;
    if (delta_eff_out) *delta_eff_out = h.delta_eff;
    if (df && h.M > 0 && convert) {
        if (convert_after) {
            cudaEvent_t ev;
            CDS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            CDS_CUDA_TRY(cudaEventRecord(ev, convert_after));
            CDS_CUDA_TRY(cudaStreamWaitEvent(stream, ev, 0));
            CDS_CUDA_TRY(cudaEventDestroy(ev));
        }
        const int64_t cnt = (int64_t)h.M * n;
        k_pairs_to_fp64<<<(unsigned)((cnt + 255) / 256), 256, 0, stream>>>(L, cnt);
        CDS_LAUNCH_CHECK();
    }
    if (!h.done) return CDS_ERR_RANK_CAP;
    return h.status;
}

}  // namespace cds

extern "C" int cds_cd_decompose(int32_t nbf, const double* xyz, const double* alpha,
                                const int32_t* atom, double delta, int32_t scheme,
                                int32_t max_rank, int32_t precision, double* L, int32_t* piv,
                                double* D, int32_t* M_out, double* delta_eff_out,
                                void* workspace, size_t workspace_bytes, cudaStream_t stream) {
    return cds::cd_decompose_run(nbf, xyz, alpha, atom, delta, scheme, max_rank, precision, L,
                                 piv, D, M_out, delta_eff_out, workspace, workspace_bytes, stream,
                                 nullptr, nullptr);
}

extern "C" int cds_cd_gemm_timing(int32_t enable) {
    cds::g_gemm_timing.on = enable != 0;
    cds::g_gemm_timing.ms = 0.0;
    cds::g_gemm_timing.launches = 0;
    return CDS_OK;
}

extern "C" int cds_cd_gemm_time(double* ms, int64_t* launches) {
    if (!ms || !launches) return CDS_ERR_ARG;
    *ms = cds::g_gemm_timing.ms;
    *launches = cds::g_gemm_timing.launches;
    return CDS_OK;
}

namespace cds {
int shell_diag(int32_t nbf, const double* xyz, const int32_t* lmn, const int32_t* start,
               const double* exps, const double* coefs, double* D, cudaStream_t stream);
int shell_column(int32_t nbf, const double* xyz, const int32_t* lmn, const int32_t* start,
                 const double* exps, const double* coefs, const int64_t* P, const int32_t* done,
                 double* ecol, cudaStream_t stream);
}  // namespace cds

// The same decomposition over contracted Cartesian shells (FP64): the
// diagonal and the columns come from the contracted-shell integral kernels
// (shells.cu), the projections, updates and pivot rule are the s-type ones.
extern "C" int cds_cd_decompose_shells(int32_t nbf, const double* xyz, const int32_t* lmn,
                                       const int32_t* start, const double* exps,
                                       const double* coefs, const int32_t* atom, double delta,
                                       int32_t scheme, int32_t max_rank, double* L, int32_t* piv,
                                       double* D, int32_t* M_out, double* delta_eff_out,
                                       void* workspace, size_t workspace_bytes,
                                       cudaStream_t stream) {
    if (nbf <= 0 || !xyz || !lmn || !start || !exps || !coefs || !L || !piv || !D || !M_out ||
        max_rank < 0 || !(delta >= 0.0))
        return CDS_ERR_ARG;
    if (scheme != CDS_SCHEME_FULL && scheme != CDS_SCHEME_ATOMIC) return CDS_ERR_ARG;
    if (scheme == CDS_SCHEME_ATOMIC && !atom) return CDS_ERR_ARG;
    {   // every function s, p or d (l + m + n <= 2): the kernels' bound
        std::vector<int32_t> h(3 * (size_t)nbf);
        CDS_CUDA_TRY(cudaMemcpyAsync(h.data(), lmn, sizeof(int32_t) * 3 * nbf,
                                     cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
        for (int32_t f = 0; f < nbf; ++f) {
            const int32_t l = h[3 * f], m = h[3 * f + 1], k = h[3 * f + 2];
            if (l < 0 || m < 0 || k < 0 || l + m + k > 2) return CDS_ERR_UNSUPPORTED;
        }
    }
    const int64_t n = npair_of(nbf);
    CdLayout lay = cd_layout(workspace, nbf, false);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    int st = shell_diag(nbf, xyz, lmn, start, exps, coefs, D, stream);
    if (st) return st;
    CDS_CUDA_TRY(cudaMemsetAsync(lay.ctrl, 0, sizeof(CdCtrl), stream));
    const int nb = cd_blocks(n), ns = sel_blocks(n), nu = step_blocks(n);
    k_cd_init<<<nb, kCdThreads, 0, stream>>>(lay.pd, atom, scheme, n, delta, D, lay.cand,
                                            lay.blk_a, lay.blk_b, lay.ctrl, 1);
    CDS_LAUNCH_CHECK();
    k_cd_select<<<ns, kCdThreads, 0, stream>>>(n, 0, max_rank, D, lay.cand, lay.blk_i, piv,
                                              lay.ctrl);
    CDS_LAUNCH_CHECK();
    CdCtrl h{};
    for (int32_t k0 = 0; k0 <= max_rank; k0 += kHostCheckEvery) {
        const int32_t k1 = std::min(max_rank, k0 + kHostCheckEvery);
        for (int32_t k = k0; k < k1; ++k) {
            st = shell_column(nbf, xyz, lmn, start, exps, coefs, &lay.ctrl->P, &lay.ctrl->done,
                              lay.ecol, stream);
            if (st) return st;
            k_cd_project<false><<<dot_tiles(n), kUpdThreads, 0, stream>>>(lay.pd, n, k, L, lay.ecol,
                                                                           0, lay.ctrl);
            k_cd_update<false, false><<<nu, kUpdThreads, 0, stream>>>(
                n, k, max_rank, L, D, lay.cand, lay.ecol, nullptr, lay.blk_a, lay.blk_b,
                lay.blk_i, piv, lay.ctrl);
        }
        count_launches(3ull * (unsigned long long)(k1 - k0));
        CDS_CUDA_TRY(cudaGetLastError());
        CDS_CUDA_TRY(cudaMemcpyAsync(&h, lay.ctrl, sizeof(CdCtrl), cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
        if (h.done) break;
    }
    *M_out = h.M;
    if (delta_eff_out) *delta_eff_out = h.delta_eff;
    if (!h.done) return CDS_ERR_RANK_CAP;
    return h.status;
}


// ===========================================================================
// Batched decomposition: the steps of many molecules advance together, one
// update and one select launch per step for the whole batch; each block
// finds its molecule from the per-molecule block ranges.
// ===========================================================================
namespace cds {

struct CdMol {
    PairSoA pd;
    PairF2 pf;        // float-pair mode: pair data as float pairs
    float2* G;        // float-pair mode: [kSpec][n] candidate projections
    const int32_t* atom;
    double* L;
    double* D;
    uint8_t* cand;
    double* ecol;
    int32_t* piv;
    double* blk_a;
    double* blk_b;
    long long* blk_i;
    CdCtrl* ctrl;
    int64_t n;
    int32_t max_rank;
    int32_t b0_init, nb_init, b0_sel, nb_sel, b0_epi, nb_epi;
    int32_t b0_prj, nb_eri, nb_dot;   // project grid: nb_eri integral blocks, then nb_dot tiles
};

// Molecule owning block bid of a batch grid (kind: 0 init, 1 project,
// 2 select, 3 update).
__device__ __forceinline__ int find_mol(const CdMol* mols, int nmol, int bid, int kind) {
    int lo = 0, hi = nmol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int b0 = kind == 0 ? mols[mid].b0_init
                     : kind == 1 ? mols[mid].b0_prj
                     : kind == 2 ? mols[mid].b0_sel
                                 : mols[mid].b0_epi;
        if (b0 <= bid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_bcd_init(const CdMol* __restrict__ mols, int nmol, int32_t scheme, double delta) {
    const int c = find_mol(mols, nmol, blockIdx.x, 0);
    const CdMol& m = mols[c];
    cd_init_body(m.pd, m.atom, scheme, m.n, delta, m.D, m.cand, m.blk_a, m.blk_b, m.ctrl,
                 blockIdx.x - m.b0_init, m.nb_init);
}

__global__ void k_bcd_select(const CdMol* __restrict__ mols, int nmol, int32_t k) {
    const int c = find_mol(mols, nmol, blockIdx.x, 2);
    const CdMol& m = mols[c];
    cd_select_body(m.n, k, m.max_rank, m.D, m.cand, m.blk_i, m.piv, m.ctrl,
                   blockIdx.x - m.b0_sel, m.nb_sel);
}

__global__ void __launch_bounds__(kUpdThreads, 3) k_bcd_project(const CdMol* __restrict__ mols,
                                                                int nmol, int32_t k) {
    const int c = find_mol(mols, nmol, blockIdx.x, 1);
    const CdMol& m = mols[c];
    if (k >= m.max_rank || m.ctrl->done) return;
    const int local = blockIdx.x - m.b0_prj;
    if (local < m.nb_eri) cd_eri_body(m.pd, m.n, m.ctrl, m.ecol, local, m.nb_eri);
    else if (k > 0) cd_dot_body<false>(m.n, k, m.L, m.ctrl, local - m.nb_eri);
}

// Float-pair form, as the single-molecule k_cd_project_spec: each molecule's
// integral column in float pairs, then, when its step starts a batch of
// speculative candidates, the 4-candidate projection tiles.
__global__ void __launch_bounds__(kUpdThreads, 3) k_bcd_project_spec(const CdMol* __restrict__ mols,
                                                                     int nmol, int32_t k) {
    const int c = find_mol(mols, nmol, blockIdx.x, 1);
    const CdMol& m = mols[c];
    if (k >= m.max_rank || m.ctrl->done) return;
    const int local = blockIdx.x - m.b0_prj;
    if (local < m.nb_eri)
        cd_eri_body_df(m.pd, m.pf, m.n, m.ctrl, reinterpret_cast<float2*>(m.ecol), local, m.nb_eri);
    else if (m.ctrl->pass)
        cd_spec_dot_body(m.n, k, m.L, m.G, m.ctrl, local - m.nb_eri);
}

template <bool SPEC>
__global__ void __launch_bounds__(kUpdThreads) k_bcd_update(const CdMol* __restrict__ mols,
                                                            int nmol, int32_t k) {
    const int c = find_mol(mols, nmol, blockIdx.x, 3);
    const CdMol& m = mols[c];
    if (k >= m.max_rank || m.ctrl->done) return;
    cd_step_body<SPEC, SPEC>(m.n, k, m.max_rank, m.L, m.D, m.cand, m.ecol, SPEC ? m.G : nullptr,
                               reinterpret_cast<long long*>(m.blk_a),
                               reinterpret_cast<long long*>(m.blk_b), m.blk_i, m.piv, m.ctrl,
                               blockIdx.x - m.b0_epi, m.nb_epi);
}

struct CdBatchLayout {
    CdMol* mols;          // device descriptors
    CdCtrl* ctrl;         // [nmol]
    char* per_mol;        // pair data, masks, block partials of every molecule
    size_t bytes;
};

static size_t cd_mol_bytes(int64_t n) {
    const size_t nb = (size_t)part_blocks(n);
    return 6 * align_up(n * sizeof(double)) + align_up(n) + 3 * align_up(nb * sizeof(double)) +
           5 * align_up(n * sizeof(float2)) + align_up((size_t)kSpec * n * sizeof(float2));
}

static CdBatchLayout cd_batch_layout(void* ws, int32_t nmol, const BatchMol* mols) {
    Carver c(ws);
    CdBatchLayout l;
    l.mols = c.take<CdMol>(std::max(nmol, 1));
    l.ctrl = c.take<CdCtrl>(std::max(nmol, 1));
    size_t per = 0;
    for (int i = 0; i < nmol; ++i) per += cd_mol_bytes(npair_of(mols[i].nbf));
    l.per_mol = c.take<char>(std::max<size_t>(per, 1));
    l.bytes = c.off;
    return l;
}

size_t cd_batch_workspace_bytes(int32_t nmol, const BatchMol* mols) {
    return cd_batch_layout(nullptr, nmol, mols).bytes;
}

// Blocking: M[c] receives molecule c's rank; returns the first non-OK status.
int cd_batch_decompose(int32_t nmol, const BatchMol* mols, const BatchOffsets* off,
                       const double* xyz, const double* alpha, const int32_t* atom, double delta,
                       int32_t scheme, int32_t precision, double* L, int32_t* piv, double* D,
                       int32_t* M_out, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (precision != CDS_PREC_FP64 && precision != CDS_PREC_F32X2) return CDS_ERR_UNSUPPORTED;
    const bool df = precision == CDS_PREC_F32X2;
    CdBatchLayout lay = cd_batch_layout(ws, nmol, mols);
    if (!ws || ws_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    std::vector<CdMol> h(nmol);
    char* p = lay.per_mol;
    int b_init = 0, b_prj = 0, b_sel = 0, b_epi = 0, kmax = 0;
    const int nsm = sm_count();
    for (int c = 0; c < nmol; ++c) {
        const int64_t n = npair_of(mols[c].nbf);
        const size_t nb = (size_t)part_blocks(n);
        CdMol& m = h[c];
        Carver cv(p);
        m.pd.p = cv.take<double>(n);
        m.pd.Px = cv.take<double>(n);
        m.pd.Py = cv.take<double>(n);
        m.pd.Pz = cv.take<double>(n);
        m.pd.Kp = cv.take<double>(n);
        m.cand = cv.take<uint8_t>(n);
        m.ecol = cv.take<double>(n);
        m.blk_a = cv.take<double>(nb);
        m.blk_b = cv.take<double>(nb);
        m.blk_i = cv.take<long long>(nb);
        m.pf = PairF2{cv.take<float2>(n), cv.take<float2>(n), cv.take<float2>(n),
                      cv.take<float2>(n), cv.take<float2>(n)};
        m.G = cv.take<float2>((size_t)kSpec * n);
        p += cd_mol_bytes(n);
        m.atom = atom + off[c].basis;
        m.L = L + off[c].L;
        m.D = D + off[c].pair;
        m.piv = piv + off[c].piv;
        m.ctrl = lay.ctrl + c;
        m.n = n;
        m.max_rank = mols[c].max_rank;
        m.b0_init = b_init; m.nb_init = cd_blocks(n); b_init += m.nb_init;
        m.b0_prj = b_prj; m.nb_eri = eri_blocks(n, nsm); m.nb_dot = dot_tiles(n);
        b_prj += m.nb_eri + m.nb_dot;
        m.b0_epi = b_epi; m.nb_epi = step_blocks(n); b_epi += m.nb_epi;
        m.b0_sel = b_sel; m.nb_sel = sel_blocks(n); b_sel += m.nb_sel;
        kmax = std::max(kmax, mols[c].max_rank);
        int st = build_pairs(mols[c].nbf, xyz + 3 * off[c].basis, alpha + off[c].basis, m.pd, stream);
        if (st) return st;
        if (df) {
            k_pairs_to_f2<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(m.pd, m.pf, n);
            CDS_LAUNCH_CHECK();
        }
    }
    CDS_CUDA_TRY(cudaMemcpyAsync(lay.mols, h.data(), sizeof(CdMol) * nmol, cudaMemcpyHostToDevice,
                                 stream));
    CDS_CUDA_TRY(cudaMemsetAsync(lay.ctrl, 0, sizeof(CdCtrl) * nmol, stream));
    k_bcd_init<<<b_init, kCdThreads, 0, stream>>>(lay.mols, nmol, scheme, delta);
    CDS_LAUNCH_CHECK();
    k_bcd_select<<<b_sel, kCdThreads, 0, stream>>>(lay.mols, nmol, 0);
    CDS_LAUNCH_CHECK();
    std::vector<CdCtrl> hc(nmol);
    for (int32_t k0 = 0; k0 <= kmax; k0 += kHostCheckEvery) {
        int32_t k1 = std::min(kmax, k0 + kHostCheckEvery);
        for (int32_t k = k0; k < k1; ++k) {
            if (df) {
                k_bcd_project_spec<<<b_prj, kUpdThreads, 0, stream>>>(lay.mols, nmol, k);
                k_bcd_update<true><<<b_epi, kUpdThreads, 0, stream>>>(lay.mols, nmol, k);
            } else {
                k_bcd_project<<<b_prj, kUpdThreads, 0, stream>>>(lay.mols, nmol, k);
                k_bcd_update<false><<<b_epi, kUpdThreads, 0, stream>>>(lay.mols, nmol, k);
            }
        }
        count_launches(2ull * (unsigned long long)(k1 - k0));
        CDS_CUDA_TRY(cudaGetLastError());
        CDS_CUDA_TRY(cudaMemcpyAsync(hc.data(), lay.ctrl, sizeof(CdCtrl) * nmol,
                                     cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
        bool all = true;
        for (int c = 0; c < nmol; ++c) all = all && hc[c].done;
        if (all) break;
    }
    int status = CDS_OK;
    for (int c = 0; c < nmol; ++c) {
        M_out[c] = hc[c].M;
        int st = hc[c].done ? hc[c].status : CDS_ERR_RANK_CAP;
        if (st && !status) status = st;
        if (df && hc[c].M > 0) {   // the float-pair vectors back to FP64, in place
            const int64_t cnt = (int64_t)hc[c].M * npair_of(mols[c].nbf);
            k_pairs_to_fp64<<<(unsigned)((cnt + 255) / 256), 256, 0, stream>>>(L + off[c].L, cnt);
            CDS_LAUNCH_CHECK();
        }
    }
    return status;
}

// ---------------------------------------------------------------------------
// Batched tensor-core form: every molecule's screening, then the steps of all
// molecules together, three launches per step for the whole batch (slicing,
// projection GEMM, update), each molecule with its own control block, live
// pairs, slice store and stop test.  A molecule's compact vectors ([max_rank]
// rows of its live pairs, float pairs) live at the start of its own rows of
// L and are spread into the full rows at the end.
// ---------------------------------------------------------------------------
struct CdMolTC {
    PairF2 pf;            // live pairs' data as float pairs
    double* L;            // compact vectors [max_rank][n] (float pairs)
    double* D;            // compact residual diagonal
    uint8_t* cand;
    int32_t* piv;         // compact pivots
    float* sigA;
    __nv_bfloat16* A;
    __nv_bfloat16* B;
    float* sigB;
    float2* G;
    double* blk_a;
    double* blk_b;
    long long* blk_i;
    CdCtrl* ctrl;
    int64_t n;            // live pairs
    int32_t max_rank;
    int32_t b0_epi, nb_epi;
    int32_t _pad;
};
static_assert(sizeof(CdMolTC) % 8 == 0 && sizeof(CdMolTC) / 8 <= kUpdThreads, "table entry copy");

// Slicing before the passes of the molecules that start one at this step:
// their items numbered molecule by molecule, spread over the grid.
__global__ void __launch_bounds__(kUpdThreads, 4)
k_bcd_project_tc(const CdMolTC* __restrict__ mols, int nmol) {
    pdl_trigger();
    pdl_wait();
    __shared__ long long s_pre[kMaxMolsTC + 1];
    for (int c = threadIdx.x; c < nmol; c += blockDim.x) {
        int32_t k, s0, nseg;
        int64_t a, b;
        tc_slice_counts(mols[c].ctrl, mols[c].n, k, s0, nseg, a, b);
        s_pre[c + 1] = a + b;
    }
    __syncthreads();
    if (threadIdx.x < 32) warp_prefix_smem(s_pre, nmol);
    __syncthreads();
    const long long total = s_pre[nmol];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int c = -1;
    long long lo = 0, hi = 0;
    int32_t k = 0, s0 = 0, nseg = 0;
    int64_t itemsA = 0, itemsB = 0;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total; it += stride) {
        if (it >= hi) {   // the molecule of item it: the last one with s_pre[c] <= it
            int l = 0, h = nmol - 1;
            while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (s_pre[mid] <= it) l = mid; else h = mid - 1;
            }
            c = l;
            lo = s_pre[c];
            hi = s_pre[c + 1];
            tc_slice_counts(mols[c].ctrl, mols[c].n, k, s0, nseg, itemsA, itemsB);
        }
        const CdMolTC& m = mols[c];
        tc_slice_item(it - lo, itemsA, m.n, reinterpret_cast<const float2*>(m.L), m.sigA, m.A,
                      m.B, m.sigB, m.ctrl, k, s0, nseg);
    }
}

// Vector k, residuals and next pivot of every molecule still running; block b
// belongs to molecule blk_mol[b].
__global__ void __launch_bounds__(kUpdThreads, 4)
k_bcd_update_tc(const CdMolTC* __restrict__ mols, const int32_t* __restrict__ blk_mol) {
    pdl_trigger();
    pdl_wait();
    __shared__ CdMolTC m;   // the molecule's table entry, read by every thread from here
    if (threadIdx.x < sizeof(CdMolTC) / 8)
        reinterpret_cast<long long*>(&m)[threadIdx.x] =
            reinterpret_cast<const long long*>(mols + blk_mol[blockIdx.x])[threadIdx.x];
    __syncthreads();
    if (m.ctrl->done) return;
    cd_step_body<true, true, true>(m.n, m.ctrl->kstep, m.max_rank, m.L, m.D, m.cand, nullptr, m.G,
                                   reinterpret_cast<long long*>(m.blk_a),
                                   reinterpret_cast<long long*>(m.blk_b), m.blk_i, m.piv, m.ctrl,
                                   (int)blockIdx.x - m.b0_epi, m.nb_epi, m.pf);
}

// Rows [0, M) of the compact vectors (float pairs, a copy) into the full FP64
// rows of L, whose screened entries were zeroed.
__global__ void k_bcd_tc_scatter(const float2* __restrict__ Lc, int64_t nc,
                                 const int32_t* __restrict__ live, double* __restrict__ L,
                                 int64_t n, int32_t M) {
    const int64_t total = (int64_t)M * nc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / nc, j = i - r * nc;
        const float2 v = Lc[i];
        L[r * n + live[j]] = (double)v.x + (double)v.y;
    }
}

// One molecule's region of the batched tensor-core workspace.
struct TcMolLay {
    PairSoA pd;
    PairF2 pf;
    uint8_t* cand;
    int32_t* live;
    int32_t* scan;
    double* Dc;
    uint8_t* candc;
    int32_t* pivc;
    float2* G;
    __nv_bfloat16* A;
    __nv_bfloat16* B;
    float* sigA;
    float* sigB;
    double* blk_a;
    double* blk_b;
    long long* blk_i;
    int32_t kcap;
};

static TcMolLay tc_mol_carve(Carver& c, int64_t n, int32_t max_rank) {
    TcMolLay l;
    const int nb = part_blocks(n);
    l.kcap = tc_kcap(max_rank);
    l.pd.p = c.take<double>(n);
    l.pd.Px = c.take<double>(n);
    l.pd.Py = c.take<double>(n);
    l.pd.Pz = c.take<double>(n);
    l.pd.Kp = c.take<double>(n);
    l.pf.p = c.take<float2>(n);
    l.pf.Px = c.take<float2>(n);
    l.pf.Py = c.take<float2>(n);
    l.pf.Pz = c.take<float2>(n);
    l.pf.Kp = c.take<float2>(n);
    l.cand = c.take<uint8_t>(n);
    l.live = c.take<int32_t>(n);
    l.scan = c.take<int32_t>(n / kScanChunk + 2);
    l.Dc = c.take<double>(n);
    l.candc = c.take<uint8_t>(n);
    l.pivc = c.take<int32_t>(std::max(max_rank, 1));
    l.G = c.take<float2>((size_t)kSpecTC * n);
    l.A = c.take<__nv_bfloat16>((size_t)kSlicesTC * n * l.kcap);
    l.B = c.take<__nv_bfloat16>((size_t)kSlicesTC * kSpecTC * l.kcap);
    l.sigA = c.take<float>(n);
    l.sigB = c.take<float>(kSpecTC);
    l.blk_a = c.take<double>(nb);
    l.blk_b = c.take<double>(nb);
    l.blk_i = c.take<long long>(nb);
    return l;
}

struct CdTcBatchLayout {
    CdMolTC* mols;
    CdTcMolGemm* gmols;
    char* maps;           // [nmol] tensor-map pairs
    CdCtrl* ctrl;
    int32_t* blk_mol;
    int32_t* err;
    float2* scratch;      // the compact rows of one molecule, copied before the scatter
    size_t bytes;
};

static CdTcBatchLayout cd_tc_batch_layout(void* ws, int32_t nmol, const BatchMol* mols,
                                          std::vector<TcMolLay>* per) {
    Carver c(ws);
    CdTcBatchLayout l;
    int64_t nblk = 0, scratch = 1;
    for (int i = 0; i < nmol; ++i) {
        const int64_t n = npair_of(mols[i].nbf);
        nblk += step_blocks(n);
        scratch = std::max<int64_t>(scratch, (int64_t)mols[i].max_rank * n);
    }
    l.mols = c.take<CdMolTC>(std::max(nmol, 1));
    l.gmols = c.take<CdTcMolGemm>(std::max(nmol, 1));
    l.maps = c.take<char>(cd_tc_maps_bytes() * std::max(nmol, 1));
    l.ctrl = c.take<CdCtrl>(std::max(nmol, 1));
    l.blk_mol = c.take<int32_t>(std::max<int64_t>(nblk, 1));
    l.err = c.take<int32_t>(4);
    l.scratch = c.take<float2>(scratch);
    if (per) per->resize(nmol);
    for (int i = 0; i < nmol; ++i) {
        TcMolLay m = tc_mol_carve(c, npair_of(mols[i].nbf), mols[i].max_rank);
        if (per) (*per)[i] = m;
    }
    l.bytes = c.off;
    return l;
}

size_t cd_tc_batch_workspace_bytes(int32_t nmol, const BatchMol* mols) {
    return cd_tc_batch_layout(nullptr, nmol, mols, nullptr).bytes;
}

// Molecules [g0, g1) of the batch (at most kMaxMolsTC), their screening done:
// the steps, then every molecule's rows, pivots and residuals.
static int cd_tc_batch_group(int32_t g0, int32_t g1, const BatchMol* mols,
                             const BatchOffsets* off, const std::vector<TcMolLay>& ml,
                             const CdTcBatchLayout& lay, double* L, int32_t* piv, double* D,
                             int32_t* M_out, int* status, cudaStream_t stream) {
    const int nm = g1 - g0;
    const int nsm = sm_count();
    std::vector<CdCtrl> hc(nm);
    CDS_CUDA_TRY(cudaMemcpyAsync(hc.data(), lay.ctrl + g0, sizeof(CdCtrl) * nm,
                                 cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    std::vector<CdMolTC> h(nm);
    std::vector<CdTcMolGemm> hg(nm);
    // host copies of the tensor maps (64-byte aligned, as the type requires)
    std::vector<char> maps_raw(cd_tc_maps_bytes() * nm + 64);
    char* hmaps = maps_raw.data() + (64 - reinterpret_cast<uintptr_t>(maps_raw.data()) % 64) % 64;
    std::vector<int32_t> bm;
    std::vector<int64_t> nlive(nm, 0);
    int32_t kmax = 0;
    for (int i = 0; i < nm; ++i) {
        const int c = g0 + i;
        const TcMolLay& m = ml[c];
        const int64_t nc = hc[i].nlive;
        CdMolTC& d = h[i];
        d = CdMolTC{};
        d.ctrl = lay.ctrl + c;
        if (nc <= 0) {   // no diagonal passed the test: NaN or a zero scale
            CdCtrl stop = hc[i];
            stop.done = 1;
            stop.status = CDS_ERR_NOT_PD;
            stop.M = 0;
            CDS_CUDA_TRY(cudaMemcpyAsync(lay.ctrl + c, &stop, sizeof(CdCtrl),
                                         cudaMemcpyHostToDevice, stream));
            CDS_CUDA_TRY(cudaStreamSynchronize(stream));   // `stop` is a stack copy
            hc[i] = stop;
            hg[i] = CdTcMolGemm{1, m.sigA, m.sigB, m.G, lay.ctrl + c};
            const int st = cd_tc_maps_encode(hmaps + cd_tc_maps_bytes() * i, 1, m.kcap,
                                             m.A, m.B);
            if (st) return st;
            continue;
        }
        if (step_blocks(nc) > kMaxBlocksTC) return CDS_ERR_UNSUPPORTED;
        nlive[i] = nc;
        d.pf = m.pf;
        d.L = L + off[c].L;
        d.D = m.Dc;
        d.cand = m.candc;
        d.piv = m.pivc;
        d.sigA = m.sigA;
        d.A = m.A;
        d.B = m.B;
        d.sigB = m.sigB;
        d.G = m.G;
        d.blk_a = m.blk_a;
        d.blk_b = m.blk_b;
        d.blk_i = m.blk_i;
        d.n = nc;
        d.max_rank = mols[c].max_rank;
        d.nb_epi = step_blocks(nc);
        kmax = std::max(kmax, mols[c].max_rank);
        k_cd_select<<<sel_blocks(nc), kCdThreads, 0, stream>>>(nc, 0, d.max_rank, m.Dc, m.candc,
                                                               m.blk_i, m.pivc, lay.ctrl + c);
        CDS_LAUNCH_CHECK();
        k_cd_tc_scales<<<(unsigned)((nc + 255) / 256), 256, 0, stream>>>(m.Dc, nc, m.sigA);
        CDS_LAUNCH_CHECK();
        hg[i] = CdTcMolGemm{nc, m.sigA, m.sigB, m.G, lay.ctrl + c};
        const int st = cd_tc_maps_encode(hmaps + cd_tc_maps_bytes() * i, nc, m.kcap, m.A,
                                         m.B);
        if (st) return st;
    }
    // the update grid: the largest molecules' blocks first, so the blocks
    // scheduled last (and the serial ends of their steps) are short
    std::vector<int> order;
    for (int i = 0; i < nm; ++i)
        if (nlive[i] > 0) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return nlive[a] > nlive[b]; });
    for (int i : order) {
        h[i].b0_epi = (int32_t)bm.size();
        for (int b = 0; b < h[i].nb_epi; ++b) bm.push_back(i);
    }
    if (!bm.empty()) {
        CDS_CUDA_TRY(cudaMemcpyAsync(lay.mols + g0, h.data(), sizeof(CdMolTC) * nm,
                                     cudaMemcpyHostToDevice, stream));
        CDS_CUDA_TRY(cudaMemcpyAsync(lay.gmols + g0, hg.data(), sizeof(CdTcMolGemm) * nm,
                                     cudaMemcpyHostToDevice, stream));
        CDS_CUDA_TRY(cudaMemcpyAsync(lay.maps + cd_tc_maps_bytes() * g0, hmaps,
                                     cd_tc_maps_bytes() * nm, cudaMemcpyHostToDevice, stream));
        CDS_CUDA_TRY(cudaMemcpyAsync(lay.blk_mol, bm.data(), sizeof(int32_t) * bm.size(),
                                     cudaMemcpyHostToDevice, stream));
        const CdMolTC* dm = lay.mols + g0;
        const unsigned nupd = (unsigned)bm.size();
        for (int32_t k0 = 0; k0 <= kmax; k0 += kHostCheckEvery) {
            const int32_t k1 = std::min(kmax, k0 + kHostCheckEvery);
            for (int32_t k = k0; k < k1; ++k) {
                CDS_CUDA_TRY(launch_pdl(k_bcd_project_tc, (unsigned)(4 * nsm), kUpdThreads, 0,
                                        stream, dm, nm));
                const int s2 = cd_tc_batch_gemm_launch(lay.gmols + g0,
                                                       lay.maps + cd_tc_maps_bytes() * g0, nm,
                                                       lay.err, stream);
                if (s2) return s2;
                CDS_CUDA_TRY(launch_pdl(k_bcd_update_tc, nupd, kUpdThreads, 0, stream, dm,
                                        (const int32_t*)lay.blk_mol));
            }
            count_launches(3ull * (unsigned long long)(k1 - k0));
            CDS_CUDA_TRY(cudaGetLastError());
            CDS_CUDA_TRY(cudaMemcpyAsync(hc.data(), lay.ctrl + g0, sizeof(CdCtrl) * nm,
                                         cudaMemcpyDeviceToHost, stream));
            CDS_CUDA_TRY(cudaStreamSynchronize(stream));
            bool all = true;
            for (int i = 0; i < nm; ++i) all = all && hc[i].done;
            if (all) break;
        }
    }
    for (int i = 0; i < nm; ++i) {
        const int c = g0 + i;
        const int64_t n = npair_of(mols[c].nbf), nc = nlive[i];
        M_out[c] = hc[i].M;
        status[c] = hc[i].done ? hc[i].status : CDS_ERR_RANK_CAP;
        if (nc <= 0) continue;
        const int32_t M = hc[i].M;
        double* Lm = L + off[c].L;
        if (M > 0) {
            CDS_CUDA_TRY(cudaMemcpyAsync(lay.scratch, Lm, (size_t)M * nc * sizeof(float2),
                                         cudaMemcpyDeviceToDevice, stream));
            CDS_CUDA_TRY(cudaMemsetAsync(Lm, 0, (size_t)M * n * sizeof(double), stream));
            const int64_t items = (int64_t)M * nc;
            k_bcd_tc_scatter<<<(unsigned)std::min<int64_t>((items + 255) / 256, 8 * nsm), 256, 0,
                               stream>>>(lay.scratch, nc, ml[c].live, Lm, n, M);
            CDS_LAUNCH_CHECK();
        }
        const int64_t fin = std::max<int64_t>(M, nc);
        k_screen_finish<<<(unsigned)((fin + 255) / 256), 256, 0, stream>>>(
            ml[c].pivc, M, ml[c].live, piv + off[c].piv, ml[c].Dc, nc, D + off[c].pair);
        CDS_LAUNCH_CHECK();
    }
    return CDS_OK;
}

// Blocking: M_out[c] receives molecule c's rank; returns the first non-OK
// status in molecule order.
int cd_batch_decompose_tc(int32_t nmol, const BatchMol* mols, const BatchOffsets* off,
                          const double* xyz, const double* alpha, const int32_t* atom,
                          double delta, int32_t scheme, double* L, int32_t* piv, double* D,
                          int32_t* M_out, void* ws, size_t ws_bytes, cudaStream_t stream) {
    std::vector<TcMolLay> ml;
    const CdTcBatchLayout lay = cd_tc_batch_layout(ws, nmol, mols, &ml);
    if (!ws || ws_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    CDS_CUDA_TRY(cudaMemsetAsync(lay.ctrl, 0, sizeof(CdCtrl) * nmol, stream));
    CDS_CUDA_TRY(cudaMemsetAsync(lay.err, 0, sizeof(int32_t), stream));
    // every molecule's diagonal, candidates and live pairs
    for (int c = 0; c < nmol; ++c) {
        const int64_t n = npair_of(mols[c].nbf);
        const TcMolLay& m = ml[c];
        int st = build_pairs(mols[c].nbf, xyz + 3 * off[c].basis, alpha + off[c].basis, m.pd,
                             stream);
        if (st) return st;
        double* Dm = D + off[c].pair;
        k_cd_init<<<cd_blocks(n), kCdThreads, 0, stream>>>(m.pd, atom + off[c].basis, scheme, n,
                                                           delta, Dm, m.cand, m.blk_a, m.blk_b,
                                                           lay.ctrl + c);
        CDS_LAUNCH_CHECK();
        const int nsb = (int)((n + kScanChunk - 1) / kScanChunk);
        k_screen_count<<<nsb, kScanThreads, 0, stream>>>(Dm, n, lay.ctrl + c, m.scan);
        CDS_LAUNCH_CHECK();
        k_screen_scan<<<1, 1024, 0, stream>>>(m.scan, nsb, lay.ctrl + c);
        CDS_LAUNCH_CHECK();
        k_screen_gather<<<nsb, kScanThreads, 0, stream>>>(m.pd, Dm, m.cand, n, lay.ctrl + c,
                                                          m.scan, m.live, m.pf, m.Dc, m.candc);
        CDS_LAUNCH_CHECK();
    }
    std::vector<int> status(nmol, CDS_OK);
    for (int32_t g0 = 0; g0 < nmol; g0 += kMaxMolsTC) {
        const int st = cd_tc_batch_group(g0, std::min(nmol, g0 + kMaxMolsTC), mols, off, ml, lay,
                                         L, piv, D, M_out, status.data(), stream);
        if (st) return st;
    }
    int32_t e = 0;   // a bounded wait of the projection GEMM gave up
    CDS_CUDA_TRY(cudaMemcpyAsync(&e, lay.err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    if (e) return CDS_ERR_TIMEOUT;
    for (int c = 0; c < nmol; ++c)
        if (status[c]) return status[c];
    return CDS_OK;
}

}  // namespace cds
