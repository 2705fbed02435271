// Float-pair arithmetic and the integral-column bodies shared by the
// Cholesky decomposition (cd.cu) and the atomic-basis fit (acd.cu).
#pragma once

#include "common.cuh"

namespace cds {

// Float-pair ("double-float") arithmetic: a value is hi + lo with two FP32
// numbers, |lo| <= ulp(hi)/2; products get their exact error from an FMA and
// sums from two-sum, so each operation is good to ~2^-44 relative, on the
// FP32 units (the FP64 pipe of this part does 2 FMA/clk/SM).
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bp = s - a.x;
    float e = (a.x - (s - bp)) + (b.x - bp);
    e += a.y + b.y;
    const float h = s + e;
    return make_float2(h, e - (h - s));
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float h = p + e;
    return make_float2(h, e - (h - p));
}

// 1/sqrt(x) for x > 0: a FP32 seed y, then one third-order Newton-type
// correction y (1 + r/2 + 3 r^2/8) with the residual r = 1 - x y^2 formed in
// float pairs (the seed's error ~2^-22 becomes ~2^-64, below the pair's own).
__device__ __forceinline__ float2 df_rsqrt(float2 x) {
    const float y = rsqrtf(x.x);
    const float y2 = y * y;
    const float2 yy = make_float2(y2, fmaf(y, y, -y2));
    const float2 r2 = df_add(make_float2(1.f, 0.f), df_neg(df_mul(x, yy)));
    const float r = r2.x + r2.y;
    const float c = y * (r * fmaf(0.375f, r, 0.5f));
    const float h = y + c;
    return make_float2(h, c - (h - y));
}

// acc += a * b in float pairs.
__device__ __forceinline__ void df_fma(float2& acc, float2 a, float2 b) {
    const float p = a.x * b.x;
    float pe = fmaf(a.x, b.x, -p);
    pe = fmaf(a.x, b.y, pe);
    pe = fmaf(a.y, b.x, pe);
    const float s = acc.x + p;
    const float bp = s - acc.x;
    const float err = (acc.x - (s - bp)) + (p - bp);
    acc.x = s;
    acc.y += err + pe;
}

// Pair data as float pairs (float-pair decomposition).
struct PairF2 {
    float2 *p, *Px, *Py, *Pz, *Kp;
};

__device__ __forceinline__ float2 to_f2(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

static __global__ void k_pairs_to_f2(PairSoA pd, PairF2 pf, int64_t n) {
    const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (I >= n) return;
    pf.p[I] = to_f2(pd.p[I]);
    pf.Px[I] = to_f2(pd.Px[I]);
    pf.Py[I] = to_f2(pd.Py[I]);
    pf.Pz[I] = to_f2(pd.Pz[I]);
    pf.Kp[I] = to_f2(pd.Kp[I]);
}

constexpr float kFarT = 36.f;   // erf(sqrt T) rounds to 1 in binary64 above
constexpr float kMidT = 16.f;   // erfc(sqrt T) small enough for FP32 above
constexpr float kPi3Hi = (float)kPi3;
constexpr float kPi3Lo = (float)(kPi3 - (double)kPi3Hi);

constexpr float kTwoPi52Hi = (float)kTwoPi52;
constexpr float kTwoPi52Lo = (float)(kTwoPi52 - (double)kTwoPi52Hi);

// Integral column (rho_I|rho_P) in float pairs from the float-pair pair data
// (grid-stride over the pairs, NT per pass), T = x / (p + q):
//   T >= 16: the point-charge form pi^3 (K_I/p)(K_P/q) / sqrt(p q |P-Q|^2),
//            times 1 - erfc(sqrt T) below T = 36;
//   T < 16:  2 pi^(5/2) (K_I/p)(K_P/q) / sqrt(p + q) F0(T), F0 from its Taylor
//            expansion around the nearest point of the 1/16 grid
//            (kBoysTaylorF2, eight float-pair terms).
// Values below the FP32 range (|K/p| < 1e-38, pairs of far-apart centres)
// come out as 0, an absolute error far below any other in the decomposition.
// The column is stored as float pairs.
// The pivot density's part of the float-pair column: its pair data and the
// constants pi^3 K_P/q and 2 pi^(5/2) K_P/q.
struct PivotF2 {
    float2 q, qx, qy, qz, pi3kq, tpkq;
};
__device__ __forceinline__ PivotF2 pivot_f2(PairF2 pf, int64_t P) {
    PivotF2 v;
    v.q = pf.p[P];
    v.qx = pf.Px[P];
    v.qy = pf.Py[P];
    v.qz = pf.Pz[P];
    const float2 kq = pf.Kp[P];
    v.pi3kq = df_mul(make_float2(kPi3Hi, kPi3Lo), kq);
    v.tpkq = df_mul(make_float2(kTwoPi52Hi, kTwoPi52Lo), kq);
    return v;
}

// One element (rho_I|rho_P) of the column.
__device__ __forceinline__ float2 eri_elem_df(PairF2 pf, int64_t I, const PivotF2& v) {
    const float2 pI = pf.p[I];
    const float2 dx = df_add(pf.Px[I], df_neg(v.qx));
    const float2 dy = df_add(pf.Py[I], df_neg(v.qy));
    const float2 dz = df_add(pf.Pz[I], df_neg(v.qz));
    const float2 d2 = df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
    const float2 x = df_mul(df_mul(pI, v.q), d2);
    const float sf = pI.x + v.q.x;
    float2 e;
    if (x.x >= kMidT * sf) {
        // T >= 16: F0 = (1/2) sqrt(pi/T) (1 - erfc(sqrt T)), and erfc(sqrt T)
        // <= 1.6e-8 is needed only to FP32 precision (its error then stays
        // below 1e-14 of F0); above T = 36 it is below half an ulp
        e = df_mul(df_mul(pf.Kp[I], v.pi3kq), df_rsqrt(x));
        if (x.x < kFarT * sf) e = df_mul(e, make_float2(1.f, -erfcf(sqrtf(x.x / sf))));
    } else {
        const float2 rs = df_rsqrt(df_add(pI, v.q));                  // 1 / sqrt(p + q)
        const float2 T = df_mul(x, df_mul(rs, rs));
        const int i = min(max(__float2int_rn(T.x * (float)kBoysPerUnit), 0), kBoysPoints - 1);
        const float2 d = df_add(T, make_float2(-(float)i * (1.f / (float)kBoysPerUnit), 0.f));
        const float2* c = kBoysTaylorF2[i];
        float2 f = c[kBoysOrder - 1];
#pragma unroll
        for (int m = kBoysOrder - 2; m >= 0; --m) f = df_add(df_mul(f, d), c[m]);
        e = df_mul(df_mul(df_mul(pf.Kp[I], v.tpkq), rs), f);
    }
    return e;
}

template <int NT>
__device__ __forceinline__ void eri_column_df(PairSoA pd, PairF2 pf, int64_t n, int64_t P,
                                              float2* __restrict__ ecol, int bid, int nblk) {
    (void)pd;
    const PivotF2 v = pivot_f2(pf, P);
    for (int64_t I = (int64_t)bid * NT + threadIdx.x; I < n; I += (int64_t)nblk * NT)
        ecol[I] = eri_elem_df(pf, I, v);
}

// Integral column (rho_I|rho_P) into ecol (blockDim.x == NT, grid-stride over
// the pairs of the molecule, NT per pass).  Most pairs lie far from a compact
// pivot density (T >= 36: one reciprocal square root, the point-charge form);
// the few nearer ones (F0 from the Taylor table) are gathered in shared memory
// and evaluated together, so the warps do not all run that path for one lane
// each.
template <int NT>
__device__ __forceinline__ void eri_column_fp64(PairSoA pd, int64_t n, int64_t P,
                                                double* __restrict__ ecol, int bid, int nblk) {
    __shared__ double near_x[NT], near_s[NT], near_k[NT];
    __shared__ int near_i[NT];
    __shared__ int near_n;
    const double q = pd.p[P], qx = pd.Px[P], qy = pd.Py[P], qz = pd.Pz[P], kq = pd.Kp[P];
    for (int64_t I0 = (int64_t)bid * NT; I0 < n; I0 += (int64_t)nblk * NT) {
        if (threadIdx.x == 0) near_n = 0;
        __syncthreads();
        const int64_t I = I0 + threadIdx.x;
        if (I < n) {
            double x, sm;
            eri_xs(pd.p[I], pd.Px[I], pd.Py[I], pd.Pz[I], q, qx, qy, qz, x, sm);
            const double kk = pd.Kp[I] * kq;
            if (eri_is_far(x, sm)) {
                ecol[I] = eri_far(kk, x);
            } else {
                const int slot = atomicAdd(&near_n, 1);
                near_x[slot] = x;
                near_s[slot] = sm;
                near_k[slot] = kk;
                near_i[slot] = threadIdx.x;
            }
        }
        __syncthreads();
        const int cnt = near_n;
        for (int j = threadIdx.x; j < cnt; j += NT)
            ecol[I0 + near_i[j]] = eri_near(near_k[j], near_x[j], near_s[j]);
        __syncthreads();   // near_n is reset by the next pass
    }
}

}  // namespace cds
