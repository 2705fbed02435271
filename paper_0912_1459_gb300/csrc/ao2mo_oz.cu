// AO->MO transform of the Cholesky vectors (paper Eq. transformation) on the
// tensor cores with exact slice products (the error-free splitting of Ozaki,
// Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", 2012),
// accurate enough for ill-conditioned MO coefficients.
//
// Why: the transform's terms cancel by up to ~1e6 here (C = S^-1/2 Q reaches
// |C| ~ 100-300), so TF32 / BF16 split products accumulated in FP32 lose all
// digits.  With exact products and exact sums the only errors left are the
// truncation of the inputs and of the last accumulator.
//
// Slicing (per operand row, one warp per row): sigma = the power of two just
// above the row's largest |x|; q = trunc(x 2^42 / sigma) (a 42-bit integer);
// its magnitude is cut into six 7-bit digits d_1..d_6 (most significant
// first) and slice s holds sign(x) d_s 2^(-7 s) as BF16 (exact: 7 significant
// bits).  x = sigma (sum_s slice_s + O(2^-42)).
// Products: slice pairs (s, t) with s + t <= 7 (21 pairs; the dropped ones
// are below 2^-49).  For one pair sum_k |d_s e_t| <= K 127^2 < 2^24 when
// K <= 1040, so each of the six leading pairs (s + t <= 4) accumulates
// exactly in its own FP32 TMEM accumulator; the 15 others share a seventh,
// whose rounding is below 2^-45 of sigma_A sigma_B K.  The epilogue adds the
// seven in float-pair arithmetic and scales by sigma_A sigma_B.
//
// Per batch of kb vectors, as in the split-precision form:
//   GEMM 1   T^T[(K, nu)][r] = sum_mu A^K[nu][mu] Cj[mu][r]   -> T as float pairs
//   GEMM 2   Lov[i][a][K]    = sum_nu T[(i, K)][nu] C[nu][o + a]
//   GEMM 3   Lp[t][q][K]     = sum_nu T[(o + t, K)][nu] C[nu][q]
// with every operand sliced by rows (U rows (K, nu), Cj / C columns, T rows).
//
// Kernel: M tile 128, N tile 64, tiles ordered N fastest (the CTAs that share
// an A tile run together, so it is read from DRAM once); 3 TMA stages of
// {6 A slices, 6 B slices}
// (64-byte swizzled rows of 32 BF16); warp 0 = TMA producer, warp 1 = TMEM
// allocator + MMA issuer (21 MMAs per 16 k), warps 2..5 = epilogue.  Every
// wait is bounded and sets an error word instead of hanging.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "tcgen05.cuh"
#include "ao2mo_tc.cuh"

namespace cds {
namespace oz {

using namespace tc;

constexpr int S = 6;                             // slices per operand
constexpr int BETA = 7;                          // bits per slice
constexpr int QBITS = S * BETA;                  // 42-bit fixed point
constexpr int NACC = 7;                          // TMEM accumulators
constexpr int TM = 128;
constexpr int TN = 64;
constexpr int KE = 32;                           // BF16 per k-block (64-byte rows)
constexpr int NSTAGE = 3;
constexpr int A_SLICE = TM * 64;                 // 8 KB
constexpr int B_SLICE = TN * 64;                 // 4 KB
constexpr int STAGE_BYTES = S * (A_SLICE + B_SLICE);   // 72 KB
constexpr int EPI_WARPS = 4;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;              // 7 x 64 used
constexpr size_t SMEM_BYTES = 1024 + NSTAGE * STAGE_BYTES + 256;
constexpr int MAX_K = 1040;                      // exact accumulation bound (K 127^2 < 2^24)

// kind::f16 descriptor: D f32, A/B bf16, K-major, N = 64, M = 128
constexpr uint32_t ID = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                        ((uint32_t)(TM >> 4) << 24);

// (s, t) slice pairs with s + t <= 7 (0-based u = s + t <= 5), leading
// first; accumulators 0..5 take the pairs with u <= 2 one each, 6 the rest;
// first = the pair is the first one issued into its accumulator.
constexpr int NPAIRS = 21;
struct PairTab {
    int s[NPAIRS], t[NPAIRS], acc[NPAIRS], first[NPAIRS];
};
__host__ __device__ constexpr PairTab make_pairs() {
    PairTab p{};
    bool seen[NACC] = {};
    int n = 0;
    for (int u = 0; u <= S - 1; ++u)
        for (int s = 0; s <= u; ++s) {
            const int t = u - s;
            const int acc = u == 0 ? 0 : u == 1 ? 1 + s : u == 2 ? 3 + s : 6;
            p.s[n] = s;
            p.t[n] = t;
            p.acc[n] = acc;
            p.first[n] = seen[acc] ? 0 : 1;
            seen[acc] = true;
            ++n;
        }
    return p;
}
static_assert(make_pairs().acc[NPAIRS - 1] == 6 && make_pairs().s[NPAIRS - 1] == 5, "pair table");

struct Maps {
    CUtensorMap a, b;   // 3-D {k, rows, slice}
};

struct Args {
    int32_t m, n, kblocks, mtiles, ntiles;
    const float* sa;   // row scales of A (powers of two)
    const float* sb;   // row scales of B
    // output element (row m, column c) at (m / kdiv) rs_hi + (m % kdiv) rs_lo + c cs
    int64_t kdiv, rs_hi, rs_lo, cs;
    double* out;       // FP64 output, or
    float2* outf;      // float-pair output
};

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    return make_float2(s, (a - (s - v)) + (b - v));
}
// (hi, lo) + b, renormalised
__device__ __forceinline__ float2 pair_add(float2 x, float b) {
    const float2 s = two_sum(x.x, b);
    const float lo = s.y + x.y;
    const float h = s.x + lo;
    return make_float2(h, lo - (h - s.x));
}

__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(THREADS, 1)
k_oz_gemm(const __grid_constant__ Maps maps, const Args g, int32_t* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stages = smem;
    uint64_t* bars = (uint64_t*)(smem + NSTAGE * STAGE_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + NSTAGE;
    uint64_t* tfull = bars + 2 * NSTAGE;
    uint64_t* tempty = tfull + 1;
    uint32_t* tmem_slot = (uint32_t*)(tempty + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (int64_t)g.mtiles * g.ntiles;
    volatile int32_t* verr = err;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSTAGE; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        mbar_init(tfull, 1);
        mbar_init(tempty, EPI_WARPS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int32_t last_parity[NSTAGE];
            for (int i = 0; i < NSTAGE; ++i) last_parity[i] = -1;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                const int nt = (int)(tile % g.ntiles), mt = (int)(tile / g.ntiles);
                for (int kb = 0; kb < g.kblocks; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, verr)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[stage], (uint32_t)STAGE_BYTES);
                    last_parity[stage] = (int32_t)phase;
                    const uint32_t st = smem_u32(stages + stage * STAGE_BYTES);
                    for (int s = 0; s < S; ++s) {
                        tma_load_3d(st + s * A_SLICE, &maps.a, &full[stage], kb * KE, mt * TM, s);
                        tma_load_3d(st + S * A_SLICE + s * B_SLICE, &maps.b, &full[stage], kb * KE,
                                    nt * TN, s);
                    }
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
            }
            for (int i = 0; i < NSTAGE; ++i)
                if (last_parity[i] >= 0) mbar_wait(&full[i], (uint32_t)last_parity[i], verr, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr PairTab kPairs = make_pairs();
            int stage = 0;
            uint32_t phase = 0, aphase = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                if (!mbar_wait(tempty, aphase ^ 1u, verr)) break;
                fence_after();
                for (int kb = 0; kb < g.kblocks; ++kb) {
                    if (!mbar_wait(&full[stage], phase, verr)) { ok = false; break; }
                    fence_after();
                    const uint32_t base = smem_u32(stages + stage * STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {   // 16 BF16 (32 bytes) of k per MMA
                        const uint32_t off = kk * 32;
#pragma unroll
                        for (int p = 0; p < NPAIRS; ++p) {
                            const uint32_t en = ((kb | kk) || !kPairs.first[p]) ? 1u : 0u;
                            mma_f16(tmem + (uint32_t)kPairs.acc[p] * TN,
                                    sdesc(base + kPairs.s[p] * A_SLICE + off),
                                    sdesc(base + S * A_SLICE + kPairs.t[p] * B_SLICE + off), ID, en);
                        }
                    }
                    mma_commit(&empty[stage]);
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(tfull);
                aphase ^= 1u;
            }
        }
    } else {
        // ---------------- epilogue (4 warps, one output row per thread) ----------------
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        uint32_t aphase = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const bool bad = !mbar_wait(tfull, aphase, verr) || *verr;
            if (epi_any(bad)) break;
            fence_after();
            const int nt = (int)(tile % g.ntiles), mt = (int)(tile / g.ntiles);
            const int64_t m = (int64_t)mt * TM + row;
            const bool mok = m < g.m;
            const int64_t ob = mok ? (m / g.kdiv) * g.rs_hi + (m % g.kdiv) * g.rs_lo : 0;
            const float sa = mok ? g.sa[m] : 0.f;
            const int c_base = nt * TN;
            const int ncols = min(TN, g.n - c_base);
            const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16);
            if ((int64_t)mt * TM + quad * 32 < g.m) {
#pragma unroll 1
                for (int c0 = 0; c0 < ncols; c0 += 16) {
                    float a[NACC][16];
#pragma unroll
                    for (int q = 0; q < NACC; ++q) tmem_ld16(ta + (uint32_t)q * TN + c0, a[q]);
                    tmem_wait_ld();
                    if (mok) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int c = c_base + c0 + j;
                            if (c0 + j < ncols) {
                                // smallest first: rest, then the exact leading pairs
                                float2 v = make_float2(a[6][j], 0.f);
#pragma unroll
                                for (int q = 5; q >= 0; --q) v = pair_add(v, a[q][j]);
                                const float st = sa * g.sb[c];   // power of two
                                const int64_t e = ob + (int64_t)c * g.cs;
                                if (g.out) g.out[e] = (double)(v.x * st) + (double)(v.y * st);
                                else g.outf[e] = make_float2(v.x * st, v.y * st);
                            }
                        }
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty);
            aphase ^= 1u;
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// slicing (one warp per row)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pair_of(double x, float& f, float& r) {
    f = (float)x;
    r = (float)(x - (double)f);
}

// Operand row sources: element k of row `row` as a float pair.
struct SrcPackedL {      // U rows (K, nu) over mu: A^K[nu][mu] from rows of L
    const double* L;
    const float2* Lf;
    int64_t npair;
    int32_t K0, N;
    __device__ __forceinline__ void get(int64_t row, int k, float& f, float& r) const {
        const int K = (int)(row / N), nu = (int)(row % N);
        const int hi = max(k, nu), lo = min(k, nu);
        const int64_t I = (int64_t)(K0 + K) * npair + (int64_t)hi * (hi + 1) / 2 + lo;
        if (Lf) { const float2 v = Lf[I]; f = v.x; r = v.y; }
        else pair_of(L[I], f, r);
    }
};
struct SrcCols {         // row j over nu: C[nu][col(j)], col(j) = j < nocc ? j : orb[j - nocc] (orb may be null)
    const double* C;
    const int32_t* orb;
    int32_t nmo, nocc, first;
    __device__ __forceinline__ void get(int64_t row, int k, float& f, float& r) const {
        int q = (int)row + first;
        if (orb && q >= nocc) q = orb[q - nocc];
        if (q < 0 || q >= nmo) { f = __int_as_float(0x7fc00000); r = 0.f; return; }
        pair_of(C[(int64_t)k * nmo + q], f, r);
    }
};
struct SrcPairs {        // rows of a float-pair matrix [rows][ld]
    const float2* X;
    int32_t ld;
    __device__ __forceinline__ void get(int64_t row, int k, float& f, float& r) const {
        const float2 v = X[row * ld + k];
        f = v.x;
        r = v.y;
    }
};

template <typename Src>
__global__ void __launch_bounds__(256) k_oz_slice(Src src, int64_t rows, int32_t kdim, int32_t ld,
                                                  __nv_bfloat16* __restrict__ slices,
                                                  float* __restrict__ scale) {
    const int64_t row = blockIdx.x * 8LL + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    float mx = 0.f;
    for (int k = lane; k < kdim; k += 32) {
        float f, r;
        src.get(row, k, f, r);
        mx = fmaxf(mx, fabsf(f));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);          // mx = fr 2^e, fr in [0.5, 1): mx < 2^e
    if (lane == 0) scale[row] = ldexpf(1.f, e);   // the row scale (1 for a zero row)
    const int64_t plane = rows * (int64_t)ld;
    for (int k = lane; k < kdim; k += 32) {
        float f, r;
        src.get(row, k, f, r);
        // q = trunc(x 2^42 / sigma), |q| < 2^42 (f and r scaled by a power of two: exact)
        const long long q = __float2ll_rz(ldexpf(f, QBITS - e)) + __float2ll_rz(ldexpf(r, QBITS - e));
        const bool neg = q < 0;
        const unsigned long long aq = (unsigned long long)(neg ? -q : q);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int d = (int)((aq >> (QBITS - BETA * (s + 1))) & 127ull);
            const float v = ldexpf((float)(neg ? -d : d), -BETA * (s + 1));
            slices[s * plane + row * ld + k] = __float2bfloat16_rn(v);   // exact
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline int32_t ld_of(int32_t N) { return (N + 7) / 8 * 8; }

struct Layout {
    __nv_bfloat16 *ct, *cj, *u, *t;   // slices [S][rows][ld]
    float *ct_s, *cj_s, *u_s, *t_s;   // row scales
    float2* T;                        // GEMM 1 output [(o + np) kb][ld]
    int32_t* err;
    size_t bytes;
};

Layout layout(void* ws, int32_t N, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max) {
    const size_t ld = (size_t)ld_of(N), nc = (size_t)std::max(nocc + np, 1);
    const size_t urows = (size_t)kb_max * N, trows = nc * kb_max;
    Carver c(ws);
    Layout l;
    l.ct = c.take<__nv_bfloat16>(S * (size_t)nmo * ld);
    l.cj = c.take<__nv_bfloat16>(S * nc * ld);
    l.u = c.take<__nv_bfloat16>(S * urows * ld);
    l.t = c.take<__nv_bfloat16>(S * trows * ld);
    l.ct_s = c.take<float>((size_t)nmo);
    l.cj_s = c.take<float>(nc);
    l.u_s = c.take<float>(urows);
    l.t_s = c.take<float>(trows);
    l.T = c.take<float2>(trows * ld);
    l.err = c.take<int32_t>(4);
    l.bytes = c.off;
    return l;
}

// Slices [S][plane rows][ld] of which rows [0, rows) from base are used.
bool make_slice_map(CUtensorMap* m, const void* base, uint64_t kdim, uint64_t rows, uint64_t ld,
                    uint64_t plane, uint32_t box_rows) {
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {kdim, rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {ld * 2, plane * 2};
    cuuint32_t box[3] = {(cuuint32_t)KE, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// D = A B^T from sliced operands: rows [0, a_rows) of the A planes (plane
// stride a_plane elements) and [0, b_rows) of the B planes.
int run_gemm(const __nv_bfloat16* a, int64_t a_plane, const float* sa, int64_t a_rows,
             const __nv_bfloat16* b, int64_t b_plane, const float* sb, int64_t b_rows, int32_t kdim,
             int32_t ld, int64_t kdiv, int64_t rs_hi, int64_t rs_lo, int64_t cs, double* out,
             float2* outf, int32_t* err, cudaStream_t stream) {
    if (a_rows <= 0 || b_rows <= 0 || kdim <= 0) return CDS_OK;
    if (a_rows > INT32_MAX - TM || kdim > MAX_K) return CDS_ERR_ARG;
    Args g;
    g.m = (int32_t)a_rows;
    g.n = (int32_t)b_rows;
    g.kblocks = (kdim + KE - 1) / KE;
    g.mtiles = (g.m + TM - 1) / TM;
    g.ntiles = (g.n + TN - 1) / TN;
    g.sa = sa;
    g.sb = sb;
    g.kdiv = kdiv;
    g.rs_hi = rs_hi;
    g.rs_lo = rs_lo;
    g.cs = cs;
    g.out = out;
    g.outf = outf;
    Maps maps;
    if (!make_slice_map(&maps.a, a, kdim, a_rows, ld, a_plane, TM) ||
        !make_slice_map(&maps.b, b, kdim, b_rows, ld, b_plane, TN))
        return CDS_ERR_CUDA;
    // per launch: the attribute belongs to the current device
    CDS_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SMEM_BYTES));
    const int64_t tiles = (int64_t)g.mtiles * g.ntiles;
    const int cap = pipe_tr_ctas() > 0 ? std::min(pipe_tr_ctas(), device_sms()) : device_sms();
    const int grid = (int)std::min<int64_t>(tiles, cap);
    k_oz_gemm<<<grid, THREADS, SMEM_BYTES, stream>>>(maps, g, err);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

template <typename Src>
int slice(const Src& src, int64_t rows, int32_t kdim, int32_t ld, __nv_bfloat16* out, float* scale,
          cudaStream_t stream) {
    if (rows <= 0) return CDS_OK;
    k_oz_slice<Src><<<(unsigned)((rows + 7) / 8), 256, 0, stream>>>(src, rows, kdim, ld, out, scale);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

}  // namespace oz

size_t tr_oz_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max) {
    return oz::layout(nullptr, nbf, nmo, nocc, np, kb_max).bytes;
}

int tr_oz_columns(int32_t nbf, int32_t nmo, int32_t nocc, const double* C, const int32_t* orb,
                  int32_t np, int32_t kb_max, void* ws, cudaStream_t stream) {
    if (!tc::device_ok()) return CDS_ERR_UNSUPPORTED;
    if (nbf > oz::MAX_K) return CDS_ERR_UNSUPPORTED;
    const oz::Layout l = oz::layout(ws, nbf, nmo, nocc, np, kb_max);
    const int32_t ld = oz::ld_of(nbf);
    CDS_CUDA_TRY(cudaMemsetAsync(l.err, 0, sizeof(int32_t), stream));
    int st = oz::slice(oz::SrcCols{C, nullptr, nmo, nmo, 0}, nmo, nbf, ld, l.ct, l.ct_s, stream);
    if (st) return st;
    return oz::slice(oz::SrcCols{C, orb, nmo, nocc, 0}, nocc + np, nbf, ld, l.cj, l.cj_s, stream);
}

int tr_oz_batch(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, const double* L,
                const float2* Lf, int32_t K0, int32_t kb, int64_t ldK, double* Lov, double* Lp,
                int32_t kb_max, void* ws, cudaStream_t stream) {
    if (kb > kb_max) return CDS_ERR_ARG;
    const oz::Layout l = oz::layout(ws, nbf, nmo, nocc, np, kb_max);
    const int32_t N = nbf, nv = nmo - nocc, nc = nocc + np, ld = oz::ld_of(N);
    const bool ov = nocc > 0 && nv > 0;
    if ((!ov && np == 0) || kb <= 0) return CDS_OK;
    const int64_t urows = (int64_t)kb * N, trows = (int64_t)nc * kb;
    int st = oz::slice(oz::SrcPackedL{L, Lf, npair_of(N), K0, N}, urows, N, ld, l.u, l.u_s, stream);
    if (st) return st;
    // GEMM 1: T^T[(K, nu)][r] -> T[(r, K)][nu] as float pairs
    st = oz::run_gemm(l.u, urows * ld, l.u_s, urows, l.cj, (int64_t)nc * ld, l.cj_s, nc, N, ld, N,
                      ld, 1, (int64_t)kb * ld, nullptr, l.T, l.err, stream);
    if (st) return st;
    st = oz::slice(oz::SrcPairs{l.T, ld}, trows, N, ld, l.t, l.t_s, stream);
    if (st) return st;
    if (ov) {   // GEMM 2: rows (i, K) of T against the virtual rows of C
        st = oz::run_gemm(l.t, trows * ld, l.t_s, (int64_t)nocc * kb, l.ct + (size_t)nocc * ld,
                          (int64_t)nmo * ld, l.ct_s + nocc, nv, N, ld, kb, (int64_t)nv * ldK, 1, ldK,
                          Lov + K0, nullptr, l.err, stream);
        if (st) return st;
    }
    if (np > 0) {   // GEMM 3: rows (o + t, K) of T against all rows of C
        st = oz::run_gemm(l.t + (size_t)nocc * kb * ld, trows * ld, l.t_s + (size_t)nocc * kb,
                          (int64_t)np * kb, l.ct, (int64_t)nmo * ld, l.ct_s, nmo, N, ld, kb,
                          (int64_t)nmo * ldK, 1, ldK, Lp + K0, nullptr, l.err, stream);
        if (st) return st;
    }
    return CDS_OK;
}

int tr_oz_status(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max, void* ws,
                 cudaStream_t stream) {
    const oz::Layout l = oz::layout(ws, nbf, nmo, nocc, np, kb_max);
    int32_t h = 0;
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, l.err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    return h;
}

}  // namespace cds
