// Exact-slice tensor-core projections of the Cholesky decomposition's
// streaming passes (CDS_PREC_OZAKI; paper Eq. gs_coulomb / Eq. CD: the
// projections sum_{K<k} L^K_I L^K_P of the left-looking Gram-Schmidt step).
//
// At a pass (step k0) the projections of kSpecTC candidate pivots S_c are
//   G[c][I] = sum_{K < k0} L^K_I L^K_{S_c},
// an (npair x k0) . (k0 x 32) product.  Every stored element L^K_I is held in
// the slice store as a 56-bit fixed-point number below the pair's scale
// sigma_I = a power of two above sqrt(D0_I) (so |L^K_I| < sigma_I for every K,
// Cauchy-Schwarz on the residual matrix), cut into eight 7-bit digits stored
// as exact BF16 slices (the error-free splitting of Ozaki, Ogita, Oishi and
// Rump, 2012, as in the exact-slice transform).  The products of slice pairs
// (s, t) with s + t <= 9 (1-based; 36 pairs) are exact; the dropped ones are
// below 2^-56 of sigma_I sigma_S per term.  Each of the 15 leading pairs
// (s + t <= 6) has a TMEM accumulator of its own, where its FP32 sum is exact
// for up to 1040 terms (K 127^2 < 2^24), so the K range runs in chunks of
// 1024; the 21 smaller pairs (terms below 2^-35 of sigma_I sigma_S) share a
// sixteenth, whose rounding stays near 1e-14 of sigma_I sigma_S.  The
// epilogue adds the sixteen in float pairs, scales by sigma_I sigma_S and
// adds the chunk to G.  Fewer bits or more sharing are not enough: a 42-bit
// store (~4e-11 on the vectors) or 15 pairs in one rounded accumulator
// (~1e-10) break the symmetry ties of the pivot rule differently from FP64,
// whose band is 1e-12 of the largest diagonal.
//
// Kernel: M tile 128 pairs, N = 32 candidates (16 accumulators x 32 columns
// fill TMEM), 2 TMA stages of {8 A slices, 8 B slices} (64-byte swizzled rows
// of 32 BF16), warp 0 = TMA producer, warp 1 = TMEM allocator + MMA issuer (72
// MMAs per 32 columns), warps 2..5 = epilogue.  The launch is enqueued at every step and returns at once unless
// the control block marks a pass.  Every wait is bounded and sets an error
// word instead of hanging.
#include <cuda_bf16.h>

#include <algorithm>
#include <new>

#include "cd.cuh"
#include "tcgen05.cuh"

namespace cds {
namespace cdtc {

using namespace tc;

constexpr int S = kSlicesTC;
constexpr int NACC = 16;
constexpr int TM = 128;
constexpr int TN = kSpecTC;                      // 32 candidates
constexpr int KE = kGroupTC;                     // BF16 per k-block (64-byte rows)
constexpr int CHUNK_KB = 32;                     // k-blocks per exact chunk (1024 <= 1040)
constexpr int NSTAGE = 2;
constexpr int A_SLICE = TM * 64;                 // 8 KB
constexpr int B_SLICE = TN * 64;                 // 2 KB
constexpr int STAGE_BYTES = S * (A_SLICE + B_SLICE);   // 80 KB
constexpr int EPI_WARPS = 4;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;              // 16 x 32
constexpr size_t SMEM_BYTES = 1024 + NSTAGE * STAGE_BYTES + 256;
static_assert(TN == 32 && NACC * TN <= (int)TMEM_COLS, "accumulators fit TMEM");

// kind::f16 descriptor: D f32, A/B bf16, K-major, N = 32, M = 128
constexpr uint32_t ID = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                        ((uint32_t)(TM >> 4) << 24);

// Slice pairs (s, t), s + t <= 7 (0-based), leading first; accumulators
// 0..14 take the pairs with s + t <= 4 one each, 15 the 21 with s + t in 5..7.
constexpr int UMAX = 7;
constexpr int NPAIRS = (UMAX + 1) * (UMAX + 2) / 2;   // 36 (every s, t < 8 with s + t <= 7)
struct PairTab {
    int s[NPAIRS], t[NPAIRS], acc[NPAIRS], first[NPAIRS];
};
__host__ __device__ constexpr PairTab make_pairs() {
    PairTab p{};
    bool seen[NACC] = {};
    int n = 0;
    for (int u = 0; u <= UMAX; ++u)
        for (int s = 0; s <= u; ++s) {
            const int acc = u <= 4 ? n : NACC - 1;
            p.s[n] = s;
            p.t[n] = u - s;
            p.acc[n] = acc;
            p.first[n] = seen[acc] ? 0 : 1;
            seen[acc] = true;
            ++n;
        }
    return p;
}
static_assert(make_pairs().acc[14] == 14 && make_pairs().acc[NPAIRS - 1] == NACC - 1,
              "pair table");

struct Maps {
    CUtensorMap a, b;   // 3-D {k, rows, slice}
};

struct Args {
    int64_t n;          // pair rows
    int32_t mtiles;
    const float* sa;    // [n] pair scales
    const float* sb;    // [TN] candidate scales
    float2* G;          // [TN][n]
    const CdCtrl* ctrl;
};

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    return make_float2(s, (a - (s - v)) + (b - v));
}
__device__ __forceinline__ float2 pair_add(float2 x, float b) {
    const float2 s = two_sum(x.x, b);
    const float lo = s.y + x.y;
    const float h = s.x + lo;
    return make_float2(h, lo - (h - s.x));
}
__device__ __forceinline__ float2 pair_add2(float2 x, float2 y) {
    const float2 s = two_sum(x.x, y.x);
    const float lo = s.y + x.y + y.y;
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
k_cd_gemm_tc(const __grid_constant__ Maps maps, const Args g, int32_t* __restrict__ err) {
    // the same decision in every thread: nothing to do unless this step starts a pass
    if (g.ctrl->done || !g.ctrl->pass) return;
    const int32_t k0 = g.ctrl->k0;
    if (k0 <= 0) return;   // the first step projects on nothing (the update takes 0)
    const int kblocks = (k0 + KE - 1) / KE;
    const int nchunk = (kblocks + CHUNK_KB - 1) / CHUNK_KB;

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
    // work unit = (tile, chunk): a CTA takes tiles round robin and every chunk
    // of its tile in order, so the chunks of one G tile are added by one CTA
    const int64_t my_units = g.mtiles > (int64_t)blockIdx.x
                                 ? ((g.mtiles - 1 - blockIdx.x) / gridDim.x + 1) * nchunk
                                 : 0;
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
            for (int64_t j = 0; ok && j < my_units; ++j) {
                const int mt = (int)(blockIdx.x + (j / nchunk) * gridDim.x), ch = (int)(j % nchunk);
                const int kb1 = min(kblocks, (ch + 1) * CHUNK_KB);
                for (int kb = ch * CHUNK_KB; kb < kb1; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, verr)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[stage], (uint32_t)STAGE_BYTES);
                    last_parity[stage] = (int32_t)phase;
                    const uint32_t st = smem_u32(stages + stage * STAGE_BYTES);
                    for (int s = 0; s < S; ++s) {
                        tma_load_3d(st + s * A_SLICE, &maps.a, &full[stage], kb * KE, mt * TM, s);
                        tma_load_3d(st + S * A_SLICE + s * B_SLICE, &maps.b, &full[stage], kb * KE,
                                    0, s);
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
            for (int64_t j = 0; ok && j < my_units; ++j) {
                const int ch = (int)(j % nchunk);
                const int kbeg = ch * CHUNK_KB, kb1 = min(kblocks, (ch + 1) * CHUNK_KB);
                if (!mbar_wait(tempty, aphase ^ 1u, verr)) break;
                fence_after();
                for (int kb = kbeg; kb < kb1; ++kb) {
                    if (!mbar_wait(&full[stage], phase, verr)) { ok = false; break; }
                    fence_after();
                    const uint32_t base = smem_u32(stages + stage * STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {   // 16 BF16 (32 bytes) of k per MMA
                        const uint32_t off = kk * 32;
#pragma unroll
                        for (int p = 0; p < NPAIRS; ++p) {
                            const uint32_t en = ((kb > kbeg) || kk || !kPairs.first[p]) ? 1u : 0u;
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
        // ---------------- epilogue (4 warps, one pair row per thread) ----------------
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        uint32_t aphase = 0;
        for (int64_t j = 0; j < my_units; ++j) {
            const bool bad = !mbar_wait(tfull, aphase, verr) || *verr;
            if (epi_any(bad)) break;
            fence_after();
            const int mt = (int)(blockIdx.x + (j / nchunk) * gridDim.x), ch = (int)(j % nchunk);
            const int64_t I = (int64_t)mt * TM + row;
            const bool ok = I < g.n;
            const float sa = ok ? g.sa[I] : 0.f;
            const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16);
            if ((int64_t)mt * TM + quad * 32 < g.n) {
#pragma unroll 1
                for (int c0 = 0; c0 < TN; c0 += 8) {
                    float a[NACC][8];
#pragma unroll
                    for (int q = 0; q < NACC; ++q) tmem_ld8(ta + (uint32_t)q * TN + c0, a[q]);
                    tmem_wait_ld();
                    if (ok) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int c = c0 + j;
                            // smallest first: the shared rest, then the exact pairs
                            float2 v = make_float2(a[NACC - 1][j], 0.f);
#pragma unroll
                            for (int q = NACC - 2; q >= 0; --q) v = pair_add(v, a[q][j]);
                            const float st = sa * g.sb[c];   // power of two: exact scaling
                            v = make_float2(v.x * st, v.y * st);
                            float2* dst = g.G + (int64_t)c * g.n + I;
                            *dst = ch == 0 ? v : pair_add2(*dst, v);
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

bool make_map(CUtensorMap* m, const void* base, uint64_t kcap, uint64_t rows, uint32_t box_rows) {
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {kcap, rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {kcap * 2, rows * kcap * 2};
    cuuint32_t box[3] = {(cuuint32_t)KE, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace cdtc

struct CdTcGemm {
    cdtc::Maps maps;
    cdtc::Args args;
    int32_t* err;
    int grid;
};

int cd_tc_gemm_setup(CdTcGemm** out, int64_t n, int32_t kcap, const void* a_planes,
                     const void* b_planes, const float* sigA, const float* sigB, float2* G,
                     const CdCtrl* ctrl, int32_t* err) {
    using namespace cdtc;
    *out = nullptr;
    if (!tc::device_ok()) return CDS_ERR_UNSUPPORTED;
    if (n <= 0 || kcap <= 0 || kcap % KE != 0 || n > INT32_MAX - TM) return CDS_ERR_ARG;
    CdTcGemm* g = new (std::nothrow) CdTcGemm;
    if (!g) return CDS_ERR_ARG;
    if (!make_map(&g->maps.a, a_planes, (uint64_t)kcap, (uint64_t)n, TM) ||
        !make_map(&g->maps.b, b_planes, (uint64_t)kcap, (uint64_t)TN, TN)) {
        delete g;
        return CDS_ERR_CUDA;
    }
    g->args.n = n;
    g->args.mtiles = (int32_t)((n + TM - 1) / TM);
    g->args.sa = sigA;
    g->args.sb = sigB;
    g->args.G = G;
    g->args.ctrl = ctrl;
    g->err = err;
    g->grid = (int)std::min<int64_t>(g->args.mtiles, tc::device_sms());
    // the attribute belongs to the current device: set it at every setup
    if (cudaFuncSetAttribute(k_cd_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES) != cudaSuccess) {
        delete g;
        return CDS_ERR_CUDA;
    }
    *out = g;
    return CDS_OK;
}

int cd_tc_gemm_launch(const CdTcGemm* g, cudaStream_t stream) {
    cdtc::k_cd_gemm_tc<<<g->grid, cdtc::THREADS, cdtc::SMEM_BYTES, stream>>>(g->maps, g->args,
                                                                            g->err);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

void cd_tc_gemm_free(CdTcGemm* g) { delete g; }

}  // namespace cds
