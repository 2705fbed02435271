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
// Rump, 2012, as in the exact-slice transform): slice s holds d_s 2^-7(s+1).
// The products of slice pairs (s, t) with s + t <= 7 (36 pairs) are kept; the
// dropped ones are below 2^-56 of sigma_I sigma_S per term.  Fewer bits are
// not enough: a 42-bit store (~4e-11 on the vectors) breaks the symmetry ties
// of the pivot rule differently from FP64, whose band is 1e-12 of the largest
// diagonal.
//
// Shape.  The MMA's M side is 128 pairs (one pair slice s per MMA), its N
// side 128 columns: four groups g = 0..3 of the 32 candidates, read as a
// window of a stack of candidate slices [3 zero groups][t = 0]..[t = 7]
// shifted so that column group g holds slice t = g - s (zero when negative)
// or t = g + 4 - s.  Each column group then receives products of one weight
// u = s + t, and two accumulators cover the 36 pairs with 12 MMAs of
// 128 x 128 x 16 per 16 columns of K:
//   X (u = g):      s = 0..3,  t = g - s;
//   Y (u = g + 4):  s = 0..7,  t = g + 4 - s.
// (One MMA of N = 32 per slice pair would re-read the 128-row pair operand
// 36 times; the tensor pipe's operand reads then bound the kernel.)  A column
// of an accumulator adds at most eight slice pairs of one weight, each term
// below 127^2 units of 2^-7(u+2), so its FP32 sum is exact for up to 128
// columns of K (8 x 128 x 127^2 < 2^24): K runs in chunks of 128, and the
// epilogue adds a chunk's eight group values per candidate in float pairs,
// finest first, keeps the tile's sum over the chunks in registers and at the
// end scales it by sigma_I sigma_S (powers of two).
//
// Kernel: M tile 128 pairs; TMEM holds two buffers of the two accumulators
// (2 x 2 x 128 columns), so the epilogue of one chunk overlaps the MMAs of
// the next; 2 TMA stages of {8 pair slices (64 KB), 8 candidate slices
// (16 KB) behind 6 KB of zero groups}; the stores are blocked by 32-column
// groups, [group][slice][row][32], so each stage is two boxes of contiguous
// rows (64-byte swizzled).  Warp 0 = TMA producer, warp 1 = TMEM allocator +
// MMA issuer, warps 2..5 = epilogue (one pair row per thread).  The launch is
// enqueued at every step and returns at once unless the control block marks a
// pass.  Every wait is bounded and sets an error word instead of hanging.
#include <cuda_bf16.h>

#include <algorithm>
#include <new>

#include "cd.cuh"
#include "tcgen05.cuh"

namespace cds {
namespace cdtc {

using namespace tc;

constexpr int S = kSlicesTC;                     // 8 slices
constexpr int NC = kSpecTC;                      // 32 candidates
constexpr int KE = kGroupTC;                     // BF16 per k-block (64-byte rows)
constexpr int TM = 128;                          // pairs per tile
constexpr int TN = 4 * NC;                       // 128: four column groups of candidates
constexpr int ZG = 3;                            // zero groups below the candidate slices
constexpr int A_SLICE = TM * 64;                 // 8 KB
constexpr int GRP = NC * 64;                     // 2 KB: one group of 32 candidate rows
constexpr int B_OFF = S * A_SLICE;               // 64 KB
constexpr int STAGE_BYTES = B_OFF + (ZG + S) * GRP;  // 86 KB
constexpr uint32_t TX_BYTES = S * A_SLICE + S * GRP; // loaded per stage (the zeros are not)
constexpr int NSTAGE = 2;
constexpr int CHUNK_KB = 4;                      // k-blocks per exact chunk (128 columns)
constexpr int NACC = 2;
constexpr int BUF_COLS = NACC * TN;              // 256 TMEM columns per buffer
constexpr uint32_t TMEM_COLS = 512;
constexpr int EPI_WARPS = 4;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr size_t SMEM_BYTES = 1024 + NSTAGE * STAGE_BYTES + 256;
static_assert(2 * BUF_COLS <= (int)TMEM_COLS, "two accumulator buffers fit TMEM");
static_assert(SMEM_BYTES <= 232448, "shared memory");
static_assert(A_SLICE % 512 == 0 && GRP % 512 == 0 && STAGE_BYTES % 1024 == 0,
              "swizzle atoms stay aligned");
static_assert(8 * CHUNK_KB * KE * 127 * 127 < (1 << 24), "chunk sums are exact in FP32");

// kind::f16 descriptor: D f32, A/B bf16, K-major, N = 128, M = 128
constexpr uint32_t ID = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                        ((uint32_t)(TM >> 4) << 24);

// The 12 MMAs of 16 columns of K: accumulator, pair slice s and the first
// stack group of the candidate window (column group g reads stack group
// w + g, candidate slice w + g - ZG).
struct MmaTab {
    int acc[12], s[12], w[12], first[12];
};
__host__ __device__ constexpr MmaTab make_mmas() {
    MmaTab m{};
    int n = 0;
    for (int s = 0; s < 4; ++s, ++n) { m.acc[n] = 0; m.s[n] = s; m.w[n] = ZG - s; m.first[n] = s == 0; }
    for (int s = 0; s < 8; ++s, ++n) { m.acc[n] = 1; m.s[n] = s; m.w[n] = ZG + 4 - s; m.first[n] = s == 0; }
    return m;
}
static_assert(make_mmas().w[3] == 0 && make_mmas().w[11] == 0 && make_mmas().w[4] + 3 == ZG + S - 1,
              "windows stay inside the stack");

struct Maps {
    CUtensorMap a, b;   // a: pair slices, b: candidate slices; 3-D {k in group, rows, group x S + slice}
};

struct Args {
    int64_t n;          // pair rows
    int32_t mtiles;
    const float* sa;    // [n] pair scales
    const float* sb;    // [NC] candidate scales
    float2* G;          // [NC][n]
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

// One M tile of a pass: the molecule's maps, the tile row, its K extent and
// where the projections go.
struct TileRef {
    const CUtensorMap* a;
    const CUtensorMap* b;
    int mt;             // tile of 128 pair rows
    int kblocks;        // 32-column k-blocks of the pass (k0 rounded up)
    int nchunk;         // exact chunks of CHUNK_KB k-blocks
    int64_t n;          // pair rows of the molecule
    const float* sa;
    const float* sb;
    float2* G;
};

// The three roles over the tiles src.tile(0 .. src.count()-1) of this CTA,
// every chunk of a tile in order (one CTA sums a tile's chunks).  The TMEM
// buffer of the u-th chunk overall is u & 1, in every role.
template <class Src>
__device__ __forceinline__ void gemm_roles(const Src& src, uint8_t* smem, int32_t* err) {
    uint8_t* stages = smem;
    uint64_t* bars = (uint64_t*)(smem + NSTAGE * STAGE_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + NSTAGE;
    uint64_t* tfull = bars + 2 * NSTAGE;    // [2]
    uint64_t* tempty = tfull + 2;           // [2]
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = src.count();
    volatile int32_t* verr = err;

    // the zero groups below the candidate slices of every stage (never loaded)
    constexpr int ZQ = ZG * GRP / 16;
    for (int i = threadIdx.x; i < NSTAGE * ZQ; i += blockDim.x)
        reinterpret_cast<uint4*>(stages + (i / ZQ) * STAGE_BYTES + B_OFF)[i % ZQ] =
            make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int i = 0; i < NSTAGE; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], EPI_WARPS); }
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
            for (int j = 0; ok && j < ntiles; ++j) {
                const TileRef t = src.tile(j);
                for (int kb = 0; kb < t.kblocks; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, verr)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[stage], TX_BYTES);
                    last_parity[stage] = (int32_t)phase;
                    const uint32_t st = smem_u32(stages + stage * STAGE_BYTES);
                    tma_load_3d(st, t.a, &full[stage], 0, t.mt * TM, kb * S);
                    tma_load_3d(st + B_OFF + ZG * GRP, t.b, &full[stage], 0, 0, kb * S);
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
            }
            for (int i = 0; i < NSTAGE; ++i)
                if (last_parity[i] >= 0) mbar_wait(&full[i], (uint32_t)last_parity[i], verr, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr MmaTab kM = make_mmas();
            int stage = 0;
            uint32_t phase = 0, u = 0;
            bool ok = true;
            for (int j = 0; ok && j < ntiles; ++j) {
                const TileRef t = src.tile(j);
                for (int ch = 0; ok && ch < t.nchunk; ++ch, ++u) {
                    const int buf = (int)(u & 1);
                    const uint32_t use = (u >> 1) & 1;
                    const int kbeg = ch * CHUNK_KB, kb1 = min(t.kblocks, (ch + 1) * CHUNK_KB);
                    if (!mbar_wait(&tempty[buf], use ^ 1u, verr)) { ok = false; break; }
                    fence_after();
                    const uint32_t dbase = tmem + (uint32_t)(buf * BUF_COLS);
                    for (int kb = kbeg; kb < kb1; ++kb) {
                        if (!mbar_wait(&full[stage], phase, verr)) { ok = false; break; }
                        fence_after();
                        const uint32_t base = smem_u32(stages + stage * STAGE_BYTES);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {   // 16 BF16 (32 bytes) of k per MMA
                            const uint32_t off = kk * 32;
#pragma unroll
                            for (int q = 0; q < 12; ++q) {
                                const uint32_t en = ((kb > kbeg) || kk || !kM.first[q]) ? 1u : 0u;
                                mma_f16(dbase + (uint32_t)(kM.acc[q] * TN),
                                        sdesc(base + kM.s[q] * A_SLICE + off),
                                        sdesc(base + B_OFF + kM.w[q] * GRP + off), ID, en);
                            }
                        }
                        mma_commit(&empty[stage]);
                        if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mma_commit(&tfull[buf]);
                }
            }
        }
    } else {
        // ---------------- epilogue (4 warps, one pair row per thread) ----------------
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        float2 acc[NC];
        uint32_t u = 0;
        bool stop = false;
        for (int j = 0; !stop && j < ntiles; ++j) {
            const TileRef t = src.tile(j);
            for (int ch = 0; ch < t.nchunk; ++ch, ++u) {
                const int buf = (int)(u & 1);
                const uint32_t use = (u >> 1) & 1;
                const bool bad = !mbar_wait(&tfull[buf], use, verr) || *verr;
                if (epi_any(bad)) { stop = true; break; }
                fence_after();
                const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BUF_COLS);
#pragma unroll
                for (int c0 = 0; c0 < NC; c0 += 8) {
                    float x[4][8], y[4][8];
#pragma unroll
                    for (int gq = 0; gq < 4; ++gq) {
                        tmem_ld8(ta + (uint32_t)(gq * NC + c0), x[gq]);
                        tmem_ld8(ta + (uint32_t)(TN + gq * NC + c0), y[gq]);
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        // weights 7, 6, 5, 4 (Y), then 3, 2, 1, 0 (X): finest first
                        float2 v = two_sum(y[3][i], y[2][i]);
                        v = pair_add(v, y[1][i]);
                        v = pair_add(v, y[0][i]);
                        v = pair_add(v, x[3][i]);
                        v = pair_add(v, x[2][i]);
                        v = pair_add(v, x[1][i]);
                        v = pair_add(v, x[0][i]);
                        acc[c0 + i] = ch == 0 ? v : pair_add2(acc[c0 + i], v);
                    }
                }
                // this buffer is read: the MMAs may reuse it
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
                if (ch == t.nchunk - 1) {   // the tile's last chunk: scale and store
                    const int64_t I = (int64_t)t.mt * TM + row;
                    if (I < t.n) {
                        const float sa = t.sa[I];
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            const float st = sa * t.sb[c];   // power of two: exact scaling
                            t.G[(int64_t)c * t.n + I] = make_float2(acc[c].x * st, acc[c].y * st);
                        }
                    }
                }
            }
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

// The tiles of one molecule, round robin over the grid.
struct OneSrc {
    const Maps* maps;
    const Args* g;
    int kblocks, nchunk;
    __device__ int count() const {
        return g->mtiles > (int)blockIdx.x ? (g->mtiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    }
    __device__ TileRef tile(int j) const {
        return TileRef{&maps->a, &maps->b, (int)blockIdx.x + j * (int)gridDim.x, kblocks, nchunk,
                       g->n, g->sa, g->sb, g->G};
    }
};

__global__ void __launch_bounds__(THREADS, 1)
k_cd_gemm_tc(const __grid_constant__ Maps maps, const Args g, int32_t* __restrict__ err) {
    pdl_trigger();
    pdl_wait();
    // the same decision in every thread: nothing to do unless this step starts a pass
    if (g.ctrl->done || !g.ctrl->pass) return;
    const int32_t k0 = g.ctrl->k0;
    if (k0 <= 0) return;   // the first step projects on nothing (the update takes 0)
    const int kblocks = (k0 + KE - 1) / KE;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const OneSrc src{&maps, &g, kblocks, (kblocks + CHUNK_KB - 1) / CHUNK_KB};
    gemm_roles(src, smem, err);
}

// Batched form: the tiles of every molecule that starts a pass at this step,
// numbered molecule by molecule (s_pre: exclusive prefix of the molecules'
// tile counts), round robin over the grid.
struct BatchSrc {
    const CdTcMolGemm* mols;
    const Maps* maps;
    const int* pre;     // shared: [nmol + 1]
    int nmol, total;
    __device__ int count() const {
        return total > (int)blockIdx.x ? (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    }
    __device__ TileRef tile(int j) const {
        const int t = (int)blockIdx.x + j * (int)gridDim.x;
        int lo = 0, hi = nmol - 1;   // last molecule with pre[c] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const CdTcMolGemm& m = mols[lo];
        const int kblocks = (m.ctrl->k0 + KE - 1) / KE;
        return TileRef{&maps[lo].a, &maps[lo].b, t - pre[lo], kblocks,
                       (kblocks + CHUNK_KB - 1) / CHUNK_KB, m.n, m.sa, m.sb, m.G};
    }
};

__global__ void __launch_bounds__(THREADS, 1)
k_bcd_gemm_tc(const CdTcMolGemm* __restrict__ mols, const Maps* __restrict__ maps, int nmol,
              int32_t* __restrict__ err) {
    pdl_trigger();
    pdl_wait();
    __shared__ int s_pre[kMaxMolsTC + 1];
    for (int c = threadIdx.x; c < nmol; c += blockDim.x) {
        const CdCtrl* ctrl = mols[c].ctrl;
        const bool on = !ctrl->done && ctrl->pass && ctrl->k0 > 0;
        s_pre[c + 1] = on ? (int)((mols[c].n + TM - 1) / TM) : 0;
    }
    __syncthreads();
    if (threadIdx.x < 32) warp_prefix_smem(s_pre, nmol);
    __syncthreads();
    const int total = s_pre[nmol];
    if (total == 0) return;   // the same decision in every thread
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const BatchSrc src{mols, maps, s_pre, nmol, total};
    gemm_roles(src, smem, err);
}

// Group-blocked store [kcap / 32][S][rows][32] BF16: a box is the S slices of
// box_rows rows of one group.
bool make_map(CUtensorMap* m, const void* base, uint64_t kcap, uint64_t rows, uint32_t box_rows) {
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)KE, rows, (kcap / KE) * S};
    cuuint64_t strides[2] = {KE * 2, rows * KE * 2};
    cuuint32_t box[3] = {(cuuint32_t)KE, box_rows, (cuuint32_t)S};
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
        !make_map(&g->maps.b, b_planes, (uint64_t)kcap, (uint64_t)NC, NC)) {
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
    // in the pipeline the transform holds pipe_tr_ctas() SMs: take the others
    const int sms = tc::device_sms();
    const int avail = pipe_tr_ctas() > 0 && pipe_tr_ctas() < sms ? sms - pipe_tr_ctas() : sms;
    g->grid = (int)std::min<int64_t>(g->args.mtiles, avail);
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
    CDS_CUDA_TRY(launch_pdl(cdtc::k_cd_gemm_tc, (unsigned)g->grid, cdtc::THREADS, cdtc::SMEM_BYTES,
                            stream, g->maps, g->args, g->err));
    return CDS_OK;
}

void cd_tc_gemm_free(CdTcGemm* g) { delete g; }

size_t cd_tc_maps_bytes() { return sizeof(cdtc::Maps); }

int cd_tc_maps_encode(void* out, int64_t n, int32_t kcap, const void* a_planes,
                      const void* b_planes) {
    using namespace cdtc;
    if (!tc::device_ok()) return CDS_ERR_UNSUPPORTED;
    if (n <= 0 || kcap <= 0 || kcap % KE != 0 || n > INT32_MAX - TM) return CDS_ERR_ARG;
    Maps* m = static_cast<Maps*>(out);
    if (!make_map(&m->a, a_planes, (uint64_t)kcap, (uint64_t)n, TM) ||
        !make_map(&m->b, b_planes, (uint64_t)kcap, (uint64_t)NC, NC))
        return CDS_ERR_CUDA;
    return CDS_OK;
}

int cd_tc_batch_gemm_launch(const CdTcMolGemm* mols, const void* maps, int32_t nmol,
                            int32_t* err, cudaStream_t stream) {
    using namespace cdtc;
    if (nmol <= 0 || nmol > kMaxMolsTC) return CDS_ERR_ARG;
    static thread_local int attr_dev = -1;   // the attribute belongs to a device
    int dev = 0;
    CDS_CUDA_TRY(cudaGetDevice(&dev));
    if (attr_dev != dev) {
        CDS_CUDA_TRY(cudaFuncSetAttribute(k_bcd_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_BYTES));
        attr_dev = dev;
    }
    CDS_CUDA_TRY(launch_pdl(k_bcd_gemm_tc, (unsigned)tc::device_sms(), THREADS, SMEM_BYTES, stream,
                            mols, static_cast<const Maps*>(maps), (int)nmol, err));
    return CDS_OK;
}

}  // namespace cds
