// AO->MO transform of the Cholesky vectors (paper Eq. transformation) on the
// tensor cores: tcgen05 MMAs with TMEM accumulators, operands staged by TMA.
//
// Per batch of kb vectors with A^K the unpacked N x N matrix of vector K:
//   GEMM 1   T^T[(K, nu)][r] = sum_mu A^K[nu][mu] Cj[mu][r]      (Cj = [C_occ | C_P])
//   GEMM 2   Lov[i][a][K]    = sum_nu T[(i, K)][nu] C[nu][o + a]
//   GEMM 3   Lp[t][q][K]     = sum_nu T[(o + t, K)][nu] C[nu][q]
// GEMM 1 is the transposed form so that its epilogue writes T[r][K][nu]
// along nu (coalesced), and T's rows (r, K) are then the A operand of GEMMs 2
// and 3, whose epilogues write 32 consecutive K of Lov / Lp per warp store.
//
// Precision: every operand x is split into x = hi + lo with hi = r(x) and
// lo = x - hi rounded to the same format, and each contraction is
//   hi.hi + (hi.lo + lo.hi)
// with FP32 accumulation in TMEM, the cross products in an accumulator of
// their own (the lo.lo product is dropped).
//   TF32X3: r = TF32 (11 significant bits, FP32 range), ~2^-21 per product.
//   BF16X3: r = BF16 (8 significant bits), ~2^-17 per product.
// Both need no scaling (FP32 exponent range).
//
// One kernel serves the three GEMMs: D[m][n] = sum_k A[m][k] B[n][k], both
// operands K-major (k contiguous), M tile 128, N tile tn <= 128 (multiple of
// 16), a persistent grid walking the tiles.  Warp 0 = TMA producer, warp 1 =
// TMEM allocator + MMA issuer, warps 2..5 = epilogue (one output row per
// thread).  Shared memory holds NSTAGE stages of {A_hi, A_lo, B_hi, B_lo}
// (rows of 64 bytes, 64-byte swizzle); TMEM holds two accumulator pairs so
// the epilogue of one tile overlaps the MMAs of the next.  Every wait is
// bounded (2 s of %globaltimer) and sets an error word instead of hanging.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "tcgen05.cuh"
#include "ao2mo_tc.cuh"
#include "split.cuh"

namespace cds {
namespace trc {

using namespace tc;

constexpr int TM = 128;                         // MMA M, rows per tile
constexpr int ROW_BYTES = 64;                   // one k-block row (64-byte swizzle)
constexpr int NSTAGE = 4;
constexpr int A_TILE = TM * ROW_BYTES;          // 8 KB
constexpr int B_TILE = 128 * ROW_BYTES;         // 8 KB (tn <= 128 rows)
constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;
constexpr int EPI_WARPS = 4;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;             // 2 buffers x (hi.hi + cross) x 128
constexpr size_t SMEM_BYTES = 1024 + NSTAGE * STAGE_BYTES + 256;

template <bool TF32>
struct Fmt {
    using E = SplitE<TF32>;                                   // operand container
    static constexpr int KE = ROW_BYTES / (int)sizeof(E);   // elements per k-block
    // instruction descriptor (without N): D f32, A/B tf32 (format 2) or
    // bf16 (format 1), both K-major, M = 128
    static constexpr uint32_t ID = (1u << 4) | ((TF32 ? 2u : 1u) << 7) | ((TF32 ? 2u : 1u) << 10) |
                                   ((uint32_t)(TM >> 4) << 24);
};

struct Maps {
    CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

struct Args {
    int32_t m, n, kblocks, tn, mtiles, ntiles;
    // output element (row m, column c) at (m / kdiv) rs_hi + (m % kdiv) rs_lo + c cs
    int64_t kdiv, rs_hi, rs_lo, cs;
    double* out;   // FP64 output, or null for the split output
    void* out_hi;  // split output (operand containers)
    void* out_lo;
    int32_t accumulate;   // FP64 output: add to it instead of overwriting
};

// Barrier over the 128 epilogue threads that ORs a flag across them.
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

template <bool TF32>
__global__ void __launch_bounds__(THREADS, 1)
k_tr_gemm(const __grid_constant__ Maps maps, const Args g, int32_t* __restrict__ err) {
    using F = Fmt<TF32>;
    using E = typename F::E;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stages = smem;
    uint64_t* bars = (uint64_t*)(smem + NSTAGE * STAGE_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + NSTAGE;
    uint64_t* tfull = bars + 2 * NSTAGE;
    uint64_t* tempty = tfull + 2;
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (int64_t)g.mtiles * g.ntiles;
    volatile int32_t* verr = err;

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
            const uint32_t bytes = 2u * A_TILE + 2u * (uint32_t)g.tn * ROW_BYTES;
            int stage = 0;
            uint32_t phase = 0;
            int32_t last_parity[NSTAGE];
            for (int i = 0; i < NSTAGE; ++i) last_parity[i] = -1;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                const int mt = (int)(tile % g.mtiles), nt = (int)(tile / g.mtiles);
                for (int kb = 0; kb < g.kblocks; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, verr)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[stage], bytes);
                    last_parity[stage] = (int32_t)phase;
                    const uint32_t st = smem_u32(stages + stage * STAGE_BYTES);
                    const int k0 = kb * F::KE;
                    tma_load_3d(st, &maps.a_hi, &full[stage], k0, mt * TM, 0);
                    tma_load_3d(st + A_TILE, &maps.a_lo, &full[stage], k0, mt * TM, 0);
                    tma_load_3d(st + 2 * A_TILE, &maps.b_hi, &full[stage], k0, nt * g.tn, 0);
                    tma_load_3d(st + 2 * A_TILE + B_TILE, &maps.b_lo, &full[stage], k0, nt * g.tn, 0);
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
            }
            // drain: the copies of every issued stage land before the CTA exits
            for (int i = 0; i < NSTAGE; ++i)
                if (last_parity[i] >= 0) mbar_wait(&full[i], (uint32_t)last_parity[i], verr, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t ID = F::ID | ((uint32_t)(g.tn >> 3) << 17);
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                if (!mbar_wait(&tempty[acc], aphase ^ 1u, verr)) break;
                fence_after();
                const uint32_t dh = tmem + (uint32_t)acc * 256u, dx = dh + 128u;
                for (int kb = 0; kb < g.kblocks; ++kb) {
                    if (!mbar_wait(&full[stage], phase, verr)) { ok = false; break; }
                    fence_after();
                    const uint32_t base = smem_u32(stages + stage * STAGE_BYTES);
                    const uint32_t ah = base, al = base + A_TILE;
                    const uint32_t bh = base + 2 * A_TILE, bl = bh + B_TILE;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {   // 32 bytes of k per MMA
                        const uint32_t off = kk * 32;
                        const uint32_t first = (kb | kk) ? 1u : 0u;
                        if constexpr (TF32) {
                            mma_tf32(dh, sdesc(ah + off), sdesc(bh + off), ID, first);
                            mma_tf32(dx, sdesc(ah + off), sdesc(bl + off), ID, first);
                            mma_tf32(dx, sdesc(al + off), sdesc(bh + off), ID, 1u);
                        } else {
                            mma_f16(dh, sdesc(ah + off), sdesc(bh + off), ID, first);
                            mma_f16(dx, sdesc(ah + off), sdesc(bl + off), ID, first);
                            mma_f16(dx, sdesc(al + off), sdesc(bh + off), ID, 1u);
                        }
                    }
                    mma_commit(&empty[stage]);
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
                if (++acc == 2) { acc = 0; aphase ^= 1u; }
            }
        }
    } else {
        // ---------------- epilogue (4 warps, one output row per thread) ----------------
        const int quad = warp & 3;   // TMEM lanes this warp may read
        const int row = quad * 32 + lane;
        int acc = 0;
        uint32_t aphase = 0;
        E* ohi = (E*)g.out_hi;
        E* olo = (E*)g.out_lo;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const bool bad = !mbar_wait(&tfull[acc], aphase, verr) || *verr;
            if (epi_any(bad)) break;
            fence_after();
            const int mt = (int)(tile % g.mtiles), nt = (int)(tile / g.mtiles);
            const int64_t m = (int64_t)mt * TM + row;
            const bool mok = m < g.m;
            const int64_t ob = mok ? (m / g.kdiv) * g.rs_hi + (m % g.kdiv) * g.rs_lo : 0;
            const int c_base = nt * g.tn;
            const int ncols = min(g.tn, g.n - c_base);
            const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)acc * 256u;
            if (nt * g.tn < g.n && (int64_t)mt * TM + quad * 32 < g.m) {
#pragma unroll 1
                for (int c0 = 0; c0 < ncols; c0 += 16) {
                    float xh[16], xx[16];
                    tmem_ld16(ta + c0, xh);
                    tmem_ld16(ta + 128u + c0, xx);
                    tmem_wait_ld();
                    if (mok) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (c0 + j < ncols) {
                                const int64_t e = ob + (int64_t)(c_base + c0 + j) * g.cs;
                                if (g.out) {
                                    const double v = (double)xh[j] + (double)xx[j];
                                    g.out[e] = g.accumulate ? g.out[e] + v : v;
                                } else {
                                    // hi.hi + cross as an exact FP32 pair (two-sum)
                                    const float s = xh[j] + xx[j];
                                    const float v = s - xh[j];
                                    const float r = (xh[j] - (s - v)) + (xx[j] - v);
                                    split_store<TF32>(s, r, ohi, olo, e);
                                }
                            }
                        }
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
            if (++acc == 2) { acc = 0; aphase ^= 1u; }
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

// Operand rows of C: CT[q][nu] = C[nu][q] (all nmo orbitals), and
// Cj[r][nu] = C[nu][r] for the occupied r < nocc, C[nu][orb[r - nocc]] after.
template <bool TF32>
__global__ void k_split_c(const double* __restrict__ C, int32_t N, int32_t nmo, int32_t nocc,
                          const int32_t* __restrict__ orb, int32_t np, int32_t ldk,
                          typename Fmt<TF32>::E* __restrict__ ct_hi,
                          typename Fmt<TF32>::E* __restrict__ ct_lo,
                          typename Fmt<TF32>::E* __restrict__ cj_hi,
                          typename Fmt<TF32>::E* __restrict__ cj_lo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nct = (int64_t)nmo * N, ncj = (int64_t)(nocc + np) * N;
    if (e >= nct + ncj) return;
    float f, r;
    if (e < nct) {
        const int q = (int)(e / N), nu = (int)(e % N);
        pair_of_double(C[(int64_t)nu * nmo + q], f, r);
        split_store<TF32>(f, r, ct_hi, ct_lo, (int64_t)q * ldk + nu);
    } else {
        const int64_t e2 = e - nct;
        const int rr = (int)(e2 / N), nu = (int)(e2 % N);
        const int q = rr < nocc ? rr : orb[rr - nocc];
        if (q >= 0 && q < nmo) pair_of_double(C[(int64_t)nu * nmo + q], f, r);
        else { f = __int_as_float(0x7fc00000); r = 0.f; }   // invalid orbital: NaN
        split_store<TF32>(f, r, cj_hi, cj_lo, (int64_t)rr * ldk + nu);
    }
}

// U[(K, nu)][mu] = A^K[nu][mu] for vectors K0 .. K0 + kb - 1, from FP64 rows
// of L or float-pair rows Lf.
template <bool TF32>
__global__ void k_unpack_split(const double* __restrict__ L, const float2* __restrict__ Lf,
                               int64_t npair, int32_t K0, int32_t kb, int32_t N, int32_t ldk,
                               typename Fmt<TF32>::E* __restrict__ u_hi,
                               typename Fmt<TF32>::E* __restrict__ u_lo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)kb * N * N) return;
    const int mu = (int)(e % N);
    const int64_t rn = e / N;   // K * N + nu
    const int nu = (int)(rn % N), K = (int)(rn / N);
    const int hi = max(mu, nu), lo = min(mu, nu);
    const int64_t I = (int64_t)(K0 + K) * npair + (int64_t)hi * (hi + 1) / 2 + lo;
    float f, r;
    if (Lf) {
        const float2 v = Lf[I];
        f = v.x;
        r = v.y;
    } else {
        pair_of_double(L[I], f, r);
    }
    split_store<TF32>(f, r, u_hi, u_lo, rn * ldk + mu);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline int32_t ld_of(int32_t N) { return (N + 7) / 8 * 8; }   // 16-byte row strides for both formats

struct Layout {
    void *ct_hi, *ct_lo, *cj_hi, *cj_lo, *u_hi, *u_lo, *t_hi, *t_lo;
    int32_t* err;
    unsigned long long* cnorm;   // largest column 1-norm of C (FP64 bits)
    size_t bytes;
};

Layout layout(void* ws, int32_t N, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max, bool tf32) {
    const size_t es = tf32 ? 4 : 2;
    const size_t ld = (size_t)ld_of(N), nc = (size_t)std::max(nocc + np, 1);
    Carver c(ws);
    Layout l;
    auto take = [&](size_t elems) { return (void*)c.take<char>(elems * es); };
    l.ct_hi = take((size_t)nmo * ld);
    l.ct_lo = take((size_t)nmo * ld);
    l.cj_hi = take(nc * ld);
    l.cj_lo = take(nc * ld);
    l.u_hi = take((size_t)kb_max * N * ld);
    l.u_lo = take((size_t)kb_max * N * ld);
    l.t_hi = take(nc * kb_max * ld);
    l.t_lo = take(nc * kb_max * ld);
    l.err = c.take<int32_t>(4);
    l.cnorm = c.take<unsigned long long>(1);
    l.bytes = c.off;
    return l;
}

// out = max_q sum_mu |C[mu][q]| (non-negative doubles order as their bits).
__global__ void k_col_norm1(const double* __restrict__ C, int32_t N, int32_t nmo,
                            unsigned long long* __restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nmo) return;
    double s = 0.0;
    for (int mu = 0; mu < N; ++mu) s += fabs(C[(int64_t)mu * nmo + q]);
    atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

// 2-D operand {k (contiguous, extent kdim), rows} as a 3-D map with a unit
// third dimension; box {KE, box_rows, 1}, 64-byte swizzle, zero fill outside.
bool make_operand_map(CUtensorMap* m, bool tf32, const void* base, uint64_t kdim, uint64_t rows,
                      uint64_t ld_elems, uint32_t box_rows) {
    auto enc = encoder();
    if (!enc) return false;
    const uint64_t es = tf32 ? 4 : 2;
    cuuint64_t dims[3] = {kdim, rows, 1};
    cuuint64_t strides[2] = {ld_elems * es, ld_elems * es * rows};
    cuuint32_t box[3] = {(cuuint32_t)(ROW_BYTES / es), box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                     const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// N tile for n columns: the fewest tiles of at most 128, each a multiple of 16.
int32_t tile_n(int32_t n) {
    const int32_t t = (n + 127) / 128;
    return std::min(128, ((n + t - 1) / t + 15) / 16 * 16);
}

template <bool TF32>
int run_gemm(const void* a_hi, const void* a_lo, int64_t a_rows, const void* b_hi,
             const void* b_lo, int64_t b_rows, int32_t kdim, int32_t ld, int64_t kdiv,
             int64_t rs_hi, int64_t rs_lo, int64_t cs, double* out, void* out_hi, void* out_lo,
             int32_t* err, cudaStream_t stream, bool accumulate = false) {
    if (a_rows <= 0 || b_rows <= 0 || kdim <= 0) return CDS_OK;
    if (a_rows > INT32_MAX - TM) return CDS_ERR_ARG;
    Args g;
    g.m = (int32_t)a_rows;
    g.n = (int32_t)b_rows;
    g.tn = tile_n(g.n);
    g.kblocks = (kdim + Fmt<TF32>::KE - 1) / Fmt<TF32>::KE;
    g.mtiles = (g.m + TM - 1) / TM;
    g.ntiles = (g.n + g.tn - 1) / g.tn;
    g.kdiv = kdiv;
    g.rs_hi = rs_hi;
    g.rs_lo = rs_lo;
    g.cs = cs;
    g.out = out;
    g.out_hi = out_hi;
    g.out_lo = out_lo;
    g.accumulate = accumulate ? 1 : 0;
    Maps maps;
    if (!make_operand_map(&maps.a_hi, TF32, a_hi, kdim, a_rows, ld, TM) ||
        !make_operand_map(&maps.a_lo, TF32, a_lo, kdim, a_rows, ld, TM) ||
        !make_operand_map(&maps.b_hi, TF32, b_hi, kdim, b_rows, ld, g.tn) ||
        !make_operand_map(&maps.b_lo, TF32, b_lo, kdim, b_rows, ld, g.tn))
        return CDS_ERR_CUDA;
    // per launch: the attribute belongs to the current device
    CDS_CUDA_TRY(cudaFuncSetAttribute(k_tr_gemm<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SMEM_BYTES));
    const int64_t tiles = (int64_t)g.mtiles * g.ntiles;
    const int grid = (int)std::min<int64_t>(tiles, device_sms());
    k_tr_gemm<TF32><<<grid, THREADS, SMEM_BYTES, stream>>>(maps, g, err);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

// The split products carry ~u = 2^-21 (TF32X3) or 2^-17 (BF16X3) of each
// product, so an element of C^T A C is off by up to ~u |C_p|_1 |C_q|_1 max|A|
// while the element itself is O(max|A|) (C^T S C = 1): ill-conditioned C
// (large column 1-norms, strong cancellation) makes the result meaningless.
// The call is refused when u max_q |C_q|_1^2 > 2^-8 (the exact-slice form
// serves those bases).  Blocking.
template <bool TF32>
int check_conditioning(int32_t N, int32_t nmo, const double* C, const Layout& l,
                       cudaStream_t stream) {
    CDS_CUDA_TRY(cudaMemsetAsync(l.cnorm, 0, sizeof(unsigned long long), stream));
    k_col_norm1<<<(nmo + 127) / 128, 128, 0, stream>>>(C, N, nmo, l.cnorm);
    CDS_LAUNCH_CHECK();
    unsigned long long h = 0;
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, l.cnorm, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    double n1;
    memcpy(&n1, &h, sizeof(n1));
    const double u = TF32 ? std::ldexp(1.0, -21) : std::ldexp(1.0, -17);
    return (u * n1 * n1 <= std::ldexp(1.0, -8)) ? CDS_OK : CDS_ERR_UNSUPPORTED;
}

template <bool TF32>
int columns(int32_t N, int32_t nmo, int32_t nocc, const double* C, const int32_t* orb, int32_t np,
            const Layout& l, cudaStream_t stream) {
    using E = typename Fmt<TF32>::E;
    const int64_t tot = (int64_t)(nmo + nocc + np) * N;
    const int cst = check_conditioning<TF32>(N, nmo, C, l, stream);
    if (cst) return cst;
    CDS_CUDA_TRY(cudaMemsetAsync(l.err, 0, sizeof(int32_t), stream));
    k_split_c<TF32><<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(
        C, N, nmo, nocc, orb, np, ld_of(N), (E*)l.ct_hi, (E*)l.ct_lo, (E*)l.cj_hi, (E*)l.cj_lo);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

template <bool TF32>
int batch(int32_t N, int32_t nmo, int32_t nocc, int32_t np, const double* L, const float2* Lf,
          int32_t K0, int32_t kb, int64_t ldK, double* Lov, double* Lp, const Layout& l,
          cudaStream_t stream) {
    using E = typename Fmt<TF32>::E;
    const int64_t npair = npair_of(N);
    const int32_t nv = nmo - nocc, nc = nocc + np, ld = ld_of(N);
    const bool ov = nocc > 0 && nv > 0;
    if ((!ov && np == 0) || kb <= 0) return CDS_OK;
    const int64_t tot = (int64_t)kb * N * N;
    k_unpack_split<TF32><<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(
        L, Lf, npair, K0, kb, N, ld, (E*)l.u_hi, (E*)l.u_lo);
    CDS_LAUNCH_CHECK();
    // GEMM 1: T^T[(K, nu)][r]; element ((K, nu), r) of T at (r kb + K) ld + nu
    int st = run_gemm<TF32>(l.u_hi, l.u_lo, (int64_t)kb * N, l.cj_hi, l.cj_lo, nc, N, ld, N, ld, 1,
                            (int64_t)kb * ld, nullptr, l.t_hi, l.t_lo, l.err, stream);
    if (st) return st;
    const size_t es = TF32 ? 4 : 2;
    if (ov) {   // GEMM 2: rows (i, K) of T against the virtual rows of CT
        st = run_gemm<TF32>(l.t_hi, l.t_lo, (int64_t)nocc * kb, (char*)l.ct_hi + (size_t)nocc * ld * es,
                            (char*)l.ct_lo + (size_t)nocc * ld * es, nv, N, ld, kb,
                            (int64_t)nv * ldK, 1, ldK, Lov + K0, nullptr, nullptr, l.err, stream);
        if (st) return st;
    }
    if (np > 0) {   // GEMM 3: rows (o + t, K) of T against all rows of CT
        const size_t toff = (size_t)nocc * kb * ld * es;
        st = run_gemm<TF32>((char*)l.t_hi + toff, (char*)l.t_lo + toff, (int64_t)np * kb, l.ct_hi,
                            l.ct_lo, nmo, N, ld, kb, (int64_t)nmo * ldK, 1, ldK, Lp + K0, nullptr,
                            nullptr, l.err, stream);
        if (st) return st;
    }
    return CDS_OK;
}

}  // namespace trc

int tr_split_gemm(int32_t precision, const void* a_hi, const void* a_lo, int64_t a_rows,
                  const void* b_hi, const void* b_lo, int64_t b_rows, int32_t kdim, int32_t ld,
                  int64_t kdiv, int64_t rs_hi, int64_t rs_lo, int64_t cs, double* out,
                  bool accumulate, int32_t* err, cudaStream_t stream) {
    if (!tc::device_ok()) return CDS_ERR_UNSUPPORTED;
    if (!out || kdiv <= 0 || ld < kdim) return CDS_ERR_ARG;
    if (precision == CDS_PREC_TF32X3)
        return trc::run_gemm<true>(a_hi, a_lo, a_rows, b_hi, b_lo, b_rows, kdim, ld, kdiv, rs_hi,
                                   rs_lo, cs, out, nullptr, nullptr, err, stream, accumulate);
    if (precision == CDS_PREC_BF16X3)
        return trc::run_gemm<false>(a_hi, a_lo, a_rows, b_hi, b_lo, b_rows, kdim, ld, kdiv, rs_hi,
                                    rs_lo, cs, out, nullptr, nullptr, err, stream, accumulate);
    return CDS_ERR_UNSUPPORTED;
}

size_t tr_tc_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max,
                             int32_t precision) {
    return trc::layout(nullptr, nbf, nmo, nocc, np, kb_max, precision == CDS_PREC_TF32X3).bytes;
}

int tr_tc_columns(int32_t nbf, int32_t nmo, int32_t nocc, const double* C, const int32_t* orb,
                  int32_t np, int32_t kb_max, int32_t precision, void* ws, cudaStream_t stream) {
    if (!tc::device_ok()) return CDS_ERR_UNSUPPORTED;
    const bool tf32 = precision == CDS_PREC_TF32X3;
    const trc::Layout l = trc::layout(ws, nbf, nmo, nocc, np, kb_max, tf32);
    return tf32 ? trc::columns<true>(nbf, nmo, nocc, C, orb, np, l, stream)
                : trc::columns<false>(nbf, nmo, nocc, C, orb, np, l, stream);
}

int tr_tc_batch(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, const double* L,
                const float2* Lf, int32_t K0, int32_t kb, int64_t ldK, double* Lov, double* Lp,
                int32_t kb_max, int32_t precision, void* ws, cudaStream_t stream) {
    if (kb > kb_max) return CDS_ERR_ARG;
    const bool tf32 = precision == CDS_PREC_TF32X3;
    const trc::Layout l = trc::layout(ws, nbf, nmo, nocc, np, kb_max, tf32);
    return tf32 ? trc::batch<true>(nbf, nmo, nocc, np, L, Lf, K0, kb, ldK, Lov, Lp, l, stream)
                : trc::batch<false>(nbf, nmo, nocc, np, L, Lf, K0, kb, ldK, Lov, Lp, l, stream);
}

int tr_tc_status(int32_t nbf, int32_t nmo, int32_t nocc, int32_t np, int32_t kb_max,
                 int32_t precision, void* ws, cudaStream_t stream) {
    const trc::Layout l =
        trc::layout(ws, nbf, nmo, nocc, np, kb_max, precision == CDS_PREC_TF32X3);
    int32_t h = 0;
    CDS_CUDA_TRY(cudaMemcpyAsync(&h, l.err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    return h;
}

}  // namespace cds
