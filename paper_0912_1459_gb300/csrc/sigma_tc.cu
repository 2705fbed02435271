// Tensor-core path of the diagonal self-energy (paper Eq. SE) for sm_103a:
// tcgen05 MMAs with TMEM accumulators, operands staged by TMA.
//
// Precision: every factor L^J_pq is split in FP64 into two 16-bit parts,
// hi = r(s x) and lo = r(s x - hi), and each J-contraction is
//   X = (Ahi.Bhi + Ahi.Blo + Alo.Bhi) / (s_A s_B)
// with FP32 accumulation in TMEM (the lo.lo product is dropped).
//   BF16X3: r = bf16, s = 1             (~2^-17 relative per factor)
//   FP16X3: r = fp16, s = 2^k with max|s x| <= 1024, one power of two per
//           array found on the device (~2^-22 relative per factor, absolute
//           floor 2^-24 / s from fp16 subnormals).
// Denominators are double-FP32 pairs, (c_hi - e_hi) + (c_lo - e_lo), exact
// to ~1e-14 Ha so poles do not lose precision; per-element sums are FP32,
// per-tile totals are summed across tiles in FP64 in a fixed order.
//
// Work item = (term, orbital t, spectator s, x-block pair A <= B), 128 x 128
// blocks; see sigma.cuh for the exchange pairing.  Per item the CTA forms
//   D1 = Aq[A] . Bs[B]^T   and   D2 = Bs[A] . Aq[B]^T      (128 x 128 fp32)
// over the whole J range, so lane x / column y of D1 and D2 hold X_xy and
// X_yx.  A persistent grid (one CTA per SM) walks the items round robin.
//
// Warp roles (320 threads): warp 0 = TMA producer (one thread), warp 1 = TMEM
// allocator + MMA issuer (one thread), warps 2..9 = epilogue.  Shared memory
// holds 3 stages of 8 operand tiles (128 rows x 32 bf16, 64-byte swizzle);
// TMEM (512 columns) holds either one tile pair with separate hi.hi and
// cross-term accumulators (the default split modes; single-buffered, so the
// epilogue of one item and the MMAs of the next alternate) or, with the three
// products in one accumulator, two tile pairs so the epilogue of one item
// overlaps the MMAs of the next.  Every wait is bounded (2 s of %globaltimer)
// and sets an error word instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <atomic>
#include <vector>

#include "sigma_tc.cuh"
#include "tcgen05.cuh"

namespace cds {
namespace tc {

constexpr int TB = 128;                       // block of x / y = MMA M = N
constexpr int KB = 32;                        // bf16 per k-block (64-byte rows)
constexpr int NSTAGE = 3;
constexpr int TILE_BYTES = TB * KB * 2;       // 8 KB
constexpr int STAGE_BYTES = 8 * TILE_BYTES;   // 64 KB
constexpr int NUM_EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * NUM_EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr int RED_E = 64;                     // energies reduced per CTA barrier pair
constexpr int EPS_SMEM = 2048;                // orbital-energy pairs staged in shared memory
constexpr int kCacheTile = TB * TB;           // cached numerators per work item
constexpr int kGridSplitE = 1;                // energies of the grid the tensor-core epilogue evaluates
constexpr int kGridEC = 4;                    // k_sigma_cached_grid: energies per pass
constexpr size_t SMEM_BYTES = 1024 + NSTAGE * STAGE_BYTES + 256 + NUM_EPI_WARPS * RED_E * 2 * 4 +
                              EPS_SMEM * 8;

// Operand formats of the split products: FMT 0 = fp16, 1 = bf16 (kind::f16,
// 16-bit containers, K = 16 per MMA), 2 = tf32 (kind::tf32, 32-bit
// containers, K = 8 per MMA).  A k-block is one 64-byte row either way.
constexpr int FMT_TF32 = 2;
template <int FMT>
__host__ __device__ constexpr int kb_elems() { return FMT == FMT_TF32 ? KB / 2 : KB; }

// Instruction descriptor: D f32, A/B format fp16 (0), bf16 (1) or tf32 (2),
// both K-major, M = N = 128.
template <int FMT>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | ((uint32_t)FMT << 7) | ((uint32_t)FMT << 10) |
           ((uint32_t)(TB >> 3) << 17) | ((uint32_t)(TB >> 4) << 24);
}

struct Maps {
    CUtensorMap m[2][4];   // [term][aq_hi, aq_lo, bk_hi, bk_lo]
};

struct Term {
    int32_t nx, ns, nb, bulk_s_dim;   // bulk_s_dim: 1 if spectator is dim 1 of the bulk map, else 2
    int64_t npb, nitems, item0;
    int32_t eps_s_off, eps_x_off;     // offsets of the spectator / pair orbitals in eps
};

struct Params {
    Term term[2];
    int32_t kblocks;
    int32_t nE;
    int32_t nmo;
    int32_t nE_eval;   // energies the epilogue evaluates (0: all nE; the rest from the cache)
};

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Sum of two float pairs (hi, lo) by Knuth's two-sum, renormalised; exact to
// ~2^-44 relative, so small differences of O(1) energies keep their digits.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float v = s - a.x;
    const float e = (a.x - (s - v)) + (b.x - v) + (a.y + b.y);
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// Barrier over the 256 epilogue threads that also ORs a flag across them, so
// every epilogue warp takes the same branch afterwards.
__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 256, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// Fields of one term in registers (selected, never indexed dynamically, so the
// parameter block is not copied to local memory).
struct TermR {
    int32_t nx, ns, nb, bulk_s_dim;
    int64_t npb, item0, first;   // first: index of the term's first item within its molecule
    int32_t eps_s_off, eps_x_off;
};

__device__ __forceinline__ TermR term_regs(const Term& t0, const Term& t1, int term) {
    TermR r;
    r.nx = term ? t1.nx : t0.nx;
    r.ns = term ? t1.ns : t0.ns;
    r.nb = term ? t1.nb : t0.nb;
    r.bulk_s_dim = term ? t1.bulk_s_dim : t0.bulk_s_dim;
    r.npb = term ? t1.npb : t0.npb;
    r.item0 = term ? t1.item0 : t0.item0;
    r.first = term ? t0.nitems : 0;
    r.eps_s_off = term ? t1.eps_s_off : t0.eps_s_off;
    r.eps_x_off = term ? t1.eps_x_off : t0.eps_x_off;
    return r;
}

// (term, orbital t, spectator s, block pair A <= B) of item r of one molecule.
__device__ __forceinline__ TermR decode(const Term& t0, const Term& t1, int64_t r, int& term,
                                        int& t, int& s, int& A, int& B) {
    term = r < t0.nitems ? 0 : 1;
    const TermR tm = term_regs(t0, t1, term);
    r -= tm.first;
    int64_t per_t = (int64_t)tm.ns * tm.npb;
    t = (int)(r / per_t);
    r -= (int64_t)t * per_t;
    s = (int)(r / tm.npb);
    block_pair(r - (int64_t)s * tm.npb, tm.nb, A, B);
    return tm;
}

// One molecule of a batch, in global memory.  Offsets are in elements of the
// batch-wide arrays the kernel receives (E2, eps2, part, active).
struct alignas(64) MolDesc {
    CUtensorMap m[2][4];     // [term][aq_hi, aq_lo, bk_hi, bk_lo]
    Term term[2];
    int64_t item_begin;      // batch-wide index of the molecule's first item
    int64_t part_base;       // element offset of its first item's partial row
    int64_t E_off;           // its first energy pair
    int64_t eps_off;         // its first orbital-energy pair
    int32_t kblocks, nE, nmo, act_off;
    float inv;               // 1 / (s_A s_B) of its 16-bit split
    int32_t pad_[3];
};

// Everything a role needs to know about one work item.
struct View {
    TermR tm;
    int term, t, s, A, B;
    int kblocks, nE;
    const CUtensorMap* maps;   // the four maps of the item's term
    const float2* Et;          // energies of orbital t
    const float2* epsv;        // orbital energies of the molecule
    double* out;               // partial row of the item
    bool act;
    float inv;
    int mol;
};

constexpr int MAX_BATCH_SMEM = 512;   // molecules whose first-item index is cached in smem

template <bool BATCH>
__device__ __forceinline__ View make_view(int64_t item, const Maps& maps, const Params& P,
                                          const MolDesc* mols, const int64_t* s_begin, int nmol,
                                          const float2* E2, const float2* epsv,
                                          const int32_t* active, const float* inv_scale,
                                          double* part) {
    View v;
    if constexpr (!BATCH) {
        v.tm = decode(P.term[0], P.term[1], item, v.term, v.t, v.s, v.A, v.B);
        v.maps = &maps.m[v.term][0];
        v.kblocks = P.kblocks;
        v.nE = P.nE_eval > 0 ? min(P.nE, P.nE_eval) : P.nE;
        v.Et = E2 + (int64_t)v.t * P.nE;
        v.epsv = epsv;
        v.out = part + (v.tm.item0 + (item - v.tm.first)) * (int64_t)P.nE * 2;
        v.act = !active || active[v.t];
        v.inv = *inv_scale;
        v.mol = 0;
    } else {
        int lo = 0, hi = nmol - 1;   // last molecule whose first item is <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const int64_t b = mid < MAX_BATCH_SMEM ? s_begin[mid] : mols[mid].item_begin;
            if (b <= item) lo = mid; else hi = mid - 1;
        }
        const MolDesc* md = mols + lo;
        const int64_t r = item - md->item_begin;
        v.tm = decode(md->term[0], md->term[1], r, v.term, v.t, v.s, v.A, v.B);
        v.maps = &md->m[v.term][0];
        v.kblocks = md->kblocks;
        v.nE = P.nE_eval > 0 ? min(md->nE, P.nE_eval) : md->nE;
        v.Et = E2 + md->E_off + (int64_t)v.t * md->nE;
        v.epsv = epsv + md->eps_off;
        v.out = part + md->part_base + r * (int64_t)md->nE * 2;
        v.act = !active || active[md->act_off + v.t];
        v.inv = md->inv;
        v.mol = lo;
    }
    return v;
}

// SEP: hi.hi and the two cross products accumulate in separate TMEM tiles
// (4 x 128 columns, one buffer); otherwise all three share one tile and two
// buffers alternate between items.  BATCH: items of many molecules, described
// by MolDesc records in global memory, in one persistent launch.
// Items of CTA c: interleaved (c, c + G, c + 2G, ...) or, with blocked order,
// the contiguous range [c n / G, (c + 1) n / G).  k-th item, or -1 when done.
__device__ __forceinline__ int64_t item_at(int64_t k, int64_t n, int order) {
    if (order == 0) {
        const int64_t it = blockIdx.x + k * gridDim.x;
        return it < n ? it : -1;
    }
    const int64_t b = n * blockIdx.x / gridDim.x, e = n * (blockIdx.x + 1) / gridDim.x;
    return b + k < e ? b + k : -1;
}

template <int EC, int FMT, bool SEP, bool BATCH>
__global__ void __launch_bounds__(THREADS, 1)
k_sigma_tc(const __grid_constant__ Maps maps, const Params P, const MolDesc* __restrict__ mols,
           int32_t nmol, int64_t nitems_batch, const float2* __restrict__ E2,
           const float2* __restrict__ eps2, const int32_t* __restrict__ active,
           const float* __restrict__ inv_scale, double* __restrict__ part,
           unsigned long long* __restrict__ stamps, int32_t* __restrict__ err, int32_t order,
           float* __restrict__ cache) {
    constexpr uint32_t ID = idesc<FMT>();
    constexpr int NBUF = SEP ? 1 : 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stages = smem;
    uint64_t* bars = (uint64_t*)(smem + NSTAGE * STAGE_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + NSTAGE;
    uint64_t* tfull = bars + 2 * NSTAGE;
    uint64_t* tempty = tfull + 2;
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    float* red = (float*)(smem + NSTAGE * STAGE_BYTES + 256);   // [8 warps][RED_E][2]
    float2* seps = (float2*)(red + NUM_EPI_WARPS * RED_E * 2);   // [EPS_SMEM]
    int64_t* s_begin = (int64_t*)seps;                          // batch: first item per molecule

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nitems = BATCH ? nitems_batch : P.term[0].nitems + P.term[1].nitems;
    volatile int32_t* verr = err;

    if (BATCH) {
        for (int i = threadIdx.x; i < min(nmol, MAX_BATCH_SMEM); i += blockDim.x)
            s_begin[i] = mols[i].item_begin;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < NSTAGE; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < NBUF; ++i) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], NUM_EPI_WARPS); }
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
#define CDS_VIEW(item_) make_view<BATCH>(item_, maps, P, mols, s_begin, nmol, E2, eps2, active, \
                                         inv_scale, part)

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int32_t last_parity[NSTAGE];
            for (int i = 0; i < NSTAGE; ++i) last_parity[i] = -1;
            bool ok = true;
            for (int64_t kq = 0, item; ok && (item = item_at(kq, nitems, order)) >= 0; ++kq) {
                const View v = CDS_VIEW(item);
                if (!v.act) continue;
                const int t = v.t, s = v.s, A = v.A, B = v.B;
                const CUtensorMap* mq_hi = v.maps + 0;
                const CUtensorMap* mq_lo = v.maps + 1;
                const CUtensorMap* mb_hi = v.maps + 2;
                const CUtensorMap* mb_lo = v.maps + 3;
                const bool diag = A == B;
                const uint32_t bytes = (diag ? 4u : 8u) * TILE_BYTES;
                const bool sd2 = v.tm.bulk_s_dim == 2;
                const int bA1 = sd2 ? A * TB : s, bA2 = sd2 ? s : A * TB;
                const int bB1 = sd2 ? B * TB : s, bB2 = sd2 ? s : B * TB;
                for (int kb = 0; kb < v.kblocks; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, verr)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[stage], bytes);
                    last_parity[stage] = (int32_t)phase;
                    const uint32_t st = smem_u32(stages + stage * STAGE_BYTES);
                    const int k0 = kb * kb_elems<FMT>();
                    tma_load_3d(st + 0 * TILE_BYTES, mq_hi, &full[stage], k0, A * TB, t);
                    tma_load_3d(st + 1 * TILE_BYTES, mq_lo, &full[stage], k0, A * TB, t);
                    tma_load_3d(st + 2 * TILE_BYTES, mb_hi, &full[stage], k0, bB1, bB2);
                    tma_load_3d(st + 3 * TILE_BYTES, mb_lo, &full[stage], k0, bB1, bB2);
                    if (!diag) {
                        tma_load_3d(st + 4 * TILE_BYTES, mb_hi, &full[stage], k0, bA1, bA2);
                        tma_load_3d(st + 5 * TILE_BYTES, mb_lo, &full[stage], k0, bA1, bA2);
                        tma_load_3d(st + 6 * TILE_BYTES, mq_hi, &full[stage], k0, B * TB, t);
                        tma_load_3d(st + 7 * TILE_BYTES, mq_lo, &full[stage], k0, B * TB, t);
                    }
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
            }
            // drain: the copies of every issued stage must have landed before
            // the CTA exits (returns at once on the normal path)
            for (int i = 0; i < NSTAGE; ++i)
                if (last_parity[i] >= 0) mbar_wait(&full[i], (uint32_t)last_parity[i], verr, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool ok = true;
            for (int64_t kq = 0, item; ok && (item = item_at(kq, nitems, order)) >= 0; ++kq) {
                const View v = CDS_VIEW(item);
                if (!v.act) continue;
                const bool diag = v.A == v.B;
                // columns of both tiles come from block B: a ragged last block
                // runs with N = its valid rows rounded up to 16 (M = 128 takes
                // N = 16..256 in steps of 16); the epilogue reads only valid columns
                const int nyB = min(TB, v.tm.nx - v.B * TB);
                const uint32_t NB = (uint32_t)((nyB + 15) & ~15);
                const uint32_t IDn = (ID & ~(0x3Fu << 17)) | ((NB >> 3) << 17);
                if (!mbar_wait(&tempty[acc], aphase ^ 1u, verr)) break;
                fence_after();
                const uint32_t d1 = tmem + (uint32_t)acc * 256u, d2 = d1 + 128u;
                const uint32_t d1x = SEP ? tmem + 256u : d1, d2x = SEP ? tmem + 384u : d2;
                for (int kb = 0; kb < v.kblocks; ++kb) {
                    if (!mbar_wait(&full[stage], phase, verr)) { ok = false; break; }
                    fence_after();
                    const uint32_t base = smem_u32(stages + stage * STAGE_BYTES);
                    const uint32_t a1h = base, a1l = base + TILE_BYTES;
                    const uint32_t b1h = base + 2 * TILE_BYTES, b1l = base + 3 * TILE_BYTES;
                    const uint32_t a2h = diag ? b1h : base + 4 * TILE_BYTES;
                    const uint32_t a2l = diag ? b1l : base + 5 * TILE_BYTES;
                    const uint32_t b2h = diag ? a1h : base + 6 * TILE_BYTES;
                    const uint32_t b2l = diag ? a1l : base + 7 * TILE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {   // 32 bytes of k per MMA
                        const uint32_t off = kk * 32;
                        const uint32_t first = (kb | kk) ? 1u : 0u;
                        if constexpr (FMT == FMT_TF32) {
                            mma_tf32(d1, sdesc(a1h + off), sdesc(b1h + off), IDn, first);
                            mma_tf32(d1x, sdesc(a1h + off), sdesc(b1l + off), IDn, SEP ? first : 1u);
                            mma_tf32(d1x, sdesc(a1l + off), sdesc(b1h + off), IDn, 1u);
                            mma_tf32(d2, sdesc(a2h + off), sdesc(b2h + off), IDn, first);
                            mma_tf32(d2x, sdesc(a2h + off), sdesc(b2l + off), IDn, SEP ? first : 1u);
                            mma_tf32(d2x, sdesc(a2l + off), sdesc(b2h + off), IDn, 1u);
                        } else {
                            mma_f16(d1, sdesc(a1h + off), sdesc(b1h + off), IDn, first);
                            mma_f16(d1x, sdesc(a1h + off), sdesc(b1l + off), IDn, SEP ? first : 1u);
                            mma_f16(d1x, sdesc(a1l + off), sdesc(b1h + off), IDn, 1u);
                            mma_f16(d2, sdesc(a2h + off), sdesc(b2h + off), IDn, first);
                            mma_f16(d2x, sdesc(a2h + off), sdesc(b2l + off), IDn, SEP ? first : 1u);
                            mma_f16(d2x, sdesc(a2l + off), sdesc(b2h + off), IDn, 1u);
                        }
                    }
                    mma_commit(&empty[stage]);
                    if (++stage == NSTAGE) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
                if (++acc == NBUF) { acc = 0; aphase ^= 1u; }
            }
        }
    } else {
        // ---------------- epilogue (8 warps) ----------------
        const int ew = warp - 2;
        const int quad = warp & 3;     // TMEM lanes this warp may read
        const int half = ew >> 2;      // column half of the tile
        const int row = quad * 32 + lane;
        int acc = 0;
        uint32_t aphase = 0;
        // orbital energies as float pairs, from shared memory when they fit
        const float2* seps_or_null = nullptr;
        if (!BATCH && P.nmo <= EPS_SMEM) {
            for (int i = threadIdx.x - 64; i < P.nmo; i += 32 * NUM_EPI_WARPS) seps[i] = eps2[i];
            epi_bar();
            seps_or_null = seps;
        }
        for (int64_t kq = 0, item; (item = item_at(kq, nitems, order)) >= 0; ++kq) {
            const View v = CDS_VIEW(item);
            if (!v.act) continue;
            const TermR& tm = v.tm;
            const int nE = v.nE;
            const float inv = v.inv;
            const float2* epsv = seps_or_null ? seps_or_null : v.epsv;
            const bool bad = !mbar_wait(&tfull[acc], aphase, verr) || *verr;
            if (epi_any(bad)) break;
            fence_after();
            const int s = v.s, A = v.A, B = v.B;
            const bool diag = A == B;
            const int x = A * TB + row;
            const bool xok = x < tm.nx;
            const bool warp_live = A * TB + quad * 32 < tm.nx;   // any valid row in this warp
            // row part of the denominator, e_s - e_x, as a float pair
            const float2 es = epsv[tm.eps_s_off + s];
            const float2 ex = xok ? epsv[tm.eps_x_off + x] : make_float2(0.f, 0.f);
            const float2 rb = df_add(es, make_float2(-ex.x, -ex.y));
            const uint32_t ta1 = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)acc * 256u +
                                 (uint32_t)half * 64u;
            const uint32_t ta2 = ta1 + 128u;
            const int ybase = B * TB + half * 64;
            const int ncols = min(64, tm.nx - ybase);             // valid columns of this half
            const float2* Et = v.Et;
            const float2* ey2 = epsv + tm.eps_x_off;
            double* out = v.out;
            for (int e0 = 0; e0 < nE; e0 += EC) {
                const int ne = min(EC, nE - e0);
                // c = E + e_s - e_x as a float pair (hi, lo)
                float ch[EC], cl[EC], as[EC], ad[EC];
#pragma unroll
                for (int e = 0; e < EC; ++e) {
                    const float2 c = df_add(Et[min(e0 + e, nE - 1)], rb);
                    ch[e] = c.x;
                    cl[e] = c.y;
                    as[e] = 0.f;
                    ad[e] = 0.f;
                }
                if (warp_live) {
#pragma unroll 1
                    for (int cc = 0; cc < ncols; cc += 16) {
                        float x1[16], x2[16];
                        tmem_ld16(ta1 + cc, x1);
                        tmem_ld16(ta2 + cc, x2);
                        if constexpr (SEP) {
                            float y1[16], y2[16];
                            tmem_ld16(ta1 + 256u + cc, y1);
                            tmem_ld16(ta2 + 256u + cc, y2);
                            tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 16; ++j) { x1[j] += y1[j]; x2[j] += y2[j]; }
                        } else {
                            tmem_wait_ld();
                        }
                        float num[16], eh[16], el[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int y = ybase + cc + j;
                            const bool ok = xok && y < tm.nx;
                            const float a = x1[j] * inv, b = x2[j] * inv;
                            const float n = diag ? (2.f * a - b) * a : 2.f * (a * a + b * b - a * b);
                            num[j] = ok ? n : 0.f;
                            const float2 e2 = ok ? ey2[y] : make_float2(-1e30f, 0.f);  // padding: 0 * tiny
                            eh[j] = e2.x;
                            el[j] = e2.y;
                        }
                        if (cache && e0 == 0) {
                            // [item][half][column][row]: a warp writes 32 consecutive rows
                            // (item: the call's, or the batch's, running item index)
                            float* ct = cache + item * (int64_t)kCacheTile +
                                        ((int64_t)(half * 64 + cc) * TB + row);
#pragma unroll
                            for (int j = 0; j < 16; ++j) ct[(int64_t)j * TB] = num[j];
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
#pragma unroll
                            for (int e = 0; e < EC; ++e) {
                                const float d = (ch[e] - eh[j]) + (cl[e] - el[j]);
                                const float r = rcp_approx(d);
                                const float tt = num[j] * r;
                                as[e] += tt;
                                ad[e] = fmaf(-tt, r, ad[e]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < EC; ++e) {
#pragma unroll
                    for (int o = 16; o; o >>= 1) {
                        as[e] += __shfl_xor_sync(0xffffffffu, as[e], o);
                        ad[e] += __shfl_xor_sync(0xffffffffu, ad[e], o);
                    }
                }
                // per-warp partials of this energy chunk; the CTA-wide sum of a
                // group of RED_E energies needs one barrier pair
                const int g0 = e0 % RED_E;
                if (lane == 0) {
#pragma unroll
                    for (int e = 0; e < EC; ++e) {
                        if (e < ne) {
                            red[(ew * RED_E + g0 + e) * 2] = as[e];
                            red[(ew * RED_E + g0 + e) * 2 + 1] = ad[e];
                        }
                    }
                }
                if (g0 + EC >= RED_E || e0 + EC >= nE) {
                    epi_bar();
                    const int gstart = e0 - g0;
                    const int gn = min(RED_E, nE - gstart);
                    for (int idx = ew * 32 + lane; idx < gn; idx += 32 * NUM_EPI_WARPS) {
                        double sv = 0.0, dv = 0.0;
#pragma unroll
                        for (int w = 0; w < NUM_EPI_WARPS; ++w) {
                            sv += (double)red[(w * RED_E + idx) * 2];
                            dv += (double)red[(w * RED_E + idx) * 2 + 1];
                        }
                        out[(gstart + idx) * 2] = sv;
                        out[(gstart + idx) * 2 + 1] = dv;
                    }
                    epi_bar();
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
            if (++acc == NBUF) { acc = 0; aphase ^= 1u; }
            // completion time of the molecule's latest item (per-molecule latency)
            if (stamps && ew == 0 && lane == 0) atomicMax(stamps + v.mol, gtimer());
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
    }
#undef CDS_VIEW
}

// amax[0] = max |x| over n doubles (non-negative doubles order like their bits).
__global__ void k_absmax(const double* __restrict__ src, int64_t n, unsigned long long* amax) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(src[i]));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, (unsigned long long)__double_as_longlong(m));
}

// Power-of-two scale with max|s x| <= 1024 (1 for bf16 or an all-zero array).
__device__ __forceinline__ double split_scale(const unsigned long long* amax, bool bf16) {
    double m = __longlong_as_double((long long)*amax);
    if (bf16 || !(m > 0.0)) return 1.0;
    int ex;
    frexp(1024.0 / m, &ex);      // 1024/m = f 2^ex, f in [0.5, 1)
    return ldexp(1.0, ex - 1);
}

// hi = r(s x), lo = r(s x - hi) in bf16 or fp16; columns J >= M are zero.
template <typename T>
__global__ void k_split16(const double* __restrict__ src, int64_t rows, int32_t M, int32_t Mp,
                          const unsigned long long* __restrict__ amax, T* __restrict__ hi,
                          T* __restrict__ lo) {
    constexpr bool BF16 = std::is_same<T, __nv_bfloat16>::value;
    const double sc = split_scale(amax, BF16);
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * Mp) return;
    int64_t r = e / Mp;
    int J = (int)(e - r * Mp);
    double x = J < M ? src[r * M + J] * sc : 0.0;
    if constexpr (BF16) {
        __nv_bfloat16 h = __double2bfloat16(x);
        hi[e] = h;
        lo[e] = __double2bfloat16(x - (double)__bfloat162float(h));
    } else {
        __half h = __double2half(x);
        hi[e] = h;
        lo[e] = __double2half(x - (double)__half2float(h));
    }
}

// hi = tf32(x) (round to nearest on the 13 dropped bits), lo = fl32(x - hi);
// the MMA reads lo's top 19 bits.  No scaling (FP32 exponent range); columns
// J >= M are zero.
__global__ void k_split_tf32(const double* __restrict__ src, int64_t rows, int32_t M, int32_t Mp,
                             float* __restrict__ hi, float* __restrict__ lo) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * Mp) return;
    int64_t r = e / Mp;
    int J = (int)(e - r * Mp);
    const double x = J < M ? src[r * M + J] : 0.0;
    const float f = (float)x;
    const float h = __uint_as_float((__float_as_uint(f) + 0x1000u) & 0xFFFFE000u);
    hi[e] = h;
    lo[e] = (float)(x - (double)h);
}

// FP64 values as (hi, lo) float pairs: hi = fl32(x), lo = fl32(x - hi).
__global__ void k_to_pairs(const double* __restrict__ x, int64_t n, float2* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h = (float)x[i];
    out[i] = make_float2(h, (float)(x[i] - (double)h));
}

__global__ void k_inv_scale(const unsigned long long* __restrict__ amax, int bf16, float* inv) {
    double sa = split_scale(amax, bf16 != 0), sb = split_scale(amax + 1, bf16 != 0);
    *inv = (float)(1.0 / (sa * sb));
}

// sigma[t][e] from the per-item partials of both terms; NaN if a wait gave up.
__global__ void k_tc_reduce(const double* __restrict__ part, int64_t per_t0, int64_t off1,
                            int64_t per_t1, int32_t nE, const int32_t* __restrict__ active,
                            const int32_t* __restrict__ err, double* __restrict__ sigma,
                            double* __restrict__ dsigma) {
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
        if (*err) a = b = __longlong_as_double(0x7ff8000000000000LL);
        sigma[(int64_t)t * nE + e] = a;
        if (dsigma) dsigma[(int64_t)t * nE + e] = b;
    }
}

struct TcLayout {
    uint16_t *lp_hi, *lp_lo, *lov_hi, *lov_lo;   // bf16 or fp16 bit patterns (tf32: pairs of
                                                 // uint16 per 32-bit element)
    double* part;
    unsigned long long* amax;                    // [2]: max |Lp|, max |Lov|
    float* inv;                                  // 1 / (s_Lp s_Lov)
    float2* eps2;                                // orbital energies as float pairs
    float2* E2;                                  // energies as float pairs
    int32_t* err;
    size_t bytes;
};

inline int32_t padded(int32_t M) { return (M + KB - 1) / KB * KB; }

int64_t tc_items(int32_t nx, int32_t ns, int32_t np) {
    if (nx <= 0 || ns <= 0) return 0;
    return (int64_t)np * ns * npairs_of(nblocks_of(nx, TB));
}

TcLayout tc_layout(void* ws, int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE,
                   bool tf32 = false) {
    const int32_t Mp = padded(std::max(M, 1)), nv = nmo - nocc;
    const size_t w = tf32 ? 2 : 1;   // uint16 units per operand element
    Carver c(ws);
    TcLayout l;
    l.lp_hi = c.take<uint16_t>((size_t)np * nmo * Mp * w);
    l.lp_lo = c.take<uint16_t>((size_t)np * nmo * Mp * w);
    l.lov_hi = c.take<uint16_t>((size_t)nocc * nv * Mp * w);
    l.lov_lo = c.take<uint16_t>((size_t)nocc * nv * Mp * w);
    int64_t items = tc_items(nocc, nv, np) + tc_items(nv, nocc, np);
    l.part = c.take<double>((size_t)std::max<int64_t>(items, 1) * nE * 2);
    l.amax = c.take<unsigned long long>(2);
    l.inv = c.take<float>(2);
    l.eps2 = c.take<float2>((size_t)nmo);
    l.E2 = c.take<float2>((size_t)std::max(np, 1) * nE);
    l.err = c.take<int32_t>(4);
    l.bytes = c.off;
    return l;
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 3-D operand map {d0 (J, contiguous), d1, d2} with byte strides s1, s2, of
// format fmt (0 fp16, 1 bf16, 2 tf32 in FP32 containers); box {one 64-byte
// row of J, b1, b2}.
bool make_map(CUtensorMap* m, int fmt, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
              uint64_t s1, uint64_t s2, uint32_t b1, uint32_t b2) {
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {s1, s2};
    cuuint32_t box[3] = {(cuuint32_t)(fmt == FMT_TF32 ? KB / 2 : KB), b1, b2};
    cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt = fmt == FMT_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : fmt == 1      ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUresult r = enc(m, dt, 3,
                     const_cast<void*>(base), dims, strides,
                     box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Run-time kernel configuration chosen by the autotuner (cds_tune_set):
// energies per epilogue pass of the batched grid pass, and item order.
static std::atomic<int> g_energy_chunk{16};
static std::atomic<int> g_item_order{0};
static std::atomic<int> g_newton_cache{1};
static std::atomic<int> g_cd_graph{512};
static std::atomic<int> g_pipe_split{0};
static std::atomic<int> g_grid_ec{kGridEC};
int tune_grid_ec() { return g_grid_ec.load(); }
int tune_pipe_split() { return g_pipe_split.load(); }
int tune_energy_chunk() { return g_energy_chunk.load(); }
int tune_cd_graph() { return g_cd_graph.load(); }
int tune_item_order() { return g_item_order.load(); }
int tune_newton_cache() { return g_newton_cache.load(); }

// Separate hi.hi / cross accumulators (default) or the shared double-buffered
// form; CDS_TC_SHARED_ACC=1 selects the latter (for comparisons).
bool separate_accumulators() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("CDS_TC_SHARED_ACC");
        v = (e && e[0] == '1') ? 0 : 1;
    }
    return v == 1;
}

int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

bool device_ok() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3;
}

}  // namespace tc

size_t tc_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE,
                          bool tf32) {
    return tc::tc_layout(nullptr, nmo, nocc, M, np, nE, tf32).bytes;
}

namespace tc {
template <int EC, int FMT, bool SEP>
static int launch_tc(int grid, const Maps& maps, const Params& P, const int32_t* active,
                     const TcLayout& lay, cudaStream_t stream, float* cache) {
    CDS_CUDA_TRY(cudaFuncSetAttribute(k_sigma_tc<EC, FMT, SEP, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
    k_sigma_tc<EC, FMT, SEP, false><<<grid, THREADS, SMEM_BYTES, stream>>>(
        maps, P, nullptr, 0, 0, lay.E2, lay.eps2, active, lay.inv, lay.part, nullptr, lay.err,
        tune_item_order(), cache);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

template <bool SEP>
static int launch_any(int grid, int fmt, int nE, const Maps& maps, const Params& P,
                      const int32_t* active, const TcLayout& lay, cudaStream_t stream,
                      float* cache = nullptr) {
    if (nE == 1)
        return fmt == FMT_TF32 ? launch_tc<1, FMT_TF32, SEP>(grid, maps, P, active, lay, stream, cache)
               : fmt == 1      ? launch_tc<1, 1, SEP>(grid, maps, P, active, lay, stream, cache)
                               : launch_tc<1, 0, SEP>(grid, maps, P, active, lay, stream, cache);
    return fmt == FMT_TF32 ? launch_tc<16, FMT_TF32, SEP>(grid, maps, P, active, lay, stream, cache)
           : fmt == 1      ? launch_tc<16, 1, SEP>(grid, maps, P, active, lay, stream, cache)
                           : launch_tc<16, 0, SEP>(grid, maps, P, active, lay, stream, cache);
}

// TF32 operands: no scale (1 / (s_A s_B) = 1).
static int split_all_tf32(const double* Lp, const double* Lov, int64_t rows_p, int64_t rows_ov,
                          int32_t M, int32_t Mp, const TcLayout& lay, cudaStream_t stream) {
    CDS_CUDA_TRY(cudaMemsetAsync(lay.amax, 0, 2 * sizeof(unsigned long long), stream));
    const int64_t n1 = rows_p * Mp;
    k_split_tf32<<<(unsigned)((n1 + 255) / 256), 256, 0, stream>>>(
        Lp, rows_p, M, Mp, (float*)lay.lp_hi, (float*)lay.lp_lo);
    CDS_LAUNCH_CHECK();
    const int64_t n2 = rows_ov * Mp;
    if (n2 > 0) {
        k_split_tf32<<<(unsigned)((n2 + 255) / 256), 256, 0, stream>>>(
            Lov, rows_ov, M, Mp, (float*)lay.lov_hi, (float*)lay.lov_lo);
        CDS_LAUNCH_CHECK();
    }
    k_inv_scale<<<1, 1, 0, stream>>>(lay.amax, 1, lay.inv);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

template <typename T>
static int split_all(const double* Lp, const double* Lov, int64_t rows_p, int64_t rows_ov,
                     int32_t M, int32_t Mp, const TcLayout& lay, cudaStream_t stream) {
    constexpr bool BF16 = std::is_same<T, __nv_bfloat16>::value;
    CDS_CUDA_TRY(cudaMemsetAsync(lay.amax, 0, 2 * sizeof(unsigned long long), stream));
    if (!BF16) {
        k_absmax<<<4 * 152, 256, 0, stream>>>(Lp, rows_p * M, lay.amax);
        CDS_LAUNCH_CHECK();
        if (rows_ov > 0) {
            k_absmax<<<4 * 152, 256, 0, stream>>>(Lov, rows_ov * M, lay.amax + 1);
            CDS_LAUNCH_CHECK();
        }
    }
    int64_t n1 = rows_p * Mp;
    k_split16<T><<<(unsigned)((n1 + 255) / 256), 256, 0, stream>>>(
        Lp, rows_p, M, Mp, lay.amax, (T*)lay.lp_hi, (T*)lay.lp_lo);
    CDS_LAUNCH_CHECK();
    int64_t n2 = rows_ov * Mp;
    if (n2 > 0) {
        k_split16<T><<<(unsigned)((n2 + 255) / 256), 256, 0, stream>>>(
            Lov, rows_ov, M, Mp, lay.amax + 1, (T*)lay.lov_hi, (T*)lay.lov_lo);
        CDS_LAUNCH_CHECK();
    }
    k_inv_scale<<<1, 1, 0, stream>>>(lay.amax, BF16 ? 1 : 0, lay.inv);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}
}  // namespace tc

namespace tc {
// Work decomposition of Eq. SE's two sums (sigma.cuh) for the factor layout
// of cds_cd_to_mo; the same for every call with these sizes.
void build_terms(int32_t nmo, int32_t nocc, int32_t np, Params& P) {
    const int32_t nv = nmo - nocc;
    const int32_t nx[2] = {nocc, nv}, ns[2] = {nv, nocc};
    int64_t item0 = 0;
    for (int k = 0; k < 2; ++k) {
        Term& tm = P.term[k];
        tm.nx = nx[k];
        tm.ns = ns[k];
        tm.nb = nblocks_of(std::max(nx[k], 1), TB);
        tm.npb = npairs_of(tm.nb);
        tm.nitems = tc_items(nx[k], ns[k], np);
        tm.item0 = item0;
        item0 += tm.nitems;
        tm.bulk_s_dim = k == 0 ? 1 : 2;
        tm.eps_s_off = k == 0 ? nocc : 0;
        tm.eps_x_off = k == 0 ? 0 : nocc;
    }
    P.nmo = nmo;
}
}  // namespace tc

size_t tc_cache_bytes(int32_t nmo, int32_t nocc, int32_t np) {
    tc::Params P{};
    tc::build_terms(nmo, nocc, np, P);
    return (size_t)(P.term[0].nitems + P.term[1].nitems) * tc::kCacheTile * sizeof(float);
}

namespace tc {
template <int EC>
__global__ void __launch_bounds__(256)
k_sigma_cached_grid(Params P, const float* __restrict__ cache, const float2* __restrict__ E2,
                    const float2* __restrict__ eps2, const int32_t* __restrict__ active,
                    double* __restrict__ part, int32_t nE, int32_t e_begin);
}  // namespace tc

int sigma2_tc(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
              int32_t np, const double* eps, const double* E, int32_t nE,
              const int32_t* active, int32_t precision, double* sigma, double* dsigma, void* ws,
              cudaStream_t stream, bool resplit, float* cache) {
    using namespace tc;
    if (!device_ok()) return CDS_ERR_UNSUPPORTED;
    const int fmt = precision == CDS_PREC_TF32X3 ? FMT_TF32 : precision == CDS_PREC_BF16X3 ? 1 : 0;
    const int32_t nv = nmo - nocc;
    const int32_t Mp = padded(std::max(M, 1));
    TcLayout lay = tc_layout(ws, nmo, nocc, M, np, nE, fmt == FMT_TF32);
    int st = CDS_OK;
    if (resplit)
        st = fmt == FMT_TF32
                 ? split_all_tf32(Lp, Lov, (int64_t)np * nmo, (int64_t)nocc * nv, M, Mp, lay, stream)
             : fmt == 1 ? split_all<__nv_bfloat16>(Lp, Lov, (int64_t)np * nmo, (int64_t)nocc * nv, M,
                                                   Mp, lay, stream)
                        : split_all<__half>(Lp, Lov, (int64_t)np * nmo, (int64_t)nocc * nv, M, Mp,
                                            lay, stream);
    if (st) return st;
    Params P{};
    Maps maps;
    memset(&maps, 0, sizeof(maps));
    const uint64_t ebytes = fmt == FMT_TF32 ? 4 : 2;
    const uint64_t rowb = (uint64_t)Mp * ebytes;
    // term 0 (first sum of Eq. SE): x = occupied rows of Lp, bulk L^J_{a j}
    // read from Lov[j][a] with spectator a as map dim 1 and y = j as dim 2.
    // term 1 (second sum): x = virtual rows of Lp, bulk Lov[i][b], spectator i dim 2.
    const int32_t nx[2] = {nocc, nv};
    build_terms(nmo, nocc, np, P);
    for (int k = 0; k < 2; ++k) {
        if (P.term[k].nitems == 0) continue;
        const char* qb_hi = (const char*)lay.lp_hi + (k == 0 ? 0 : (size_t)nocc * rowb);
        const char* qb_lo = (const char*)lay.lp_lo + (k == 0 ? 0 : (size_t)nocc * rowb);
        bool ok = make_map(&maps.m[k][0], fmt, qb_hi, Mp, nx[k], np, rowb, rowb * nmo, TB, 1) &&
                  make_map(&maps.m[k][1], fmt, qb_lo, Mp, nx[k], np, rowb, rowb * nmo, TB, 1) &&
                  make_map(&maps.m[k][2], fmt, lay.lov_hi, Mp, nv, nocc, rowb, rowb * nv,
                           k == 0 ? 1 : TB, k == 0 ? TB : 1) &&
                  make_map(&maps.m[k][3], fmt, lay.lov_lo, Mp, nv, nocc, rowb, rowb * nv,
                           k == 0 ? 1 : TB, k == 0 ? TB : 1);
        if (!ok) return CDS_ERR_CUDA;
    }
    P.kblocks = fmt == FMT_TF32 ? Mp / (KB / 2) : Mp / KB;
    P.nE = nE;
    P.nmo = nmo;
    const int64_t nitems = P.term[0].nitems + P.term[1].nitems;
    CDS_CUDA_TRY(cudaMemsetAsync(lay.err, 0, sizeof(int32_t), stream));
    if (nitems > 0) {
        k_to_pairs<<<(nmo + 255) / 256, 256, 0, stream>>>(eps, nmo, lay.eps2);
        CDS_LAUNCH_CHECK();
        k_to_pairs<<<(unsigned)(((int64_t)np * nE + 255) / 256), 256, 0, stream>>>(E, (int64_t)np * nE,
                                                                                 lay.E2);
        CDS_LAUNCH_CHECK();
        int grid = (int)std::min<int64_t>(nitems, device_sms());
        // with the numerators kept, the tensor-core epilogue evaluates the
        // first kGridSplitE energies and k_sigma_cached_grid the rest, at
        // the occupancy the epilogue warps of the tensor-core kernel lack
        // (C60 shape, 20 orbitals x 64 energies: 43.6 ms against 52.6 ms
        // with all energies in the epilogue)
        const bool split = cache && nE > kGridSplitE;
        if (split) P.nE_eval = kGridSplitE;
        const int nE_tc = split ? kGridSplitE : nE;   // picks the epilogue's energy chunk
        st = separate_accumulators()
                 ? launch_any<true>(grid, fmt, nE_tc, maps, P, active, lay, stream, cache)
                 : launch_any<false>(grid, fmt, nE_tc, maps, P, active, lay, stream, cache);
        if (st) return st;
        if (split) {
            const int g2 = (int)std::min<int64_t>(nitems, (int64_t)device_sms() * 4);
            // energies per pass: the autotuner's choice (CDS_TUNE_GRID_EC)
            const int ec = tune_grid_ec();
            if (ec == 2)
                k_sigma_cached_grid<2><<<g2, 256, 0, stream>>>(P, cache, lay.E2, lay.eps2, active,
                                                               lay.part, nE, kGridSplitE);
            else if (ec == 8)
                k_sigma_cached_grid<8><<<g2, 256, 0, stream>>>(P, cache, lay.E2, lay.eps2, active,
                                                               lay.part, nE, kGridSplitE);
            else
                k_sigma_cached_grid<kGridEC><<<g2, 256, 0, stream>>>(P, cache, lay.E2, lay.eps2,
                                                                     active, lay.part, nE,
                                                                     kGridSplitE);
            CDS_LAUNCH_CHECK();
        }
    } else {
        CDS_CUDA_TRY(cudaMemsetAsync(lay.part, 0, sizeof(double) * 2 * nE, stream));
    }
    const int64_t per0 = np ? P.term[0].nitems / np : 0, per1 = np ? P.term[1].nitems / np : 0;
    dim3 grid(nE, np);
    k_tc_reduce<<<grid, 256, 0, stream>>>(lay.part, per0, P.term[0].nitems, per1, nE, active,
                                         lay.err, sigma, dsigma);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}


// ===========================================================================
// Cached numerators.  The numerator n_xy of every element of every work item
// is independent of the energy, so Sigma(E) at any E is the sum of n_xy over
// the float-pair denominators E + e_s - e_x - e_y alone.  sigma2_tc with a
// cache stores each item's numerators ([half][column][row] floats, written by
// the epilogue of its first energy chunk); k_sigma_cached then evaluates
// Sigma and dSigma/dE at one energy per orbital from them, with the same
// per-element arithmetic as the tensor-core epilogue, streaming 64 KB per item
// instead of recomputing the integrals.
// ===========================================================================
namespace tc {
__global__ void __launch_bounds__(256)
k_sigma_cached(Params P, const float* __restrict__ cache, const float2* __restrict__ E2,
               const float2* __restrict__ eps2, const int32_t* __restrict__ active,
               double* __restrict__ part) {
    // the warps' sums of up to kItems items wait in shared memory and are
    // added over the block (fixed order) at one barrier pair per kItems items
    constexpr int kItems = 16;
    __shared__ float red[kItems][8][2];
    __shared__ int64_t slot_pidx[kItems];
    int nslot = 0;
    const int64_t nitems = P.term[0].nitems + P.term[1].nitems;
    const int row = threadIdx.x & (TB - 1), half = threadIdx.x / TB;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    auto flush = [&]() {
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * nslot; i += blockDim.x) {
            const int sl = i >> 1, k = i & 1;
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < 8; ++j) v += (double)red[sl][j][k];
            part[slot_pidx[sl] * 2 + k] = v;
        }
        __syncthreads();
        nslot = 0;
    };
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        int term, t, s, A, B;
        const TermR tm = decode(P.term[0], P.term[1], item, term, t, s, A, B);
        if (active && !active[t]) continue;   // the same for the whole block
        const int x = A * TB + row;
        const int ybase = B * TB + half * 64;
        const int ncols = min(64, tm.nx - ybase);
        const int64_t pidx = tm.item0 + (item - tm.first);
        float as = 0.f, ad = 0.f;
        if (x < tm.nx && ncols > 0) {
            const float2 es = eps2[tm.eps_s_off + s];
            const float2 ex = eps2[tm.eps_x_off + x];
            const float2 c = df_add(E2[t], df_add(es, make_float2(-ex.x, -ex.y)));
            const float* ct = cache + pidx * kCacheTile + (int64_t)half * 64 * TB + row;
            const float2* ey2 = eps2 + tm.eps_x_off + ybase;
            // all 64 numerators in flight before the sums (the same order of sums)
            float num[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) num[j] = j < ncols ? ct[(int64_t)j * TB] : 0.f;
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                if (j < ncols) {
                    const float2 e2 = ey2[j];
                    const float d = (c.x - e2.x) + (c.y - e2.y);
                    const float r = rcp_approx(d);
                    const float tt = num[j] * r;
                    as += tt;
                    ad = fmaf(-tt, r, ad);
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            as += __shfl_xor_sync(0xffffffffu, as, o);
            ad += __shfl_xor_sync(0xffffffffu, ad, o);
        }
        if (lane == 0) { red[nslot][w][0] = as; red[nslot][w][1] = ad; }
        if (threadIdx.x == 0) slot_pidx[nslot] = pidx;
        if (++nslot == kItems) flush();
    }
    if (nslot > 0) flush();
}

// Sigma and dSigma/dE of one work item at energies [e_begin, nE) of its
// orbital from its cached numerators ct (the grid's energies past the ones
// the tensor-core epilogue evaluates).  Thread = (row, column half) as in
// k_sigma_cached, its 64 numerators held in registers across the energies;
// EC energies per pass, each summed over its warp; the warps' sums wait in
// shared memory for up to kRedE energies and are then added over the block
// in a fixed order into out[e][2] (the partial row of the item, the layout
// of k_sigma_tc), so the block meets at a barrier once per kRedE energies
// instead of twice per pass.
// Et: the orbital's energies; ev: the molecule's orbital energies.
template <int EC>
__device__ __forceinline__ void cached_grid_item(const TermR& tm, int t, int s, int A, int B,
                                                 const float* __restrict__ ct_item,
                                                 const float2* __restrict__ Et,
                                                 const float2* __restrict__ ev, int32_t nE,
                                                 int32_t e_begin, double* __restrict__ out) {
    constexpr int kRedE = 64;   // a multiple of every EC
    static_assert(kRedE % EC == 0, "energy chunk");
    __shared__ float red[8][kRedE][2];
    __shared__ float2 sey[2][64];
    (void)t;
    const int row = threadIdx.x & (TB - 1), half = threadIdx.x / TB;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = A * TB + row;
    const int ybase = B * TB + half * 64;
    const int ncols = min(64, tm.nx - ybase);
    const bool xok = x < tm.nx && ncols > 0;
    float num[64];
    const float* ct = ct_item + (int64_t)half * 64 * TB + row;
#pragma unroll
    for (int j = 0; j < 64; ++j) num[j] = (xok && j < ncols) ? ct[(int64_t)j * TB] : 0.f;
    // the previous item's reads of sey ended before its last flush's barriers
    if (row < 64)      // padding columns: a far-off energy, so 0 * tiny
        sey[half][row] = row < ncols ? ev[tm.eps_x_off + ybase + row] : make_float2(-1e30f, 0.f);
    __syncthreads();
    float2 rb = make_float2(0.f, 0.f);
    if (xok) {
        const float2 es = ev[tm.eps_s_off + s];
        const float2 ex = ev[tm.eps_x_off + x];
        rb = df_add(es, make_float2(-ex.x, -ex.y));
    }
    int fbase = e_begin;   // first energy of the chunk in red
    for (int e0 = e_begin; e0 < nE; e0 += EC) {
        float ch[EC], cl[EC], as[EC], ad[EC];
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const float2 c = df_add(Et[min(e0 + e, nE - 1)], rb);
            ch[e] = c.x;
            cl[e] = c.y;
            as[e] = 0.f;
            ad[e] = 0.f;
        }
        if (xok) {
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const float2 e2 = sey[half][j];
#pragma unroll
                for (int e = 0; e < EC; ++e) {
                    const float d = (ch[e] - e2.x) + (cl[e] - e2.y);
                    const float r = rcp_approx(d);
                    const float tt = num[j] * r;
                    as[e] += tt;
                    ad[e] = fmaf(-tt, r, ad[e]);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < EC; ++e) {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                as[e] += __shfl_xor_sync(0xffffffffu, as[e], o);
                ad[e] += __shfl_xor_sync(0xffffffffu, ad[e], o);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int e = 0; e < EC; ++e) {
                red[w][e0 - fbase + e][0] = as[e];
                red[w][e0 - fbase + e][1] = ad[e];
            }
        }
        if (e0 + EC - fbase >= kRedE || e0 + EC >= nE) {   // the chunk is full or done
            __syncthreads();
            const int cnt = min(nE, e0 + EC) - fbase;
            for (int i = threadIdx.x; i < 2 * cnt; i += blockDim.x) {
                const int e = i >> 1, k = i & 1;
                double v = 0.0;
#pragma unroll
                for (int j = 0; j < 8; ++j) v += (double)red[j][e][k];
                out[(int64_t)(fbase + e) * 2 + k] = v;
            }
            __syncthreads();
            fbase = e0 + EC;
        }
    }
}

template <int EC>
__global__ void __launch_bounds__(256)
k_sigma_cached_grid(Params P, const float* __restrict__ cache, const float2* __restrict__ E2,
                    const float2* __restrict__ eps2, const int32_t* __restrict__ active,
                    double* __restrict__ part, int32_t nE, int32_t e_begin) {
    const int64_t nitems = P.term[0].nitems + P.term[1].nitems;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        int term, t, s, A, B;
        const TermR tm = decode(P.term[0], P.term[1], item, term, t, s, A, B);
        if (active && !active[t]) continue;   // the same for the whole block
        const int64_t pidx = tm.item0 + (item - tm.first);
        cached_grid_item<EC>(tm, t, s, A, B, cache + pidx * kCacheTile, E2 + (int64_t)t * nE, eps2,
                             nE, e_begin, part + pidx * (int64_t)nE * 2);
    }
}

// The same over a batch of molecules (the grid pass of tc_batch_pass).
template <int EC>
__global__ void __launch_bounds__(256)
k_sigma_cached_grid_batch(const MolDesc* __restrict__ mols, int32_t nmol, int64_t nitems,
                          const float* __restrict__ cache, const float2* __restrict__ E2,
                          const float2* __restrict__ eps2, double* __restrict__ part,
                          int32_t e_begin) {
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        int lo = 0, hi = nmol - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (mols[mid].item_begin <= item) lo = mid; else hi = mid - 1;
        }
        const MolDesc* md = mols + lo;
        const int64_t r = item - md->item_begin;
        int term, t, s, A, B;
        const TermR tm = decode(md->term[0], md->term[1], r, term, t, s, A, B);
        cached_grid_item<EC>(tm, t, s, A, B, cache + item * kCacheTile,
                             E2 + md->E_off + (int64_t)t * md->nE, eps2 + md->eps_off, md->nE,
                             e_begin, part + md->part_base + r * (int64_t)md->nE * 2);
    }
}

struct CachedLayout {
    double* part;
    float2* E2;
    float2* eps2;
    int32_t* err;
    size_t bytes;
};

CachedLayout cached_layout(void* ws, int32_t nmo, int32_t nocc, int32_t np) {
    Params P{};
    build_terms(nmo, nocc, np, P);
    Carver c(ws);
    CachedLayout l;
    l.part = c.take<double>((size_t)std::max<int64_t>(P.term[0].nitems + P.term[1].nitems, 1) * 2);
    l.E2 = c.take<float2>((size_t)std::max(np, 1));
    l.eps2 = c.take<float2>((size_t)nmo);
    l.err = c.take<int32_t>(4);
    l.bytes = c.off;
    return l;
}
}  // namespace tc

size_t tc_cached_workspace_bytes(int32_t nmo, int32_t nocc, int32_t np) {
    return tc::cached_layout(nullptr, nmo, nocc, np).bytes;
}

int sigma2_cached(int32_t nmo, int32_t nocc, int32_t np, const double* eps, const double* E,
                  const int32_t* active, const float* cache, double* sigma, double* dsigma,
                  void* ws, cudaStream_t stream, bool first) {
    using namespace tc;
    Params P{};
    build_terms(nmo, nocc, np, P);
    P.nE = 1;
    CachedLayout lay = cached_layout(ws, nmo, nocc, np);
    const int64_t nitems = P.term[0].nitems + P.term[1].nitems;
    if (first) {
        CDS_CUDA_TRY(cudaMemsetAsync(lay.err, 0, sizeof(int32_t), stream));
        k_to_pairs<<<(nmo + 255) / 256, 256, 0, stream>>>(eps, nmo, lay.eps2);
        CDS_LAUNCH_CHECK();
    }
    if (nitems == 0) {
        CDS_CUDA_TRY(cudaMemsetAsync(lay.part, 0, sizeof(double) * 2, stream));
    } else {
        k_to_pairs<<<(np + 255) / 256, 256, 0, stream>>>(E, np, lay.E2);
        CDS_LAUNCH_CHECK();
        const int grid = (int)std::min<int64_t>(nitems, 8LL * device_sms());
        k_sigma_cached<<<grid, 256, 0, stream>>>(P, cache, lay.E2, lay.eps2, active, lay.part);
        CDS_LAUNCH_CHECK();
    }
    const int64_t per0 = np ? P.term[0].nitems / np : 0, per1 = np ? P.term[1].nitems / np : 0;
    k_tc_reduce<<<dim3(1, np), 256, 0, stream>>>(lay.part, per0, P.term[0].nitems, per1, 1, active,
                                                lay.err, sigma, dsigma);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

// ===========================================================================
// MP2 correlation energy (Eq. MP2) on the same kernel.  For occupied i, j the
// sum over a, b is the second sum of Eq. SE with orbital q := i, spectator
// j and E := e_i, and both operands are rows of Lov: the orbital tiles come
// from Lov[i], the spectator tiles from Lov[j].  So the item list is term 1
// only, with nocc "orbitals", and the per-orbital totals are the per-i sums
// e_i = sum_{j,a,b}.
// ===========================================================================
namespace tc {
struct Mp2Layout {
    TcLayout tc;      // lp_hi / lp_lo unused
    double* epair;    // [nocc] when the caller passes none
    size_t bytes;
};

Mp2Layout mp2_layout(void* ws, int32_t nmo, int32_t nocc, int32_t M) {
    const int32_t Mp = padded(std::max(M, 1)), nv = nmo - nocc;
    Carver c(ws);
    Mp2Layout l;
    l.tc.lp_hi = l.tc.lp_lo = nullptr;
    l.tc.lov_hi = c.take<uint16_t>((size_t)nocc * nv * Mp);
    l.tc.lov_lo = c.take<uint16_t>((size_t)nocc * nv * Mp);
    l.tc.part = c.take<double>((size_t)std::max<int64_t>(tc_items(nv, nocc, nocc), 1) * 2);
    l.tc.amax = c.take<unsigned long long>(2);
    l.tc.inv = c.take<float>(2);
    l.tc.eps2 = c.take<float2>((size_t)nmo);
    l.tc.E2 = c.take<float2>((size_t)std::max(nocc, 1));
    l.tc.err = c.take<int32_t>(4);
    l.epair = c.take<double>((size_t)std::max(nocc, 1));
    l.tc.bytes = l.bytes = c.off;
    return l;
}
}  // namespace tc

size_t tc_mp2_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M) {
    return tc::mp2_layout(nullptr, nmo, nocc, M).bytes;
}

int mp2_tc(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* eps,
           int32_t precision, double* e_pair, double* e_total, void* ws, cudaStream_t stream) {
    using namespace tc;
    if (!device_ok()) return CDS_ERR_UNSUPPORTED;
    const bool bf16 = precision == CDS_PREC_BF16X3;
    const int32_t nv = nmo - nocc;
    const int32_t Mp = padded(std::max(M, 1));
    Mp2Layout ml = mp2_layout(ws, nmo, nocc, M);
    const TcLayout& lay = ml.tc;
    double* ep = e_pair ? e_pair : ml.epair;
    const int64_t nitems = tc_items(nv, nocc, nocc);
    if (nitems == 0 || M == 0) {
        CDS_CUDA_TRY(cudaMemsetAsync(ep, 0, sizeof(double) * std::max(nocc, 1), stream));
        return sum_fixed(ep, nocc, e_total, stream);
    }
    // one array feeds both operands: one scale, inv = 1 / s^2
    CDS_CUDA_TRY(cudaMemsetAsync(lay.amax, 0, 2 * sizeof(unsigned long long), stream));
    const int64_t rows = (int64_t)nocc * nv, n = rows * Mp;
    if (!bf16) {
        k_absmax<<<4 * 152, 256, 0, stream>>>(Lov, rows * M, lay.amax);
        CDS_LAUNCH_CHECK();
        CDS_CUDA_TRY(cudaMemcpyAsync(lay.amax + 1, lay.amax, sizeof(unsigned long long),
                                     cudaMemcpyDeviceToDevice, stream));
        k_split16<__half><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(
            Lov, rows, M, Mp, lay.amax, (__half*)lay.lov_hi, (__half*)lay.lov_lo);
    } else {
        k_split16<__nv_bfloat16><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(
            Lov, rows, M, Mp, lay.amax, (__nv_bfloat16*)lay.lov_hi, (__nv_bfloat16*)lay.lov_lo);
    }
    CDS_LAUNCH_CHECK();
    k_inv_scale<<<1, 1, 0, stream>>>(lay.amax, bf16 ? 1 : 0, lay.inv);
    CDS_LAUNCH_CHECK();
    Params P{};
    Maps maps;
    memset(&maps, 0, sizeof(maps));
    const uint64_t rowb = (uint64_t)Mp * 2;
    Term& tm = P.term[1];
    tm.nx = nv;
    tm.ns = nocc;
    tm.nb = nblocks_of(nv, TB);
    tm.npb = npairs_of(tm.nb);
    tm.nitems = nitems;
    tm.item0 = 0;
    tm.bulk_s_dim = 2;
    tm.eps_s_off = 0;
    tm.eps_x_off = nocc;
    // orbital tiles Lov[i][A-block], spectator tiles Lov[j][B-block]: the same map
    if (!make_map(&maps.m[1][0], bf16, lay.lov_hi, Mp, nv, nocc, rowb, rowb * nv, TB, 1) ||
        !make_map(&maps.m[1][1], bf16, lay.lov_lo, Mp, nv, nocc, rowb, rowb * nv, TB, 1))
        return CDS_ERR_CUDA;
    maps.m[1][2] = maps.m[1][0];
    maps.m[1][3] = maps.m[1][1];
    P.kblocks = Mp / KB;
    P.nE = 1;
    P.nmo = nmo;
    CDS_CUDA_TRY(cudaMemsetAsync(lay.err, 0, sizeof(int32_t), stream));
    k_to_pairs<<<(nmo + 255) / 256, 256, 0, stream>>>(eps, nmo, lay.eps2);
    CDS_LAUNCH_CHECK();
    k_to_pairs<<<(nocc + 255) / 256, 256, 0, stream>>>(eps, nocc, lay.E2);   // E_i = e_i
    CDS_LAUNCH_CHECK();
    const int grid = (int)std::min<int64_t>(nitems, device_sms());
    int st = separate_accumulators() ? launch_any<true>(grid, bf16, 1, maps, P, nullptr, lay, stream)
                                     : launch_any<false>(grid, bf16, 1, maps, P, nullptr, lay, stream);
    if (st) return st;
    k_tc_reduce<<<dim3(1, nocc), 256, 0, stream>>>(lay.part, 0, 0, nitems / nocc, 1, nullptr,
                                                  lay.err, ep, nullptr);
    CDS_LAUNCH_CHECK();
    return sum_fixed(ep, nocc, e_total, stream);
}

// ===========================================================================
// Batched form: the items of many molecules in one persistent launch.
// ===========================================================================
namespace tc {

// Per-orbital reduction record of a batch (one per solved orbital).
struct OrbRed {
    int64_t base0, per0;     // element offset and count of the orbital's first-sum rows
    int64_t base1, per1;     // and second-sum rows (rows are nE * 2 doubles)
    int64_t out_off;         // sigma/dsigma offset of (orbital, energy 0)
    int32_t nE, act_idx;
};

__global__ void k_tc_reduce_batch(const double* __restrict__ part, const OrbRed* __restrict__ orbs,
                                  const int32_t* __restrict__ active,
                                  const int32_t* __restrict__ err, double* __restrict__ sigma,
                                  double* __restrict__ dsigma) {
    const OrbRed o = orbs[blockIdx.y];
    const int e = blockIdx.x;
    if (e >= o.nE || (active && !active[o.act_idx])) return;
    double sv = 0.0, dv = 0.0;
    for (int64_t i = threadIdx.x; i < o.per0 + o.per1; i += blockDim.x) {
        const int64_t at = (i < o.per0 ? o.base0 + i * o.nE * 2 : o.base1 + (i - o.per0) * o.nE * 2) + e * 2;
        sv += part[at];
        dv += part[at + 1];
    }
    __shared__ double ss[32], sd[32];
    for (int off = 16; off; off >>= 1) {
        sv += __shfl_xor_sync(0xffffffffu, sv, off);
        dv += __shfl_xor_sync(0xffffffffu, dv, off);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { ss[w] = sv; sd[w] = dv; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += ss[i]; b += sd[i]; }
        if (*err) a = b = __longlong_as_double(0x7ff8000000000000LL);
        sigma[o.out_off + e] = a;
        if (dsigma) dsigma[o.out_off + e] = b;
    }
}

// 1/(s_A s_B) of molecule c into both descriptor sets.
__global__ void k_inv_scale_batch(const unsigned long long* __restrict__ amax, int bf16, int nmol,
                                  MolDesc* grid_set, MolDesc* newton_set) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nmol) return;
    double sa = split_scale(amax + 2 * c, bf16 != 0), sb = split_scale(amax + 2 * c + 1, bf16 != 0);
    float inv = (float)(1.0 / (sa * sb));
    grid_set[c].inv = inv;
    newton_set[c].inv = inv;
}

struct BatchLayout {
    MolDesc* grid_set;
    MolDesc* newton_set;
    OrbRed* grid_red;
    OrbRed* newton_red;
    uint16_t *hi, *lo;          // split operands of all molecules
    double* part;
    unsigned long long* amax;   // [nmol][2]
    float2* eps2;               // [sum nbf]
    float2* E2;                 // [sum np*nE]
    float2* w2;                 // [sum np]  (Newton energies)
    int32_t* err;
    float* cache;               // [items][kCacheTile] numerators of the grid pass
    size_t bytes;
    int64_t grid_items, newton_items;
};

static int64_t mol_items(const BatchMol& b) {
    return tc_items(b.nocc, b.nbf - b.nocc, b.np) + tc_items(b.nbf - b.nocc, b.nocc, b.np);
}

static BatchLayout batch_layout(void* ws, int32_t nmol, const BatchMol* mols) {
    int64_t split = 0, nbf_all = 0, E_all = 0, np_all = 0, part_rows = 0, part_elems = 0;
    for (int c = 0; c < nmol; ++c) {
        const BatchMol& b = mols[c];
        const int64_t Mp = padded(std::max(b.max_rank, 1));
        split += ((int64_t)b.np * b.nbf + (int64_t)b.nocc * (b.nbf - b.nocc)) * Mp;
        nbf_all += b.nbf;
        E_all += (int64_t)b.np * b.nE;
        np_all += b.np;
        const int64_t it = mol_items(b);
        part_rows += it;
        part_elems += it * std::max(b.nE, 1) * 2;
    }
    Carver c(ws);
    BatchLayout l;
    l.grid_set = c.take<MolDesc>(std::max(nmol, 1));
    l.newton_set = c.take<MolDesc>(std::max(nmol, 1));
    l.grid_red = c.take<OrbRed>(std::max<int64_t>(np_all, 1));
    l.newton_red = c.take<OrbRed>(std::max<int64_t>(np_all, 1));
    l.hi = c.take<uint16_t>(std::max<int64_t>(split, 1));
    l.lo = c.take<uint16_t>(std::max<int64_t>(split, 1));
    l.part = c.take<double>(std::max<int64_t>(part_elems, 2));
    l.amax = c.take<unsigned long long>(2 * std::max(nmol, 1));
    l.eps2 = c.take<float2>(std::max<int64_t>(nbf_all, 1));
    l.E2 = c.take<float2>(std::max<int64_t>(E_all, 1));
    l.w2 = c.take<float2>(std::max<int64_t>(np_all, 1));
    l.err = c.take<int32_t>(4);
    l.cache = c.take<float>((size_t)std::max<int64_t>(part_rows, 1) * kCacheTile);
    l.bytes = c.off;
    l.grid_items = part_rows;
    l.newton_items = part_rows;
    return l;
}

}  // namespace tc

size_t tc_batch_workspace_bytes(int32_t nmol, const BatchMol* mols) {
    return tc::batch_layout(nullptr, nmol, mols).bytes;
}

// Host part: tensor maps, descriptors and reduction records of both passes
// (the 64-energy grid and the one-energy Newton pass), copied to the device
// once; blocking (the records live in host memory until the copy is done).
int tc_batch_setup(int32_t nmol, const BatchMol* mols, const int32_t* M, int32_t precision,
                   void* ws, cudaStream_t stream) {
    using namespace tc;
    if (!device_ok()) return CDS_ERR_UNSUPPORTED;
    const bool bf16 = precision == CDS_PREC_BF16X3;
    BatchLayout lay = batch_layout(ws, nmol, mols);
    std::vector<MolDesc> grid(nmol), newton(nmol);
    std::vector<OrbRed> gred, nred;
    int64_t split_off = 0, eps_off = 0, E_off = 0, w_off = 0, item_begin = 0, part_grid = 0,
            part_newton = 0, out_grid = 0;
    for (int c = 0; c < nmol; ++c) {
        const BatchMol& b = mols[c];
        const int32_t nbf = b.nbf, nocc = b.nocc, nv = nbf - nocc, np = b.np;
        const int32_t Mp_cap = padded(std::max(b.max_rank, 1));
        const int32_t Mp = padded(std::max(M[c], 1));
        if (M[c] > b.max_rank) return CDS_ERR_ARG;
        const uint16_t* lp_hi = lay.hi + split_off;
        const uint16_t* lp_lo = lay.lo + split_off;
        const uint16_t* ov_hi = lp_hi + (int64_t)np * nbf * Mp_cap;
        const uint16_t* ov_lo = lp_lo + (int64_t)np * nbf * Mp_cap;
        MolDesc d;
        memset(&d, 0, sizeof(d));
        const uint64_t rowb = (uint64_t)Mp * 2;   // rows are packed at the actual Mp
        const int32_t nx[2] = {nocc, nv}, ns[2] = {nv, nocc};
        int64_t it0 = 0;
        for (int k = 0; k < 2; ++k) {
            Term& tm = d.term[k];
            tm.nx = nx[k];
            tm.ns = ns[k];
            tm.nb = nblocks_of(std::max(nx[k], 1), TB);
            tm.npb = npairs_of(tm.nb);
            tm.nitems = tc_items(nx[k], ns[k], np);
            tm.item0 = it0;
            it0 += tm.nitems;
            tm.bulk_s_dim = k == 0 ? 1 : 2;
            tm.eps_s_off = k == 0 ? nocc : 0;
            tm.eps_x_off = k == 0 ? 0 : nocc;
            if (tm.nitems == 0) continue;
            const uint16_t* qh = lp_hi + (k == 0 ? 0 : (size_t)nocc * Mp);
            const uint16_t* ql = lp_lo + (k == 0 ? 0 : (size_t)nocc * Mp);
            bool ok = make_map(&d.m[k][0], bf16, qh, Mp, nx[k], np, rowb, rowb * nbf, TB, 1) &&
                      make_map(&d.m[k][1], bf16, ql, Mp, nx[k], np, rowb, rowb * nbf, TB, 1) &&
                      make_map(&d.m[k][2], bf16, ov_hi, Mp, nv, nocc, rowb, rowb * nv,
                               k == 0 ? 1 : TB, k == 0 ? TB : 1) &&
                      make_map(&d.m[k][3], bf16, ov_lo, Mp, nv, nocc, rowb, rowb * nv,
                               k == 0 ? 1 : TB, k == 0 ? TB : 1);
            if (!ok) return CDS_ERR_CUDA;
        }
        d.kblocks = Mp / KB;
        d.nmo = nbf;
        d.eps_off = eps_off;
        d.act_off = (int32_t)w_off;
        d.inv = 1.f;
        d.item_begin = item_begin;
        MolDesc g = d, n = d;
        g.nE = b.nE;
        g.E_off = E_off;
        g.part_base = part_grid;
        n.nE = 1;
        n.E_off = w_off;
        n.part_base = part_newton;
        grid[c] = g;
        newton[c] = n;
        const int64_t per0 = np ? d.term[0].nitems / np : 0, per1 = np ? d.term[1].nitems / np : 0;
        for (int t = 0; t < np; ++t) {
            OrbRed r;
            r.per0 = per0;
            r.per1 = per1;
            r.base0 = part_grid + t * per0 * b.nE * 2;
            r.base1 = part_grid + (d.term[0].nitems + t * per1) * b.nE * 2;
            r.nE = b.nE;
            r.out_off = out_grid + (int64_t)t * b.nE;
            r.act_idx = (int32_t)(w_off + t);
            gred.push_back(r);
            r.base0 = part_newton + t * per0 * 2;
            r.base1 = part_newton + (d.term[0].nitems + t * per1) * 2;
            r.nE = 1;
            r.out_off = w_off + t;
            nred.push_back(r);
        }
        const int64_t items = d.term[0].nitems + d.term[1].nitems;
        item_begin += items;
        part_grid += items * b.nE * 2;
        part_newton += items * 2;
        split_off += ((int64_t)np * nbf + (int64_t)nocc * nv) * Mp_cap;
        eps_off += nbf;
        E_off += (int64_t)np * b.nE;
        out_grid += (int64_t)np * b.nE;
        w_off += np;
    }
    CDS_CUDA_TRY(cudaMemcpyAsync(lay.grid_set, grid.data(), sizeof(MolDesc) * nmol,
                                 cudaMemcpyHostToDevice, stream));
    CDS_CUDA_TRY(cudaMemcpyAsync(lay.newton_set, newton.data(), sizeof(MolDesc) * nmol,
                                 cudaMemcpyHostToDevice, stream));
    if (!gred.empty()) {
        CDS_CUDA_TRY(cudaMemcpyAsync(lay.grid_red, gred.data(), sizeof(OrbRed) * gred.size(),
                                     cudaMemcpyHostToDevice, stream));
        CDS_CUDA_TRY(cudaMemcpyAsync(lay.newton_red, nred.data(), sizeof(OrbRed) * nred.size(),
                                     cudaMemcpyHostToDevice, stream));
    }
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    return CDS_OK;
}

// Device part 1 (capturable): float pairs of eps, the 16-bit split of every
// molecule's factors (rows packed at the molecule's actual Mp) and the split
// scales.  Lov/Lp/eps offsets come from the same table as tc_batch_setup.
int tc_batch_split(int32_t nmol, const BatchMol* mols, const int32_t* M, const BatchOffsets* off,
                   const double* Lov, const double* Lp, const double* eps, int32_t precision,
                   void* ws, cudaStream_t stream) {
    using namespace tc;
    const bool bf16 = precision == CDS_PREC_BF16X3;
    BatchLayout lay = batch_layout(ws, nmol, mols);
    int64_t split_off = 0, nbf_all = 0;
    CDS_CUDA_TRY(cudaMemsetAsync(lay.amax, 0, sizeof(unsigned long long) * 2 * nmol, stream));
    CDS_CUDA_TRY(cudaMemsetAsync(lay.err, 0, sizeof(int32_t), stream));
    for (int c = 0; c < nmol; ++c) {
        const BatchMol& b = mols[c];
        const int32_t nbf = b.nbf, nocc = b.nocc, nv = nbf - nocc, np = b.np;
        const int32_t Mp_cap = padded(std::max(b.max_rank, 1));
        const int32_t Mp = padded(std::max(M[c], 1));
        const double* lp = Lp + off[c].p;
        const double* lov = Lov + off[c].ov;
        uint16_t* lp_hi = lay.hi + split_off;
        uint16_t* lp_lo = lay.lo + split_off;
        uint16_t* ov_hi = lp_hi + (int64_t)np * nbf * Mp_cap;
        uint16_t* ov_lo = lp_lo + (int64_t)np * nbf * Mp_cap;
        const int64_t rp = (int64_t)np * nbf, ro = (int64_t)nocc * nv;
        if (!bf16) {
            if (rp) { k_absmax<<<2 * 152, 256, 0, stream>>>(lp, rp * M[c], lay.amax + 2 * c); CDS_LAUNCH_CHECK(); }
            if (ro) { k_absmax<<<2 * 152, 256, 0, stream>>>(lov, ro * M[c], lay.amax + 2 * c + 1); CDS_LAUNCH_CHECK(); }
        }
        if (rp) {
            if (bf16)
                k_split16<__nv_bfloat16><<<(unsigned)((rp * Mp + 255) / 256), 256, 0, stream>>>(
                    lp, rp, M[c], Mp, lay.amax + 2 * c, (__nv_bfloat16*)lp_hi, (__nv_bfloat16*)lp_lo);
            else
                k_split16<__half><<<(unsigned)((rp * Mp + 255) / 256), 256, 0, stream>>>(
                    lp, rp, M[c], Mp, lay.amax + 2 * c, (__half*)lp_hi, (__half*)lp_lo);
            CDS_LAUNCH_CHECK();
        }
        if (ro) {
            if (bf16)
                k_split16<__nv_bfloat16><<<(unsigned)((ro * Mp + 255) / 256), 256, 0, stream>>>(
                    lov, ro, M[c], Mp, lay.amax + 2 * c + 1, (__nv_bfloat16*)ov_hi, (__nv_bfloat16*)ov_lo);
            else
                k_split16<__half><<<(unsigned)((ro * Mp + 255) / 256), 256, 0, stream>>>(
                    lov, ro, M[c], Mp, lay.amax + 2 * c + 1, (__half*)ov_hi, (__half*)ov_lo);
            CDS_LAUNCH_CHECK();
        }
        k_to_pairs<<<(nbf + 255) / 256, 256, 0, stream>>>(eps + off[c].eps, nbf, lay.eps2 + nbf_all);
        CDS_LAUNCH_CHECK();
        split_off += ((int64_t)np * nbf + (int64_t)nocc * nv) * Mp_cap;
        nbf_all += nbf;
    }
    k_inv_scale_batch<<<(nmol + 127) / 128, 128, 0, stream>>>(lay.amax, bf16 ? 1 : 0, nmol,
                                                              lay.grid_set, lay.newton_set);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

// Device part 2 (capturable): one persistent launch over every molecule's
// items, then the per-orbital reduction.  pass 0: grid energies E (batch
// order [mol][orbital][energy]); pass 1: Newton, one energy per orbital from
// E (batch order [mol][orbital]) with the active mask.
namespace tc {
// Newton pass of a batch from the numerators its grid pass stored: as
// k_sigma_cached, each item's molecule found by binary search over the
// molecules' first items.
__global__ void __launch_bounds__(256)
k_sigma_cached_batch(const MolDesc* __restrict__ mols, int32_t nmol, int64_t nitems,
                     const float* __restrict__ cache, const float2* __restrict__ w2,
                     const float2* __restrict__ eps2, const int32_t* __restrict__ active,
                     double* __restrict__ part) {
    // as k_sigma_cached: warp sums of up to kItems items, one barrier pair
    constexpr int kItems = 16;
    __shared__ float red[kItems][8][2];
    __shared__ double* slot_out[kItems];
    int nslot = 0;
    const int row = threadIdx.x & (TB - 1), half = threadIdx.x / TB;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    auto flush = [&]() {
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * nslot; i += blockDim.x) {
            const int sl = i >> 1, k = i & 1;
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < 8; ++j) v += (double)red[sl][j][k];
            slot_out[sl][k] = v;
        }
        __syncthreads();
        nslot = 0;
    };
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        int lo = 0, hi = nmol - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (mols[mid].item_begin <= item) lo = mid; else hi = mid - 1;
        }
        const MolDesc* md = mols + lo;
        const int64_t r = item - md->item_begin;
        int term, t, s, A, B;
        const TermR tm = decode(md->term[0], md->term[1], r, term, t, s, A, B);
        if (active && !active[md->act_off + t]) continue;   // the same for the whole block
        const int x = A * TB + row;
        const int ybase = B * TB + half * 64;
        const int ncols = min(64, tm.nx - ybase);
        float as = 0.f, ad = 0.f;
        if (x < tm.nx && ncols > 0) {
            const float2* ev = eps2 + md->eps_off;
            const float2 es = ev[tm.eps_s_off + s];
            const float2 ex = ev[tm.eps_x_off + x];
            const float2 c = df_add(w2[md->E_off + (int64_t)t * md->nE],
                                    df_add(es, make_float2(-ex.x, -ex.y)));
            const float* ct = cache + item * kCacheTile + (int64_t)half * 64 * TB + row;
            const float2* ey2 = ev + tm.eps_x_off + ybase;
            // all 64 numerators in flight before the sums (the same order of sums)
            float num[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) num[j] = j < ncols ? ct[(int64_t)j * TB] : 0.f;
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                if (j < ncols) {
                    const float2 e2 = ey2[j];
                    const float d = (c.x - e2.x) + (c.y - e2.y);
                    const float rr = rcp_approx(d);
                    const float tt = num[j] * rr;
                    as += tt;
                    ad = fmaf(-tt, rr, ad);
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            as += __shfl_xor_sync(0xffffffffu, as, o);
            ad += __shfl_xor_sync(0xffffffffu, ad, o);
        }
        if (lane == 0) { red[nslot][w][0] = as; red[nslot][w][1] = ad; }
        if (threadIdx.x == 0) slot_out[nslot] = part + md->part_base + r * (int64_t)md->nE * 2;
        if (++nslot == kItems) flush();
    }
    if (nslot > 0) flush();
}
}  // namespace tc

int tc_batch_pass(int32_t nmol, const BatchMol* mols, int32_t pass, int64_t nE_total,
                  int32_t max_nE, int64_t np_total, const double* E, const int32_t* active,
                  int32_t precision, double* sigma, double* dsigma, unsigned long long* stamps,
                  void* ws, cudaStream_t stream, int32_t cache_mode) {
    using namespace tc;
    const bool bf16 = precision == CDS_PREC_BF16X3;
    BatchLayout lay = batch_layout(ws, nmol, mols);
    float2* Ep = pass == 0 ? lay.E2 : lay.w2;
    const int64_t nE_pairs = pass == 0 ? nE_total : np_total;
    if (nE_pairs > 0) {
        k_to_pairs<<<(unsigned)((nE_pairs + 255) / 256), 256, 0, stream>>>(E, nE_pairs, Ep);
        CDS_LAUNCH_CHECK();
    }
    const MolDesc* set = pass == 0 ? lay.grid_set : lay.newton_set;
    const int64_t nitems = lay.grid_items;
    if (nitems > 0 && cache_mode == 2) {
        const int grid = (int)std::min<int64_t>(nitems, 8LL * device_sms());
        k_sigma_cached_batch<<<grid, 256, 0, stream>>>(set, nmol, nitems, lay.cache, Ep, lay.eps2,
                                                       active, lay.part);
        CDS_LAUNCH_CHECK();
    } else if (nitems > 0) {
        const int grid = (int)std::min<int64_t>(nitems, device_sms());
        Maps dummy_maps;
        memset(&dummy_maps, 0, sizeof(dummy_maps));
        Params dummy{};
        const float2* epsv = lay.eps2;
        const int order = tune_item_order();
        // grid pass keeping the numerators: the epilogue evaluates the first
        // kGridSplitE energies, k_sigma_cached_grid_batch the rest
        const bool split = pass == 0 && cache_mode == 1 && max_nE > kGridSplitE;
        if (split) dummy.nE_eval = kGridSplitE;
        decltype(&k_sigma_tc<1, true, true, true>) kern;
        if (pass == 1 || (split && kGridSplitE == 1))
            kern = bf16 ? k_sigma_tc<1, true, true, true> : k_sigma_tc<1, false, true, true>;
        else if (tune_energy_chunk() == 8)
            kern = bf16 ? k_sigma_tc<8, true, true, true> : k_sigma_tc<8, false, true, true>;
        else
            kern = bf16 ? k_sigma_tc<16, true, true, true> : k_sigma_tc<16, false, true, true>;
        CDS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
        kern<<<grid, THREADS, SMEM_BYTES, stream>>>(dummy_maps, dummy, set, nmol, nitems, Ep, epsv,
                                                    pass == 1 ? active : nullptr, nullptr, lay.part,
                                                    stamps, lay.err, order,
                                                    cache_mode == 1 ? lay.cache : nullptr);
        CDS_LAUNCH_CHECK();
        if (split) {
            const int g2 = (int)std::min<int64_t>(nitems, 4LL * device_sms());
            const int ec = tune_grid_ec();
            if (ec == 2)
                k_sigma_cached_grid_batch<2><<<g2, 256, 0, stream>>>(set, nmol, nitems, lay.cache, Ep,
                                                                     lay.eps2, lay.part, kGridSplitE);
            else if (ec == 8)
                k_sigma_cached_grid_batch<8><<<g2, 256, 0, stream>>>(set, nmol, nitems, lay.cache, Ep,
                                                                     lay.eps2, lay.part, kGridSplitE);
            else
                k_sigma_cached_grid_batch<kGridEC><<<g2, 256, 0, stream>>>(set, nmol, nitems,
                                                                           lay.cache, Ep, lay.eps2,
                                                                           lay.part, kGridSplitE);
            CDS_LAUNCH_CHECK();
        }
    }
    if (np_total > 0) {
        dim3 g((unsigned)std::max(pass == 0 ? max_nE : 1, 1), (unsigned)np_total);
        k_tc_reduce_batch<<<g, 256, 0, stream>>>(lay.part, pass == 0 ? lay.grid_red : lay.newton_red,
                                                 pass == 0 ? nullptr : active, lay.err, sigma, dsigma);
        CDS_LAUNCH_CHECK();
    }
    return CDS_OK;
}

}  // namespace cds

extern "C" int cds_tune_set(int32_t knob, int32_t value) {
    using namespace cds::tc;
    if (knob == CDS_TUNE_ENERGY_CHUNK) {
        if (value != 8 && value != 16) return CDS_ERR_ARG;
        g_energy_chunk = value;
        return CDS_OK;
    }
    if (knob == CDS_TUNE_ITEM_ORDER) {
        if (value != 0 && value != 1) return CDS_ERR_ARG;
        g_item_order = value;
        return CDS_OK;
    }
    if (knob == CDS_TUNE_NEWTON_CACHE) {
        if (value != 0 && value != 1) return CDS_ERR_ARG;
        g_newton_cache = value;
        return CDS_OK;
    }
    if (knob == CDS_TUNE_CD_GRAPH) {
        if (value < 0) return CDS_ERR_ARG;
        g_cd_graph = value;
        return CDS_OK;
    }
    if (knob == CDS_TUNE_PIPE_SPLIT) {
        if (value < 0) return CDS_ERR_ARG;
        g_pipe_split = value;
        return CDS_OK;
    }
    if (knob == CDS_TUNE_GRID_EC) {
        if (value != 2 && value != 4 && value != 8) return CDS_ERR_ARG;
        g_grid_ec = value;
        return CDS_OK;
    }
    return CDS_ERR_ARG;
}

extern "C" int cds_tune_get(int32_t knob) {
    using namespace cds::tc;
    if (knob == CDS_TUNE_ENERGY_CHUNK) return g_energy_chunk.load();
    if (knob == CDS_TUNE_ITEM_ORDER) return g_item_order.load();
    if (knob == CDS_TUNE_NEWTON_CACHE) return g_newton_cache.load();
    if (knob == CDS_TUNE_CD_GRAPH) return g_cd_graph.load();
    if (knob == CDS_TUNE_PIPE_SPLIT) return g_pipe_split.load();
    if (knob == CDS_TUNE_GRID_EC) return g_grid_ec.load();
    return -1;
}
