// Tensor-core path of the diagonal self-energy (paper Eq. SE) for sm_103a:
// tcgen05 MMAs with TMEM accumulators, operands staged by TMA.
//
// Precision (BF16X3): every factor L^J_pq is split in FP64 into
// hi = bf16(x) and lo = bf16(x - hi); each J-contraction is
//   X = Ahi.Bhi + Ahi.Blo + Alo.Bhi
// with FP32 accumulation in TMEM (the lo.lo product, ~2^-16 relative, is
// dropped).  Denominators and per-tile sums are FP32, with denominators
// closer than 1e-3 Ha to a pole recomputed in FP64; per-tile totals are
// summed across tiles in FP64 in a fixed order.
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
// TMEM holds two accumulator pairs (512 columns) so the epilogue of one item
// overlaps the MMAs of the next.  Every wait is bounded (2 s of %globaltimer)
// and sets an error word instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "sigma_tc.cuh"

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
constexpr float POLE_GUARD = 1e-3f;
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;
constexpr size_t SMEM_BYTES = 1024 + NSTAGE * STAGE_BYTES + 256 + NUM_EPI_WARPS * 16 * 2 * 4;

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, M=N=128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TB >> 3) << 17) |
                           ((uint32_t)(TB >> 4) << 24);

struct Maps {
    CUtensorMap m[2][4];   // [term][aq_hi, aq_lo, bk_hi, bk_lo]
};

struct Term {
    int32_t nx, ns, nb, bulk_s_dim;   // bulk_s_dim: 1 if spectator is dim 1 of the bulk map, else 2
    int64_t npb, nitems, item0;
    const double* eps_s;
    const double* eps_x;
};

struct Params {
    Term term[2];
    int32_t kblocks;
    int32_t nE;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on one mbarrier phase; false after TIMEOUT_NS or if another
// role has already flagged an error.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int32_t* err,
                                          bool stop_on_err = true) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0) {
            if (stop_on_err && *err) return false;
            if (gtimer() - t0 > TIMEOUT_NS) {
                atomicExch((int32_t*)err, (int32_t)CDS_ERR_TIMEOUT);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart (SBO), version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
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

__device__ __forceinline__ bool decode(const Params& P, int64_t item, int& term, int& t, int& s,
                                       int& A, int& B) {
    term = item < P.term[0].nitems ? 0 : 1;
    const Term& tm = P.term[term];
    int64_t r = item - (term ? P.term[0].nitems : 0);
    int64_t per_t = (int64_t)tm.ns * tm.npb;
    t = (int)(r / per_t);
    r -= (int64_t)t * per_t;
    s = (int)(r / tm.npb);
    block_pair(r - (int64_t)s * tm.npb, tm.nb, A, B);
    return true;
}

template <int EC>
__global__ void __launch_bounds__(THREADS, 1)
k_sigma_tc(const __grid_constant__ Maps maps, const Params P, const double* __restrict__ E,
           const int32_t* __restrict__ active, double* __restrict__ part,
           int32_t* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stages = smem;
    uint64_t* bars = (uint64_t*)(smem + NSTAGE * STAGE_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + NSTAGE;
    uint64_t* tfull = bars + 2 * NSTAGE;
    uint64_t* tempty = tfull + 2;
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    float* red = (float*)(smem + NSTAGE * STAGE_BYTES + 256);   // [8 warps][16][2]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nitems = P.term[0].nitems + P.term[1].nitems;
    volatile int32_t* verr = err;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSTAGE; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], NUM_EPI_WARPS); }
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
            for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                int term, t, s, A, B;
                decode(P, item, term, t, s, A, B);
                if (active && !active[t]) continue;
                const Term& tm = P.term[term];
                const CUtensorMap* mq_hi = &maps.m[term][0];
                const CUtensorMap* mq_lo = &maps.m[term][1];
                const CUtensorMap* mb_hi = &maps.m[term][2];
                const CUtensorMap* mb_lo = &maps.m[term][3];
                const bool diag = A == B;
                const uint32_t bytes = (diag ? 4u : 8u) * TILE_BYTES;
                const int bA1 = tm.bulk_s_dim == 2 ? A * TB : s, bA2 = tm.bulk_s_dim == 2 ? s : A * TB;
                const int bB1 = tm.bulk_s_dim == 2 ? B * TB : s, bB2 = tm.bulk_s_dim == 2 ? s : B * TB;
                for (int kb = 0; kb < P.kblocks; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, verr)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[stage], bytes);
                    last_parity[stage] = (int32_t)phase;
                    const uint32_t st = smem_u32(stages + stage * STAGE_BYTES);
                    const int k0 = kb * KB;
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
            for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                int term, t, s, A, B;
                decode(P, item, term, t, s, A, B);
                if (active && !active[t]) continue;
                const bool diag = A == B;
                if (!mbar_wait(&tempty[acc], aphase ^ 1u, verr)) break;
                fence_after();
                const uint32_t d1 = tmem + (uint32_t)acc * 256u, d2 = d1 + 128u;
                for (int kb = 0; kb < P.kblocks; ++kb) {
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
                    for (int kk = 0; kk < KB / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint32_t first = (kb | kk) ? 1u : 0u;
                        mma_bf16(d1, sdesc(a1h + off), sdesc(b1h + off), first);
                        mma_bf16(d1, sdesc(a1h + off), sdesc(b1l + off), 1u);
                        mma_bf16(d1, sdesc(a1l + off), sdesc(b1h + off), 1u);
                        mma_bf16(d2, sdesc(a2h + off), sdesc(b2h + off), first);
                        mma_bf16(d2, sdesc(a2h + off), sdesc(b2l + off), 1u);
                        mma_bf16(d2, sdesc(a2l + off), sdesc(b2h + off), 1u);
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
        // ---------------- epilogue (8 warps) ----------------
        const int ew = warp - 2;
        const int quad = warp & 3;     // TMEM lanes this warp may read
        const int half = ew >> 2;      // column half of the tile
        const int row = quad * 32 + lane;
        int acc = 0;
        uint32_t aphase = 0;
        const int nE = P.nE;
        for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
            int term, t, s, A, B;
            decode(P, item, term, t, s, A, B);
            if (active && !active[t]) continue;
            const Term& tm = P.term[term];
            const bool bad = !mbar_wait(&tfull[acc], aphase, verr) || *verr;
            if (epi_any(bad)) break;
            fence_after();
            const bool diag = A == B;
            const int x = A * TB + row;
            const bool xok = x < tm.nx;
            const double es = tm.eps_s[s];
            const double ex = xok ? tm.eps_x[x] : 0.0;
            const uint32_t ta1 = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)acc * 256u +
                                 (uint32_t)half * 64u;
            const uint32_t ta2 = ta1 + 128u;
            const int ybase = B * TB + half * 64;
            const double* Et = E + (int64_t)t * nE;
            double* out = part + (tm.item0 + (item - (term ? P.term[0].nitems : 0))) * (int64_t)nE * 2;
            for (int e0 = 0; e0 < nE; e0 += EC) {
                const int ne = min(EC, nE - e0);
                float c[EC], as[EC], ad[EC];
#pragma unroll
                for (int e = 0; e < EC; ++e) {
                    c[e] = e < ne ? (float)(Et[e0 + e] + es - ex) : 1.0f;
                    as[e] = 0.f;
                    ad[e] = 0.f;
                }
#pragma unroll 1
                for (int cc = 0; cc < 64; cc += 16) {
                    float x1[16], x2[16];
                    tmem_ld16(ta1 + cc, x1);
                    tmem_ld16(ta2 + cc, x2);
                    tmem_wait_ld();
                    float num[16], ey[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int y = ybase + cc + j;
                        const bool ok = xok && y < tm.nx;
                        const float a = x1[j], b = x2[j];
                        const float n = diag ? (2.f * a - b) * a : 2.f * (a * a + b * b - a * b);
                        num[j] = ok ? n : 0.f;
                        ey[j] = ok ? (float)tm.eps_x[y] : -1e30f;   // padding: 0 * tiny
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
#pragma unroll
                        for (int e = 0; e < EC; ++e) {
                            const float d = c[e] - ey[j];
                            float r = rcp_approx(d);
                            float tt = num[j] * r;
                            if (fabsf(d) < POLE_GUARD && num[j] != 0.f && e < ne) {
                                // close to a pole: the denominator in FP64
                                const double dd = (Et[e0 + e] + es - ex) - tm.eps_x[ybase + cc + j];
                                const double rr = 1.0 / dd;
                                const double t64 = (double)num[j] * rr;
                                tt = (float)t64;
                                r = (float)rr;
                            }
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
                        red[(ew * 16 + e) * 2] = as[e];
                        red[(ew * 16 + e) * 2 + 1] = ad[e];
                    }
                }
                epi_bar();
                const int idx = ew * 32 + lane;
                if (idx < ne) {
                    double sv = 0.0, dv = 0.0;
#pragma unroll
                    for (int w = 0; w < NUM_EPI_WARPS; ++w) {
                        sv += (double)red[(w * 16 + idx) * 2];
                        dv += (double)red[(w * 16 + idx) * 2 + 1];
                    }
                    out[(e0 + idx) * 2] = sv;
                    out[(e0 + idx) * 2 + 1] = dv;
                }
                epi_bar();
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

// hi = bf16(x), lo = bf16(x - hi); columns J >= M zero (rows padded to Mp).
__global__ void k_split_bf16(const double* __restrict__ src, int64_t rows, int32_t M, int32_t Mp,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * Mp) return;
    int64_t r = e / Mp;
    int J = (int)(e - r * Mp);
    double x = J < M ? src[r * M + J] : 0.0;
    __nv_bfloat16 h = __double2bfloat16(x);
    hi[e] = h;
    lo[e] = __double2bfloat16(x - (double)__bfloat162float(h));
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
    __nv_bfloat16 *lp_hi, *lp_lo, *lov_hi, *lov_lo;
    double* part;
    int32_t* err;
    size_t bytes;
};

inline int32_t padded(int32_t M) { return (M + KB - 1) / KB * KB; }

int64_t tc_items(int32_t nx, int32_t ns, int32_t np) {
    if (nx <= 0 || ns <= 0) return 0;
    return (int64_t)np * ns * npairs_of(nblocks_of(nx, TB));
}

TcLayout tc_layout(void* ws, int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE) {
    const int32_t Mp = padded(std::max(M, 1)), nv = nmo - nocc;
    Carver c(ws);
    TcLayout l;
    l.lp_hi = c.take<__nv_bfloat16>((size_t)np * nmo * Mp);
    l.lp_lo = c.take<__nv_bfloat16>((size_t)np * nmo * Mp);
    l.lov_hi = c.take<__nv_bfloat16>((size_t)nocc * nv * Mp);
    l.lov_lo = c.take<__nv_bfloat16>((size_t)nocc * nv * Mp);
    int64_t items = tc_items(nocc, nv, np) + tc_items(nv, nocc, np);
    l.part = c.take<double>((size_t)std::max<int64_t>(items, 1) * nE * 2);
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

// 3-D bf16 map {d0 (J, contiguous), d1, d2} with byte strides s1, s2.
bool make_map(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
              uint64_t s1, uint64_t s2, uint32_t b1, uint32_t b2) {
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {s1, s2};
    cuuint32_t box[3] = {(cuuint32_t)KB, b1, b2};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                     box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
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

size_t tc_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np, int32_t nE) {
    return tc::tc_layout(nullptr, nmo, nocc, M, np, nE).bytes;
}

int sigma2_tc(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
              int32_t np, const double* eps, const double* E, int32_t nE,
              const int32_t* active, double* sigma, double* dsigma, void* ws,
              cudaStream_t stream) {
    using namespace tc;
    if (!device_ok()) return CDS_ERR_UNSUPPORTED;
    const int32_t nv = nmo - nocc;
    const int32_t Mp = padded(std::max(M, 1));
    TcLayout lay = tc_layout(ws, nmo, nocc, M, np, nE);
    // split the factors into bf16 hi/lo operand arrays
    {
        int64_t n1 = (int64_t)np * nmo * Mp;
        k_split_bf16<<<(unsigned)((n1 + 255) / 256), 256, 0, stream>>>(Lp, (int64_t)np * nmo, M, Mp,
                                                                      lay.lp_hi, lay.lp_lo);
        CDS_LAUNCH_CHECK();
        int64_t n2 = (int64_t)nocc * nv * Mp;
        if (n2 > 0) {
            k_split_bf16<<<(unsigned)((n2 + 255) / 256), 256, 0, stream>>>(
                Lov, (int64_t)nocc * nv, M, Mp, lay.lov_hi, lay.lov_lo);
            CDS_LAUNCH_CHECK();
        }
    }
    Params P{};
    Maps maps;
    memset(&maps, 0, sizeof(maps));
    const uint64_t rowb = (uint64_t)Mp * 2;
    // term 0 (first sum of Eq. SE): x = occupied rows of Lp, bulk L^J_{a j}
    // read from Lov[j][a] with spectator a as map dim 1 and y = j as dim 2.
    // term 1 (second sum): x = virtual rows of Lp, bulk Lov[i][b], spectator i dim 2.
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
        tm.eps_s = k == 0 ? eps + nocc : eps;
        tm.eps_x = k == 0 ? eps : eps + nocc;
        if (tm.nitems == 0) continue;
        const __nv_bfloat16* qb_hi = lay.lp_hi + (k == 0 ? 0 : (size_t)nocc * Mp);
        const __nv_bfloat16* qb_lo = lay.lp_lo + (k == 0 ? 0 : (size_t)nocc * Mp);
        bool ok = make_map(&maps.m[k][0], qb_hi, Mp, nx[k], np, rowb, rowb * nmo, TB, 1) &&
                  make_map(&maps.m[k][1], qb_lo, Mp, nx[k], np, rowb, rowb * nmo, TB, 1) &&
                  make_map(&maps.m[k][2], lay.lov_hi, Mp, nv, nocc, rowb, rowb * nv,
                           k == 0 ? 1 : TB, k == 0 ? TB : 1) &&
                  make_map(&maps.m[k][3], lay.lov_lo, Mp, nv, nocc, rowb, rowb * nv,
                           k == 0 ? 1 : TB, k == 0 ? TB : 1);
        if (!ok) return CDS_ERR_CUDA;
    }
    P.kblocks = Mp / KB;
    P.nE = nE;
    const int64_t nitems = P.term[0].nitems + P.term[1].nitems;
    CDS_CUDA_TRY(cudaMemsetAsync(lay.err, 0, sizeof(int32_t), stream));
    if (nitems > 0) {
        int grid = (int)std::min<int64_t>(nitems, device_sms());
        if (nE == 1) {
            CDS_CUDA_TRY(cudaFuncSetAttribute(k_sigma_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)SMEM_BYTES));
            k_sigma_tc<1><<<grid, THREADS, SMEM_BYTES, stream>>>(maps, P, E, active, lay.part, lay.err);
        } else {
            CDS_CUDA_TRY(cudaFuncSetAttribute(k_sigma_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)SMEM_BYTES));
            k_sigma_tc<16><<<grid, THREADS, SMEM_BYTES, stream>>>(maps, P, E, active, lay.part, lay.err);
        }
        CDS_LAUNCH_CHECK();
    }
    if (nitems == 0) {
        CDS_CUDA_TRY(cudaMemsetAsync(lay.part, 0, sizeof(double) * 2 * nE, stream));
    }
    const int64_t per0 = np ? P.term[0].nitems / np : 0, per1 = np ? P.term[1].nitems / np : 0;
    dim3 grid(nE, np);
    k_tc_reduce<<<grid, 256, 0, stream>>>(lay.part, per0, P.term[0].nitems, per1, nE, active,
                                         lay.err, sigma, dsigma);
    CDS_LAUNCH_CHECK();
    return CDS_OK;
}

}  // namespace cds
