// Threshold-delta diagonal-pivoted Cholesky decomposition of the ERI
// supermatrix, columns generated on the fly (paper Sec. II.A, Eq. gs_coulomb,
// Eq. CD, Eq. stricterr).
//
// Left-looking form of the Gram-Schmidt steps: at step k with pivot P,
//   L^k_I = [ (rho_I|rho_P) - sum_{K<k} L^K_I L^K_P ] / sqrt(D_P),
//   D_I  -= (L^k_I)^2,  D_P := 0,
// then the next pivot is the largest candidate residual (lowest index among
// values within 1e-12 * max initial diagonal).  One launch of k_cd_update per
// step streams L[0:k][*] once (coalesced along I, the dot product in FP64);
// the grid-wide max is finished by the last block to arrive (no spin waits).
// k_cd_select then picks the pivot.  Both kernels read a device control block
// and return immediately once the decomposition has stopped, so the host can
// enqueue steps ahead and only check the control block every few steps.
#include <vector>

#include "common.cuh"
#include "sigma_tc.cuh"

namespace cds {

constexpr int kCdThreads = 128;
constexpr int kCdPairs = 2;      // pairs per thread in k_cd_update
constexpr int kCdChunk = 2048;   // pivot row L^K_P staged in shared memory in chunks
constexpr double kTieRel = 1e-12;
constexpr double kNotPdRel = 1e-10;
constexpr int kHostCheckEvery = 32;

struct CdCtrl {
    double scale;      // max initial diagonal (all pairs)
    double delta_eff;  // max(delta, npair * 2^-52 * scale)
    double G;          // max candidate residual after the last update
    double Dmin;       // min residual after the last update
    double DP;         // residual of the current pivot
    int64_t P;         // current pivot
    int32_t done;      // decomposition stopped
    int32_t status;    // cds_status
    int32_t M;         // vectors produced
    int32_t _pad;
    unsigned int counter;  // last-block-done counter
    unsigned int _pad2;
};

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
                             double* __restrict__ blk_b, CdCtrl* ctrl, int bid, int nblk) {
    double mx_all = -INFINITY, mx_cand = -INFINITY;
    for (int64_t I = bid * (int64_t)blockDim.x + threadIdx.x; I < n;
         I += (int64_t)nblk * blockDim.x) {
        double p = pd.p[I], px = pd.Px[I], py = pd.Py[I], pz = pd.Pz[I], k = pd.K[I];
        double d = eri_pair(p, px, py, pz, k, p, px, py, pz, k);
        D[I] = d;
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
                          double* __restrict__ blk_a, double* __restrict__ blk_b, CdCtrl* ctrl) {
    cd_init_body(pd, atom, scheme, n, delta, D, cand, blk_a, blk_b, ctrl, blockIdx.x, gridDim.x);
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
                piv[k] = (int32_t)m;
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

// Vector k from pivot P: column, left-looking projection, residual update.
// Each thread owns kCdPairs pairs, blockDim.x * kCdPairs apart, so one grid of
// ~npair / (kCdThreads * kCdPairs) small blocks is resident in a single wave.
__device__ __forceinline__ void cd_update_body(PairSoA pd, int64_t n, int32_t k,
                                               double* __restrict__ L, double* __restrict__ D,
                                               const uint8_t* __restrict__ cand,
                                               double* __restrict__ blk_a,
                                               double* __restrict__ blk_b, CdCtrl* ctrl, int bid,
                                               int nblk) {
    if (ctrl->done) return;
    __shared__ double lp[kCdChunk];
    const int64_t P = ctrl->P;
    const double DP = ctrl->DP;
    const double q = pd.p[P], qx = pd.Px[P], qy = pd.Py[P], qz = pd.Pz[P], kq = pd.K[P];
    const int64_t I0 = (int64_t)bid * blockDim.x * kCdPairs + threadIdx.x;
    int64_t Is[kCdPairs];
    bool live[kCdPairs];
#pragma unroll
    for (int r = 0; r < kCdPairs; ++r) {
        Is[r] = I0 + (int64_t)r * blockDim.x;
        live[r] = Is[r] < n;
    }
    // 4 independent partial sums per pair: 8 loads of L in flight per thread
    double dot[kCdPairs][4] = {};
    int64_t Ic[kCdPairs];
#pragma unroll
    for (int r = 0; r < kCdPairs; ++r) Ic[r] = live[r] ? Is[r] : 0;   // dead lanes read pair 0
    for (int K0 = 0; K0 < k; K0 += kCdChunk) {
        int kc = min(kCdChunk, k - K0);
        __syncthreads();
        for (int j = threadIdx.x; j < kc; j += blockDim.x) lp[j] = L[(int64_t)(K0 + j) * n + P];
        __syncthreads();
        const double* src = L + (int64_t)K0 * n;
        int j = 0;
        for (; j + 4 <= kc; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double lu = lp[j + u];
                const double* row = src + (int64_t)(j + u) * n;
#pragma unroll
                for (int r = 0; r < kCdPairs; ++r) dot[r][u] = fma(row[Ic[r]], lu, dot[r][u]);
            }
        }
        for (; j < kc; ++j) {
#pragma unroll
            for (int r = 0; r < kCdPairs; ++r)
                dot[r][0] = fma(src[(int64_t)j * n + Ic[r]], lp[j], dot[r][0]);
        }
    }
    double mx = -INFINITY, mn = INFINITY;
    const double rs = sqrt(DP);
#pragma unroll
    for (int r = 0; r < kCdPairs; ++r) {
        if (!live[r]) continue;
        const int64_t I = Is[r];
        double e = eri_pair(pd.p[I], pd.Px[I], pd.Py[I], pd.Pz[I], pd.K[I], q, qx, qy, qz, kq);
        double l = (e - ((dot[r][0] + dot[r][1]) + (dot[r][2] + dot[r][3]))) / rs;
        L[(int64_t)k * n + I] = l;
        double d = D[I] - l * l;
        if (I == P) d = 0.0;
        D[I] = d;
        if (cand[I]) mx = fmax(mx, fmax(d, 0.0));
        mn = fmin(mn, d);
    }
    block_maxmin(mx, mn);
    if (threadIdx.x == 0) { blk_a[bid] = mx; blk_b[bid] = mn; }
    if (last_block(&ctrl->counter, nblk)) {
        double A = -INFINITY, B = INFINITY;
        for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
            A = fmax(A, __ldcg(blk_a + i));
            B = fmin(B, __ldcg(blk_b + i));
        }
        block_maxmin(A, B);
        if (threadIdx.x == 0) {
            ctrl->G = A;
            ctrl->Dmin = B;
            ctrl->counter = 0;
        }
    }
}

__global__ void __launch_bounds__(kCdThreads)
k_cd_update(PairSoA pd, int64_t n, int32_t k, double* __restrict__ L, double* __restrict__ D,
            const uint8_t* __restrict__ cand, double* __restrict__ blk_a,
            double* __restrict__ blk_b, CdCtrl* ctrl) {
    cd_update_body(pd, n, k, L, D, cand, blk_a, blk_b, ctrl, blockIdx.x, gridDim.x);
}

struct CdLayout {
    PairSoA pd;
    uint8_t* cand;
    double* blk_a;
    double* blk_b;
    long long* blk_i;
    CdCtrl* ctrl;
    size_t bytes;
};

static int cd_blocks(int64_t n) { return (int)((n + kCdThreads - 1) / kCdThreads); }
static int upd_blocks(int64_t n) {
    return (int)((n + (int64_t)kCdThreads * kCdPairs - 1) / ((int64_t)kCdThreads * kCdPairs));
}
static int sel_blocks(int64_t n) { return (int)std::min<int64_t>(4 * 152, (n + kCdThreads - 1) / kCdThreads); }

static CdLayout cd_layout(void* ws, int32_t nbf) {
    int64_t n = npair_of(nbf);
    int nb = std::max(cd_blocks(n), 1);
    Carver c(ws);
    CdLayout l;
    l.pd.p = c.take<double>(n);
    l.pd.Px = c.take<double>(n);
    l.pd.Py = c.take<double>(n);
    l.pd.Pz = c.take<double>(n);
    l.pd.K = c.take<double>(n);
    l.cand = c.take<uint8_t>(n);
    l.blk_a = c.take<double>(nb);
    l.blk_b = c.take<double>(nb);
    l.blk_i = c.take<long long>(nb);
    l.ctrl = c.take<CdCtrl>(1);
    l.bytes = c.off;
    return l;
}

}  // namespace cds

using namespace cds;

extern "C" size_t cds_cd_workspace_bytes(int32_t nbf) {
    if (nbf < 0) return 0;
    return cd_layout(nullptr, nbf).bytes;
}

extern "C" int cds_cd_decompose(int32_t nbf, const double* xyz, const double* alpha,
                                const int32_t* atom, double delta, int32_t scheme,
                                int32_t max_rank, double* L, int32_t* piv, double* D,
                                int32_t* M_out, double* delta_eff_out, void* workspace,
                                size_t workspace_bytes, cudaStream_t stream) {
    if (nbf <= 0 || !xyz || !alpha || !L || !piv || !D || !M_out || max_rank < 0)
        return CDS_ERR_ARG;
    if (!(delta >= 0.0)) return CDS_ERR_ARG;
    if (scheme != CDS_SCHEME_FULL && scheme != CDS_SCHEME_ATOMIC) return CDS_ERR_ARG;
    if (scheme == CDS_SCHEME_ATOMIC && !atom) return CDS_ERR_ARG;
    int64_t n = npair_of(nbf);
    CdLayout lay = cd_layout(workspace, nbf);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    int st = build_pairs(nbf, xyz, alpha, lay.pd, stream);
    if (st) return st;
    CDS_CUDA_TRY(cudaMemsetAsync(lay.ctrl, 0, sizeof(CdCtrl), stream));
    int nb = cd_blocks(n), ns = sel_blocks(n), nu = upd_blocks(n);
    k_cd_init<<<nb, kCdThreads, 0, stream>>>(lay.pd, atom, scheme, n, delta, D, lay.cand,
                                            lay.blk_a, lay.blk_b, lay.ctrl);
    CDS_LAUNCH_CHECK();
    k_cd_select<<<ns, kCdThreads, 0, stream>>>(n, 0, max_rank, D, lay.cand, lay.blk_i, piv,
                                              lay.ctrl);
    CDS_LAUNCH_CHECK();
    CdCtrl h{};
    for (int32_t k0 = 0; k0 <= max_rank; k0 += kHostCheckEvery) {
        int32_t k1 = std::min(max_rank, k0 + kHostCheckEvery);
        for (int32_t k = k0; k < k1; ++k) {
            k_cd_update<<<nu, kCdThreads, 0, stream>>>(lay.pd, n, k, L, D, lay.cand, lay.blk_a,
                                                      lay.blk_b, lay.ctrl);
            k_cd_select<<<ns, kCdThreads, 0, stream>>>(n, k + 1, max_rank, D, lay.cand,
                                                      lay.blk_i, piv, lay.ctrl);
        }
        count_launches(2ull * (unsigned long long)(k1 - k0));
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
    const int32_t* atom;
    double* L;
    double* D;
    uint8_t* cand;
    int32_t* piv;
    double* blk_a;
    double* blk_b;
    long long* blk_i;
    CdCtrl* ctrl;
    int64_t n;
    int32_t max_rank;
    int32_t b0_init, nb_init, b0_upd, nb_upd, b0_sel, nb_sel;
};

// Molecule owning block bid of a batch grid (kind: 0 init, 1 update, 2 select).
__device__ __forceinline__ int find_mol(const CdMol* mols, int nmol, int bid, int kind) {
    int lo = 0, hi = nmol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int b0 = kind == 0 ? mols[mid].b0_init : kind == 1 ? mols[mid].b0_upd : mols[mid].b0_sel;
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

__global__ void __launch_bounds__(kCdThreads) k_bcd_update(const CdMol* __restrict__ mols, int nmol,
                                                           int32_t k) {
    const int c = find_mol(mols, nmol, blockIdx.x, 1);
    const CdMol& m = mols[c];
    if (k >= m.max_rank) return;
    cd_update_body(m.pd, m.n, k, m.L, m.D, m.cand, m.blk_a, m.blk_b, m.ctrl,
                   blockIdx.x - m.b0_upd, m.nb_upd);
}

struct CdBatchLayout {
    CdMol* mols;          // device descriptors
    CdCtrl* ctrl;         // [nmol]
    char* per_mol;        // pair data, masks, block partials of every molecule
    size_t bytes;
};

static size_t cd_mol_bytes(int64_t n) {
    const size_t nb = (size_t)std::max(cd_blocks(n), 1);
    return 5 * align_up(n * sizeof(double)) + align_up(n) + 3 * align_up(nb * sizeof(double));
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
                       int32_t scheme, double* L, int32_t* piv, double* D, int32_t* M_out,
                       void* ws, size_t ws_bytes, cudaStream_t stream) {
    CdBatchLayout lay = cd_batch_layout(ws, nmol, mols);
    if (!ws || ws_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    std::vector<CdMol> h(nmol);
    char* p = lay.per_mol;
    int b_init = 0, b_upd = 0, b_sel = 0, kmax = 0;
    for (int c = 0; c < nmol; ++c) {
        const int64_t n = npair_of(mols[c].nbf);
        const size_t nb = (size_t)std::max(cd_blocks(n), 1);
        CdMol& m = h[c];
        Carver cv(p);
        m.pd.p = cv.take<double>(n);
        m.pd.Px = cv.take<double>(n);
        m.pd.Py = cv.take<double>(n);
        m.pd.Pz = cv.take<double>(n);
        m.pd.K = cv.take<double>(n);
        m.cand = cv.take<uint8_t>(n);
        m.blk_a = cv.take<double>(nb);
        m.blk_b = cv.take<double>(nb);
        m.blk_i = cv.take<long long>(nb);
        p += cd_mol_bytes(n);
        m.atom = atom + off[c].basis;
        m.L = L + off[c].L;
        m.D = D + off[c].pair;
        m.piv = piv + off[c].piv;
        m.ctrl = lay.ctrl + c;
        m.n = n;
        m.max_rank = mols[c].max_rank;
        m.b0_init = b_init; m.nb_init = cd_blocks(n); b_init += m.nb_init;
        m.b0_upd = b_upd; m.nb_upd = upd_blocks(n); b_upd += m.nb_upd;
        m.b0_sel = b_sel; m.nb_sel = sel_blocks(n); b_sel += m.nb_sel;
        kmax = std::max(kmax, mols[c].max_rank);
        int st = build_pairs(mols[c].nbf, xyz + 3 * off[c].basis, alpha + off[c].basis, m.pd, stream);
        if (st) return st;
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
            k_bcd_update<<<b_upd, kCdThreads, 0, stream>>>(lay.mols, nmol, k);
            k_bcd_select<<<b_sel, kCdThreads, 0, stream>>>(lay.mols, nmol, k + 1);
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
    }
    return status;
}

}  // namespace cds
