// Batched form of the path: many molecules of uneven size, orbital count and
// energy count per call.
//
//  * Cholesky decomposition: FP64 / float pairs: one update and one select
//    launch per step for the whole batch (cd.cu, cd_batch_decompose); the
//    tensor-core form (CDS_PREC_OZAKI): every molecule's screening, then
//    three launches per step for the whole batch (cd.cu,
//    cd_batch_decompose_tc).
//  * Transform: per molecule, the molecules spread over kWorkers host
//    threads, each driving a library stream of its own.
//  * Self-energy: the work items of every molecule in one persistent
//    tcgen05 launch (sigma_tc.cu, tc_batch_pass), per-molecule descriptors in
//    device memory.
//  * Newton: one batched self-energy pass (one energy per orbital) and one
//    update kernel per iteration for all molecules' orbitals.
//  * A CUDA graph of the self-energy grid + Newton stage, captured by the
//    library with a fixed iteration count (converged orbitals skip their
//    work), replayed with one launch.
// Per-molecule completion times are stamped on the device with %globaltimer.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "sigma_tc.cuh"

namespace cds {


size_t cd_batch_workspace_bytes(int32_t nmol, const BatchMol* mols);
int cd_batch_decompose(int32_t nmol, const BatchMol* mols, const BatchOffsets* off,
                       const double* xyz, const double* alpha, const int32_t* atom, double delta,
                       int32_t scheme, int32_t precision, double* L, int32_t* piv, double* D,
                       int32_t* M_out, void* ws, size_t ws_bytes, cudaStream_t stream);
size_t cd_tc_batch_workspace_bytes(int32_t nmol, const BatchMol* mols);
int cd_batch_decompose_tc(int32_t nmol, const BatchMol* mols, const BatchOffsets* off,
                          const double* xyz, const double* alpha, const int32_t* atom,
                          double delta, int32_t scheme, double* L, int32_t* piv, double* D,
                          int32_t* M_out, void* ws, size_t ws_bytes, cudaStream_t stream);

namespace {

std::vector<BatchMol> to_internal(int32_t nmol, const cds_mol* mols) {
    std::vector<BatchMol> v(nmol);
    for (int c = 0; c < nmol; ++c)
        v[c] = BatchMol{mols[c].nbf, mols[c].nocc, mols[c].np, mols[c].nE, mols[c].max_rank};
    return v;
}

bool mols_ok(int32_t nmol, const cds_mol* mols) {
    if (nmol <= 0 || nmol > 65535 || !mols) return false;
    for (int c = 0; c < nmol; ++c) {
        const cds_mol& m = mols[c];
        if (m.nbf <= 0 || m.nocc < 0 || m.nocc > m.nbf || m.np < 0 || m.nE < 1 || m.nE > 4096 ||
            m.max_rank < 1)
            return false;
    }
    return true;
}

std::vector<BatchOffsets> offsets_of(int32_t nmol, const cds_mol* mols, BatchOffsets* total) {
    std::vector<BatchOffsets> o(nmol);
    BatchOffsets t{};
    for (int c = 0; c < nmol; ++c) {
        const cds_mol& m = mols[c];
        const int64_t nbf = m.nbf, np = npair_of(m.nbf), nv = m.nbf - m.nocc;
        o[c] = t;
        t.basis += nbf;
        t.pair += np;
        t.L += (int64_t)m.max_rank * np;
        t.piv += m.max_rank;
        t.C += nbf * nbf;
        t.eps += nbf;
        t.orb += m.np;
        t.E += (int64_t)m.np * m.nE;
        t.ov += (int64_t)m.nocc * nv * m.max_rank;
        t.p += (int64_t)m.np * nbf * m.max_rank;
    }
    if (total) *total = t;
    return o;
}

// ---- per-molecule work on worker threads with library streams of their own ----
constexpr int kWorkers = 8;

int worker_streams(cudaStream_t (&out)[kWorkers]) {
    static std::mutex lock;
    static cudaStream_t per_dev[64][kWorkers] = {};
    int dev = 0;
    CDS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CDS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(lock);
    for (int t = 0; t < kWorkers; ++t) {
        if (!per_dev[dev][t])
            CDS_CUDA_TRY(cudaStreamCreateWithFlags(&per_dev[dev][t], cudaStreamNonBlocking));
        out[t] = per_dev[dev][t];
    }
    return CDS_OK;
}

// Largest molecules first (pairs x capacity), so the threads finish together.
std::vector<int> by_size(int32_t nmol, const cds_mol* mols) {
    std::vector<int> order(nmol);
    for (int c = 0; c < nmol; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return npair_of(mols[a].nbf) * mols[a].max_rank > npair_of(mols[b].nbf) * mols[b].max_rank;
    });
    return order;
}

// job(c, stream, slot) for every molecule c, slot = the worker's index (its
// workspace slot); the workers' streams start after the work enqueued on
// `stream` so far, and `stream` waits for all of them.  Returns the first
// non-OK status in molecule order.
template <class Job>
int run_workers(int32_t nmol, const cds_mol* mols, cudaStream_t stream, Job job) {
    cudaStream_t ws[kWorkers];
    int st = worker_streams(ws);
    if (st) return st;
    int dev = 0;
    CDS_CUDA_TRY(cudaGetDevice(&dev));
    cudaEvent_t start, done[kWorkers];
    CDS_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    for (int t = 0; t < kWorkers; ++t)
        CDS_CUDA_TRY(cudaEventCreateWithFlags(&done[t], cudaEventDisableTiming));
    CDS_CUDA_TRY(cudaEventRecord(start, stream));
    const std::vector<int> order = by_size(nmol, mols);
    std::vector<int> status(nmol, CDS_OK);
    std::vector<int> werr(kWorkers, CDS_OK);
    std::atomic<int> next{0};
    auto worker = [&](int t) {
        if (cudaSetDevice(dev) != cudaSuccess || cudaStreamWaitEvent(ws[t], start, 0) != cudaSuccess) {
            werr[t] = CDS_ERR_CUDA;
            return;
        }
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nmol) break;
            status[order[i]] = job(order[i], ws[t], t);
        }
        if (cudaEventRecord(done[t], ws[t]) != cudaSuccess) werr[t] = CDS_ERR_CUDA;
    };
    const int nt = std::min<int>(kWorkers, nmol);
    std::vector<std::thread> threads;
    for (int t = 0; t < nt; ++t) threads.emplace_back(worker, t);
    for (std::thread& th : threads) th.join();
    int res = CDS_OK;
    for (int t = 0; t < nt; ++t) {
        if (!res && werr[t]) res = werr[t];
        if (!werr[t] && cudaStreamWaitEvent(stream, done[t], 0) != cudaSuccess && !res)
            res = CDS_ERR_CUDA;
    }
    for (int c = 0; c < nmol && !res; ++c) res = status[c];
    cudaEventDestroy(start);
    for (int t = 0; t < kWorkers; ++t) cudaEventDestroy(done[t]);
    return res;
}

// Bytes of one worker's slot: the largest molecule's transform workspace.
size_t worker_slot_bytes(int32_t nmol, const cds_mol* mols) {
    size_t b = 0;
    for (int c = 0; c < nmol; ++c)
        b = std::max(b, cds_cd_to_mo_workspace_bytes(mols[c].nbf, mols[c].nbf, mols[c].nocc,
                                                     mols[c].max_rank, mols[c].np));
    return align_up(b);
}

// Per-orbital data of the batched Newton solve.
struct OrbQP {
    int32_t mol;
    int32_t eps_off;   // offset of the molecule's orbital energies
    int32_t nmo;
    int32_t pad;
};

__global__ void k_bqp_init(const OrbQP* __restrict__ meta, int64_t nt, const double* __restrict__ eps,
                           const int32_t* __restrict__ orb, double* omega, double* pole,
                           int32_t* iters, int32_t* status, int32_t* active) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nt) return;
    const OrbQP m = meta[g];
    const int q = orb[g];
    const bool ok = q >= 0 && q < m.nmo;
    omega[g] = ok ? eps[m.eps_off + q] : __longlong_as_double(0x7ff8000000000000LL);
    pole[g] = 1.0;
    iters[g] = 0;
    status[g] = ok ? CDS_QP_NO_CONVERGENCE : CDS_QP_NONFINITE;
    active[g] = ok ? 1 : 0;
}

__global__ void k_bqp_step(const OrbQP* __restrict__ meta, int64_t nt, const double* __restrict__ eps,
                           const int32_t* __restrict__ orb, const double* __restrict__ sig,
                           const double* __restrict__ dsig, double conv, double* omega, double* pole,
                           int32_t* iters, int32_t* status, int32_t* active, int32_t* nactive,
                           unsigned long long* stamps) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nt || !active[g]) return;
    const OrbQP m = meta[g];
    double w = omega[g];
    double P = 1.0 / (1.0 - dsig[g]);
    double wn = w + (eps[m.eps_off + orb[g]] + sig[g] - w) * P;
    iters[g] += 1;
    pole[g] = P;
    omega[g] = wn;
    bool retire = true;
    if (!isfinite(wn)) {
        status[g] = CDS_QP_NONFINITE;
    } else if (fabs(wn - w) <= conv) {
        status[g] = CDS_QP_OK;
    } else {
        retire = false;
        atomicAdd(nactive, 1);
    }
    if (retire) {
        active[g] = 0;
        if (stamps) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            atomicMax(stamps + 1 + m.mol, t);
        }
    }
}

__global__ void k_stamp_start(unsigned long long* stamps, int nmol) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        stamps[0] = t;
    }
    if (i < nmol) stamps[1 + i] = 0;
}

struct QpBatchLayout {
    double* sig;
    double* dsig;
    int32_t* active;
    int32_t* nactive;
    OrbQP* meta;
    void* tc;          // tc batch workspace
    size_t bytes;
};

QpBatchLayout qp_batch_layout(void* ws, int32_t nmol, const BatchMol* bm, int64_t np_all) {
    Carver c(ws);
    QpBatchLayout l;
    l.sig = c.take<double>(std::max<int64_t>(np_all, 1));
    l.dsig = c.take<double>(std::max<int64_t>(np_all, 1));
    l.active = c.take<int32_t>(std::max<int64_t>(np_all, 1));
    l.nactive = c.take<int32_t>(4);
    l.meta = c.take<OrbQP>(std::max<int64_t>(np_all, 1));
    l.tc = c.take<char>(tc_batch_workspace_bytes(nmol, bm));
    l.bytes = c.off;
    return l;
}

// The whole Sigma-grid + Newton stage on a stream; fixed_iters: no host
// synchronisation (for graph capture), every orbital runs until converged
// or max_iter, converged ones skipping their work.
int sigma_qp_stage(int32_t nmol, const std::vector<BatchMol>& bm, const std::vector<BatchOffsets>& off,
                   const BatchOffsets& tot, const int32_t* M, const double* Lov, const double* Lp,
                   const int32_t* orb, const double* eps, const double* E, int32_t precision,
                   double conv, int32_t max_iter, bool fixed_iters, double* sigma, double* dsigma,
                   double* omega, double* pole, int32_t* iters, int32_t* status,
                   unsigned long long* stamps, const QpBatchLayout& lay, cudaStream_t stream,
                   int* all_converged) {
    int max_nE = 1;
    for (auto& b : bm) max_nE = std::max(max_nE, b.nE);
    const int64_t np_all = tot.orb;
    if (stamps) {
        k_stamp_start<<<(nmol + 256) / 256, 256, 0, stream>>>(stamps, nmol);
        CDS_LAUNCH_CHECK();
    }
    int st = tc_batch_split(nmol, bm.data(), M, off.data(), Lov, Lp, eps, precision, lay.tc, stream);
    if (st) return st;
    // Newton from cached numerators: the grid pass stores them, or else the
    // first Newton pass (which recomputes) does
    const bool cached = tc::tune_newton_cache() != 0;
    bool have_cache = false;
    if (sigma) {
        st = tc_batch_pass(nmol, bm.data(), 0, tot.E, max_nE, np_all, E, nullptr, precision, sigma,
                           dsigma, nullptr, lay.tc, stream, cached ? 1 : 0);
        if (st) return st;
        have_cache = cached;
    }
    if (!omega) return CDS_OK;
    const int nb = (int)((np_all + 127) / 128);
    k_bqp_init<<<std::max(nb, 1), 128, 0, stream>>>(lay.meta, np_all, eps, orb, omega, pole, iters,
                                                   status, lay.active);
    CDS_LAUNCH_CHECK();
    int32_t h_active = (int32_t)np_all;
    for (int32_t it = 0; it < max_iter && (fixed_iters || h_active > 0); ++it) {
        const int32_t mode = !cached ? 0 : have_cache ? 2 : 1;
        st = tc_batch_pass(nmol, bm.data(), 1, tot.E, max_nE, np_all, omega, lay.active, precision,
                           lay.sig, lay.dsig, nullptr, lay.tc, stream, mode);
        if (st) return st;
        have_cache = cached;
        CDS_CUDA_TRY(cudaMemsetAsync(lay.nactive, 0, sizeof(int32_t), stream));
        k_bqp_step<<<std::max(nb, 1), 128, 0, stream>>>(lay.meta, np_all, eps, orb, lay.sig, lay.dsig,
                                                       conv, omega, pole, iters, status, lay.active,
                                                       lay.nactive, stamps);
        CDS_LAUNCH_CHECK();
        if (!fixed_iters) {
            CDS_CUDA_TRY(cudaMemcpyAsync(&h_active, lay.nactive, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, stream));
            CDS_CUDA_TRY(cudaStreamSynchronize(stream));
        }
    }
    if (all_converged) *all_converged = h_active == 0;
    return CDS_OK;
}

int stage_setup(int32_t nmol, const std::vector<BatchMol>& bm, const int32_t* M, int32_t precision,
                const QpBatchLayout& lay, cudaStream_t stream) {
    int st = tc_batch_setup(nmol, bm.data(), M, precision, lay.tc, stream);
    if (st) return st;
    std::vector<OrbQP> meta;
    int32_t eo = 0;
    for (int c = 0; c < nmol; ++c) {
        for (int t = 0; t < bm[c].np; ++t) meta.push_back(OrbQP{c, eo, bm[c].nbf, 0});
        eo += bm[c].nbf;
    }
    if (!meta.empty()) {
        CDS_CUDA_TRY(cudaMemcpyAsync(lay.meta, meta.data(), sizeof(OrbQP) * meta.size(),
                                     cudaMemcpyHostToDevice, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    return CDS_OK;
}

}  // namespace
}  // namespace cds

using namespace cds;

struct cds_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" int cds_batch_offsets(int32_t nmol, const cds_mol* mols, int64_t* offs) {
    if (!mols_ok(nmol, mols) || !offs) return CDS_ERR_ARG;
    BatchOffsets tot;
    std::vector<BatchOffsets> o = offsets_of(nmol, mols, &tot);
    auto put = [&](int c, const BatchOffsets& b) {
        int64_t* r = offs + (int64_t)c * CDS_BATCH_NOFF;
        r[0] = b.basis; r[1] = b.pair; r[2] = b.L; r[3] = b.piv; r[4] = b.C;
        r[5] = b.eps; r[6] = b.orb; r[7] = b.E; r[8] = b.ov; r[9] = b.p;
    };
    for (int c = 0; c < nmol; ++c) put(c, o[c]);
    put(nmol, tot);
    return CDS_OK;
}

// [CD or transform scratch | Sigma / Newton state]: the second part must
// outlive the first when a graph of the second is replayed.  Worker slots
// (optional) follow: the per-molecule tensor-core decompositions and the
// concurrent transforms.
static size_t base_bytes(int32_t nmol, const cds_mol* mols) {
    std::vector<BatchMol> bm = to_internal(nmol, mols);
    BatchOffsets tot;
    offsets_of(nmol, mols, &tot);
    size_t cd = cd_batch_workspace_bytes(nmol, bm.data());
    size_t tr = 0;
    for (int c = 0; c < nmol; ++c)
        tr = std::max(tr, cds_cd_to_mo_workspace_bytes(mols[c].nbf, mols[c].nbf, mols[c].nocc,
                                                       mols[c].max_rank, mols[c].np));
    return align_up(std::max(cd, tr)) +
           align_up(qp_batch_layout(nullptr, nmol, bm.data(), tot.orb).bytes);
}

// The tensor-core decomposition's region (CDS_PREC_OZAKI) follows the slots.
static size_t tc_cd_bytes(int32_t nmol, const cds_mol* mols, int32_t precision) {
    if (precision != CDS_PREC_OZAKI) return 0;
    std::vector<BatchMol> bm = to_internal(nmol, mols);
    return cd_tc_batch_workspace_bytes(nmol, bm.data());
}

extern "C" size_t cds_batch_workspace_bytes(int32_t nmol, const cds_mol* mols, int32_t precision) {
    if (!mols_ok(nmol, mols)) return 0;
    return base_bytes(nmol, mols) + kWorkers * worker_slot_bytes(nmol, mols) +
           tc_cd_bytes(nmol, mols, precision);
}

// The worker slots of a workspace of `bytes` bytes, or null when it has none.
static char* worker_part(void* ws, size_t bytes, int32_t nmol, const cds_mol* mols) {
    const size_t base = base_bytes(nmol, mols);
    if (bytes < base + kWorkers * worker_slot_bytes(nmol, mols)) return nullptr;
    return static_cast<char*>(ws) + base;
}

static void* qp_part(void* ws, int32_t nmol, const cds_mol* mols) {
    std::vector<BatchMol> bm = to_internal(nmol, mols);
    size_t cd = cd_batch_workspace_bytes(nmol, bm.data());
    size_t tr = 0;
    for (int c = 0; c < nmol; ++c)
        tr = std::max(tr, cds_cd_to_mo_workspace_bytes(mols[c].nbf, mols[c].nbf, mols[c].nocc,
                                                       mols[c].max_rank, mols[c].np));
    return static_cast<char*>(ws) + align_up(std::max(cd, tr));
}

extern "C" int cds_batch_cd_decompose(int32_t nmol, const cds_mol* mols, const double* xyz,
                                      const double* alpha, const int32_t* atom, double delta,
                                      int32_t scheme, int32_t precision, double* L, int32_t* piv,
                                      double* D, int32_t* M_out, void* workspace,
                                      size_t workspace_bytes, cudaStream_t stream) {
    if (!mols_ok(nmol, mols) || !xyz || !alpha || !atom || !L || !piv || !D || !M_out)
        return CDS_ERR_ARG;
    if (!(delta >= 0.0) || (scheme != CDS_SCHEME_FULL && scheme != CDS_SCHEME_ATOMIC))
        return CDS_ERR_ARG;
    if (precision == CDS_PREC_OZAKI) {
        const size_t before = base_bytes(nmol, mols) + kWorkers * worker_slot_bytes(nmol, mols);
        const size_t need = tc_cd_bytes(nmol, mols, precision);
        if (!workspace || workspace_bytes < before + need) return CDS_ERR_WORKSPACE;
        std::vector<BatchMol> bm = to_internal(nmol, mols);
        std::vector<BatchOffsets> off = offsets_of(nmol, mols, nullptr);
        return cd_batch_decompose_tc(nmol, bm.data(), off.data(), xyz, alpha, atom, delta, scheme,
                                     L, piv, D, M_out, static_cast<char*>(workspace) + before,
                                     need, stream);
    }
    if (workspace_bytes < base_bytes(nmol, mols)) return CDS_ERR_WORKSPACE;
    std::vector<BatchMol> bm = to_internal(nmol, mols);
    std::vector<BatchOffsets> off = offsets_of(nmol, mols, nullptr);
    return cd_batch_decompose(nmol, bm.data(), off.data(), xyz, alpha, atom, delta, scheme,
                              precision, L, piv, D, M_out, workspace,
                              cd_batch_workspace_bytes(nmol, bm.data()), stream);
}

extern "C" int cds_batch_cd_to_mo(int32_t nmol, const cds_mol* mols, const int32_t* M,
                                  const double* L, const double* C, const int32_t* orb,
                                  int32_t precision, double* Lov, double* Lp, void* workspace,
                                  size_t workspace_bytes, cudaStream_t stream) {
    if (!mols_ok(nmol, mols) || !M || !L || !C || !Lov || !Lp) return CDS_ERR_ARG;
    if (workspace_bytes < base_bytes(nmol, mols)) return CDS_ERR_WORKSPACE;
    std::vector<BatchOffsets> off = offsets_of(nmol, mols, nullptr);
    for (int c = 0; c < nmol; ++c)
        if (M[c] < 0 || M[c] > mols[c].max_rank) return CDS_ERR_ARG;
    if (char* slots = worker_part(workspace, workspace_bytes, nmol, mols)) {
        const size_t slot = worker_slot_bytes(nmol, mols);
        return run_workers(nmol, mols, stream, [&](int c, cudaStream_t s, int t) {
            const cds_mol& m = mols[c];
            return cds_cd_to_mo(m.nbf, m.nbf, m.nocc, M[c], L + off[c].L, C + off[c].C,
                                orb + off[c].orb, m.np, precision, Lov + off[c].ov, Lp + off[c].p,
                                slots + (size_t)t * slot, slot, s);
        });
    }
    for (int c = 0; c < nmol; ++c) {
        const cds_mol& m = mols[c];
        size_t need = cds_cd_to_mo_workspace_bytes(m.nbf, m.nbf, m.nocc, M[c], m.np);
        int st = cds_cd_to_mo(m.nbf, m.nbf, m.nocc, M[c], L + off[c].L, C + off[c].C,
                              orb + off[c].orb, m.np, precision, Lov + off[c].ov, Lp + off[c].p,
                              workspace, need, stream);
        if (st) return st;
    }
    return CDS_OK;
}

extern "C" int cds_batch_sigma2(int32_t nmol, const cds_mol* mols, const int32_t* M,
                                const double* Lov, const double* Lp, const double* eps,
                                const double* E, int32_t precision, double* sigma, double* dsigma,
                                unsigned long long* stamps, void* workspace,
                                size_t workspace_bytes, cudaStream_t stream) {
    if (!mols_ok(nmol, mols) || !M || !Lov || !Lp || !eps || !E || !sigma) return CDS_ERR_ARG;
    if (!is_split16(precision)) return CDS_ERR_UNSUPPORTED;
    if (workspace_bytes < base_bytes(nmol, mols)) return CDS_ERR_WORKSPACE;
    std::vector<BatchMol> bm = to_internal(nmol, mols);
    BatchOffsets tot;
    std::vector<BatchOffsets> off = offsets_of(nmol, mols, &tot);
    QpBatchLayout lay = qp_batch_layout(qp_part(workspace, nmol, mols), nmol, bm.data(), tot.orb);
    int st = stage_setup(nmol, bm, M, precision, lay, stream);
    if (st) return st;
    return sigma_qp_stage(nmol, bm, off, tot, M, Lov, Lp, nullptr, eps, E, precision, 0.0, 0, false,
                          sigma, dsigma, nullptr, nullptr, nullptr, nullptr, stamps, lay, stream,
                          nullptr);
}

extern "C" int cds_batch_qp_solve(int32_t nmol, const cds_mol* mols, const int32_t* M,
                                  const double* Lov, const double* Lp, const int32_t* orb,
                                  const double* eps, double conv, int32_t max_iter,
                                  int32_t precision, double* omega, double* pole, int32_t* iters,
                                  int32_t* status, unsigned long long* stamps, void* workspace,
                                  size_t workspace_bytes, cudaStream_t stream) {
    if (!mols_ok(nmol, mols) || !M || !Lov || !Lp || !orb || !eps || !omega || !pole || !iters ||
        !status || max_iter < 1 || !(conv >= 0.0))
        return CDS_ERR_ARG;
    if (!is_split16(precision)) return CDS_ERR_UNSUPPORTED;
    if (workspace_bytes < base_bytes(nmol, mols)) return CDS_ERR_WORKSPACE;
    std::vector<BatchMol> bm = to_internal(nmol, mols);
    BatchOffsets tot;
    std::vector<BatchOffsets> off = offsets_of(nmol, mols, &tot);
    QpBatchLayout lay = qp_batch_layout(qp_part(workspace, nmol, mols), nmol, bm.data(), tot.orb);
    int st = stage_setup(nmol, bm, M, precision, lay, stream);
    if (st) return st;
    int conv_all = 0;
    st = sigma_qp_stage(nmol, bm, off, tot, M, Lov, Lp, orb, eps, nullptr, precision, conv,
                        max_iter, false, nullptr, nullptr, omega, pole, iters, status, stamps, lay,
                        stream, &conv_all);
    if (st) return st;
    return conv_all ? CDS_OK : CDS_ERR_NO_CONVERGENCE;
}

extern "C" int cds_batch_graph_create(int32_t nmol, const cds_mol* mols, const int32_t* M,
                                      const double* Lov, const double* Lp, const int32_t* orb,
                                      const double* eps, const double* E, int32_t precision,
                                      double conv, int32_t max_iter, double* sigma,
                                      double* dsigma, double* omega, double* pole, int32_t* iters,
                                      int32_t* status, unsigned long long* stamps,
                                      void* workspace, size_t workspace_bytes, cds_graph** out) {
    if (!out) return CDS_ERR_ARG;
    *out = nullptr;
    if (!mols_ok(nmol, mols) || !M || !Lov || !Lp || !orb || !eps || !E || !sigma || !omega ||
        !pole || !iters || !status || max_iter < 1 || !(conv >= 0.0))
        return CDS_ERR_ARG;
    if (!is_split16(precision)) return CDS_ERR_UNSUPPORTED;
    if (workspace_bytes < base_bytes(nmol, mols)) return CDS_ERR_WORKSPACE;
    std::vector<BatchMol> bm = to_internal(nmol, mols);
    BatchOffsets tot;
    std::vector<BatchOffsets> off = offsets_of(nmol, mols, &tot);
    QpBatchLayout lay = qp_batch_layout(qp_part(workspace, nmol, mols), nmol, bm.data(), tot.orb);
    cudaStream_t s;
    CDS_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int st = stage_setup(nmol, bm, M, precision, lay, s);
    cds_graph* g = nullptr;
    if (!st) {
        g = new cds_graph();
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = CDS_ERR_CUDA;
        } else {
            st = sigma_qp_stage(nmol, bm, off, tot, M, Lov, Lp, orb, eps, E, precision, conv,
                                max_iter, true, sigma, dsigma, omega, pole, iters, status, stamps,
                                lay, s, nullptr);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (!st && e != cudaSuccess) st = CDS_ERR_CUDA;
            g->graph = graph;
            if (!st && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) st = CDS_ERR_CUDA;
        }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (st) {
        if (g) {
            if (g->exec) cudaGraphExecDestroy(g->exec);
            if (g->graph) cudaGraphDestroy(g->graph);
            delete g;
        }
        return st;
    }
    *out = g;
    return CDS_OK;
}

extern "C" int cds_graph_launch(cds_graph* g, cudaStream_t stream) {
    if (!g || !g->exec) return CDS_ERR_ARG;
    CDS_CUDA_TRY(cudaGraphLaunch(g->exec, stream));
    return CDS_OK;
}

extern "C" int cds_graph_destroy(cds_graph* g) {
    if (!g) return CDS_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return CDS_OK;
}
