// Newton quasiparticle solve (paper Eq. qpapp, Eq. iter, Eq. ps, Eq. NR).
//
// Every iteration evaluates Sigma and dSigma/dw of all still-active orbitals
// at their own current w (one self-energy pass with nE = 1, recomputing the
// MO integrals from the factors), then a single small kernel applies
//   P = 1/(1 - dSigma/dw),  w_new = w + (e_q + Sigma(w) - w) P
// in FP64 and retires orbitals with |w_new - w| <= conv.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sigma_tc.cuh"

namespace cds {

__global__ void k_qp_init(const double* __restrict__ eps, const int32_t* __restrict__ orb,
                          int32_t np, int32_t nmo, double* omega, double* pole, int32_t* iters,
                          int32_t* status, int32_t* active, int32_t* nactive) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *nactive = 0;
    if (t >= np) return;
    int q = orb[t];
    bool ok = q >= 0 && q < nmo;
    omega[t] = ok ? eps[q] : __longlong_as_double(0x7ff8000000000000LL);
    pole[t] = 1.0;
    iters[t] = 0;
    status[t] = ok ? CDS_QP_NO_CONVERGENCE : CDS_QP_NONFINITE;
    active[t] = ok ? 1 : 0;
}

__global__ void k_qp_step(const double* __restrict__ eps, const int32_t* __restrict__ orb,
                          int32_t np, const double* __restrict__ sig,
                          const double* __restrict__ dsig, double conv, double* omega,
                          double* pole, int32_t* iters, int32_t* status, int32_t* active,
                          int32_t* nactive) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np || !active[t]) return;
    double w = omega[t];
    double P = 1.0 / (1.0 - dsig[t]);
    double wn = w + (eps[orb[t]] + sig[t] - w) * P;
    iters[t] += 1;
    pole[t] = P;
    omega[t] = wn;
    if (!isfinite(wn)) {
        status[t] = CDS_QP_NONFINITE;
        active[t] = 0;
    } else if (fabs(wn - w) <= conv) {
        status[t] = CDS_QP_OK;
        active[t] = 0;
    } else {
        atomicAdd(nactive, 1);
    }
}

struct QpLayout {
    double* sig;
    double* dsig;
    int32_t* active;
    int32_t* nactive;
    void* sigma_ws;
    size_t bytes;
};

static QpLayout qp_layout(void* ws, int32_t nmo, int32_t nocc, int32_t M, int32_t np,
                          int32_t precision) {
    Carver c(ws);
    QpLayout l;
    l.sig = c.take<double>(np);
    l.dsig = c.take<double>(np);
    l.active = c.take<int32_t>(np);
    l.nactive = c.take<int32_t>(1);
    size_t sw = sigma_ws_bytes(nmo, nocc, M, np, 1, precision);
    l.sigma_ws = c.take<char>(sw);
    l.bytes = c.off;
    return l;
}

}  // namespace cds

using namespace cds;

extern "C" size_t cds_qp_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np,
                                         int32_t precision) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || M < 0 || np < 0) return 0;
    return qp_layout(nullptr, nmo, nocc, M, np, precision).bytes;
}

extern "C" int cds_qp_solve(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                            const double* Lp, const int32_t* orb, int32_t np, const double* eps,
                            double conv, int32_t max_iter, int32_t precision, double* omega,
                            double* pole, int32_t* iters, int32_t* status, void* workspace,
                            size_t workspace_bytes, cudaStream_t stream) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || M < 0 || np < 0 || np > 65535 || max_iter < 1 ||
        !(conv >= 0.0))
        return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && !is_split_tc(precision)) return CDS_ERR_UNSUPPORTED;
    if (np == 0) return CDS_OK;
    if (!Lp || !orb || !eps || !omega || !pole || !iters || !status) return CDS_ERR_ARG;
    QpLayout lay = qp_layout(workspace, nmo, nocc, M, np, precision);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    int nb = (np + 127) / 128;
    k_qp_init<<<nb, 128, 0, stream>>>(eps, orb, np, nmo, omega, pole, iters, status, lay.active,
                                      lay.nactive);
    CDS_LAUNCH_CHECK();
    int32_t h_active = np;
    for (int32_t it = 0; it < max_iter && h_active > 0; ++it) {
        // the factors do not change during the solve: split them once
        int st = sigma2_dispatch(nmo, nocc, M, Lov, Lp, np, eps, omega, 1, precision, lay.active,
                                 lay.sig, lay.dsig, lay.sigma_ws, stream, it == 0);
        if (st) return st;
        CDS_CUDA_TRY(cudaMemsetAsync(lay.nactive, 0, sizeof(int32_t), stream));
        k_qp_step<<<nb, 128, 0, stream>>>(eps, orb, np, lay.sig, lay.dsig, conv, omega, pole,
                                          iters, status, lay.active, lay.nactive);
        CDS_LAUNCH_CHECK();
        CDS_CUDA_TRY(cudaMemcpyAsync(&h_active, lay.nactive, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    return h_active > 0 ? CDS_ERR_NO_CONVERGENCE : CDS_OK;
}

// ---------------------------------------------------------------------------
// Newton from cached numerators: the same iteration, each Sigma(w) evaluated
// by sigma2_cached from the numerators a cds_sigma2_diag_cache call stored
// (no factors needed).
// ---------------------------------------------------------------------------
namespace cds {
static QpLayout qp_cached_layout(void* ws, int32_t nmo, int32_t nocc, int32_t np) {
    Carver c(ws);
    QpLayout l;
    l.sig = c.take<double>(np);
    l.dsig = c.take<double>(np);
    l.active = c.take<int32_t>(np);
    l.nactive = c.take<int32_t>(1);
    l.sigma_ws = c.take<char>(std::max(tc_cached_workspace_bytes(nmo, nocc, np),
                                       fp64_cached_workspace_bytes(nmo, nocc, np)));
    l.bytes = c.off;
    return l;
}

// Sigma at omega from a numerator cache of either form.
static int sigma_from_cache(int32_t precision, int32_t nmo, int32_t nocc, int32_t np,
                            const double* eps, const double* omega, const QpLayout& lay,
                            const void* cache, cudaStream_t stream, bool first) {
    if (precision == CDS_PREC_FP64)
        return sigma2_cached_fp64(nmo, nocc, np, eps, omega, lay.active,
                                  static_cast<const double*>(cache), lay.sig, lay.dsig,
                                  static_cast<double*>(lay.sigma_ws), stream);
    return sigma2_cached(nmo, nocc, np, eps, omega, lay.active, static_cast<const float*>(cache),
                         lay.sig, lay.dsig, lay.sigma_ws, stream, first);
}
}  // namespace cds

extern "C" size_t cds_qp_cached_workspace_bytes(int32_t nmo, int32_t nocc, int32_t np) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || np < 0) return 0;
    return qp_cached_layout(nullptr, nmo, nocc, np).bytes;
}

extern "C" int cds_qp_solve_cached(int32_t nmo, int32_t nocc, int32_t np, const int32_t* orb,
                                   const double* eps, double conv, int32_t max_iter,
                                   const void* cache, size_t cache_bytes, int32_t precision,
                                   double* omega,
                                   double* pole, int32_t* iters, int32_t* status,
                                   void* workspace, size_t workspace_bytes,
                                   cudaStream_t stream) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || np < 0 || np > 65535 || max_iter < 1 ||
        !(conv >= 0.0))
        return CDS_ERR_ARG;
    if (np == 0) return CDS_OK;
    if (!orb || !eps || !omega || !pole || !iters || !status || !cache) return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && !is_split_tc(precision)) return CDS_ERR_UNSUPPORTED;
    if (cache_bytes < cds_sigma2_cache_bytes(nmo, nocc, np, precision)) return CDS_ERR_ARG;
    QpLayout lay = qp_cached_layout(workspace, nmo, nocc, np);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    const int nb = (np + 127) / 128;
    k_qp_init<<<nb, 128, 0, stream>>>(eps, orb, np, nmo, omega, pole, iters, status, lay.active,
                                      lay.nactive);
    CDS_LAUNCH_CHECK();
    int32_t h_active = np;
    for (int32_t it = 0; it < max_iter && h_active > 0; ++it) {
        int st = sigma_from_cache(precision, nmo, nocc, np, eps, omega, lay, cache, stream,
                                  it == 0);
        if (st) return st;
        CDS_CUDA_TRY(cudaMemsetAsync(lay.nactive, 0, sizeof(int32_t), stream));
        k_qp_step<<<nb, 128, 0, stream>>>(eps, orb, np, lay.sig, lay.dsig, conv, omega, pole,
                                          iters, status, lay.active, lay.nactive);
        CDS_LAUNCH_CHECK();
        CDS_CUDA_TRY(cudaMemcpyAsync(&h_active, lay.nactive, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    return h_active > 0 ? CDS_ERR_NO_CONVERGENCE : CDS_OK;
}

// ---------------------------------------------------------------------------
// Safeguarded Newton (not in the paper): every pole of Sigma_qq lies at
// e_i + e_j - e_a or e_a + e_b - e_i, and between neighbouring poles
// f(w) = w - e_q - Sigma(w) rises from -inf to +inf (all residues >= 0), so
// the interval around e_q holds one root.  The Newton step is kept while it
// stays inside the current bracket of that root, otherwise the step bisects.
// ---------------------------------------------------------------------------
namespace cds {
namespace {

// Nearest poles below / above e (strict).  Poles are s - z with s a sum of
// two occupied (z virtual) or two virtual (z occupied) energies; with the
// pair sums sorted, for each z the pair sum that brings s - z closest to e on
// either side is found by binary search (then checked in the same floating
// point as the poles are formed, (e_x + e_y) - e_z).
struct PoleSets {
    std::vector<double> soo, svv, eo, ev;   // sorted pair sums and energies
};

PoleSets pole_sets(const std::vector<double>& e, int32_t nocc) {
    PoleSets p;
    p.eo.assign(e.begin(), e.begin() + nocc);
    p.ev.assign(e.begin() + nocc, e.end());
    for (double x : p.eo)
        for (double y : p.eo) p.soo.push_back(x + y);
    for (double x : p.ev)
        for (double y : p.ev) p.svv.push_back(x + y);
    std::sort(p.soo.begin(), p.soo.end());
    std::sort(p.svv.begin(), p.svv.end());
    return p;
}

void pole_bracket_host(const PoleSets& ps, double e, double* lo, double* hi) {
    double L = -INFINITY, H = INFINITY;
    auto scan = [&](const std::vector<double>& S, const std::vector<double>& Z) {
        if (S.empty()) return;
        for (double z : Z) {
            // below: the largest s with s - z < e
            auto it = std::lower_bound(S.begin(), S.end(), e + z);
            for (auto k = it; k != S.end() && *k - z < e; ++k) L = std::max(L, *k - z);
            while (it != S.begin()) {
                --it;
                if (*it - z < e) { L = std::max(L, *it - z); break; }
            }
            // above: the smallest s with s - z > e
            auto jt = std::upper_bound(S.begin(), S.end(), e + z);
            for (auto k = jt; k != S.begin() && *(k - 1) - z > e; --k) H = std::min(H, *(k - 1) - z);
            for (; jt != S.end(); ++jt)
                if (*jt - z > e) { H = std::min(H, *jt - z); break; }
        }
    };
    scan(ps.soo, ps.ev);   // e_i + e_j - e_a
    scan(ps.svv, ps.eo);   // e_a + e_b - e_i
    *lo = std::isfinite(L) ? L : e - 10.0;
    *hi = std::isfinite(H) ? H : e + 10.0;
}

__global__ void k_qp_step_bracketed(const double* __restrict__ eps, const int32_t* __restrict__ orb,
                                    int32_t np, const double* __restrict__ sig,
                                    const double* __restrict__ dsig, double conv, double* omega,
                                    double* pole, double* brk, int32_t* iters, int32_t* status,
                                    int32_t* active, int32_t* nactive) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np || !active[t]) return;
    const double w = omega[t], eq = eps[orb[t]];
    const double f = w - eq - sig[t], fp = 1.0 - dsig[t];
    double lo = brk[2 * t], hi = brk[2 * t + 1];
    if (f < 0.0) lo = w; else hi = w;
    double wn = w - f / fp;
    if (!(lo < wn && wn < hi)) wn = 0.5 * (lo + hi);
    brk[2 * t] = lo;
    brk[2 * t + 1] = hi;
    iters[t] += 1;
    pole[t] = 1.0 / fp;
    omega[t] = wn;
    if (!isfinite(wn)) {
        status[t] = CDS_QP_NONFINITE;
        active[t] = 0;
    } else if (fabs(wn - w) <= conv) {
        status[t] = CDS_QP_OK;
        active[t] = 0;
    } else {
        atomicAdd(nactive, 1);
    }
}

// Initial brackets of every orbital (host, from the orbital energies), copied
// to bracket[np][2] on the device.  Blocking.
int upload_brackets(int32_t nmo, int32_t nocc, int32_t np, const int32_t* orb, const double* eps,
                    double* bracket, cudaStream_t stream) {
    std::vector<double> e(nmo), br(2 * (size_t)np);
    std::vector<int32_t> o(np);
    CDS_CUDA_TRY(cudaMemcpyAsync(e.data(), eps, sizeof(double) * nmo, cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaMemcpyAsync(o.data(), orb, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    const PoleSets ps = pole_sets(e, nocc);
    for (int32_t t = 0; t < np; ++t) {
        const double eq = (o[t] >= 0 && o[t] < nmo) ? e[o[t]] : NAN;
        pole_bracket_host(ps, eq, &br[2 * t], &br[2 * t + 1]);
    }
    CDS_CUDA_TRY(cudaMemcpyAsync(bracket, br.data(), sizeof(double) * 2 * np,
                                 cudaMemcpyHostToDevice, stream));
    CDS_CUDA_TRY(cudaStreamSynchronize(stream));   // br is a host temporary
    return CDS_OK;
}

}  // namespace
}  // namespace cds

extern "C" int cds_qp_solve_bracketed(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                                      const double* Lp, const int32_t* orb, int32_t np,
                                      const double* eps, double conv, int32_t max_iter,
                                      int32_t precision, double* omega, double* pole,
                                      int32_t* iters, int32_t* status, double* bracket,
                                      void* workspace, size_t workspace_bytes,
                                      cudaStream_t stream) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || M < 0 || np < 0 || np > 65535 || max_iter < 1 ||
        !(conv >= 0.0))
        return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && !is_split_tc(precision)) return CDS_ERR_UNSUPPORTED;
    if (np == 0) return CDS_OK;
    if (!Lp || !orb || !eps || !omega || !pole || !iters || !status || !bracket)
        return CDS_ERR_ARG;
    QpLayout lay = qp_layout(workspace, nmo, nocc, M, np, precision);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    int st = upload_brackets(nmo, nocc, np, orb, eps, bracket, stream);
    if (st) return st;
    const int nb = (np + 127) / 128;
    k_qp_init<<<nb, 128, 0, stream>>>(eps, orb, np, nmo, omega, pole, iters, status, lay.active,
                                      lay.nactive);
    CDS_LAUNCH_CHECK();
    int32_t h_active = np;
    for (int32_t it = 0; it < max_iter && h_active > 0; ++it) {
        st = sigma2_dispatch(nmo, nocc, M, Lov, Lp, np, eps, omega, 1, precision, lay.active,
                             lay.sig, lay.dsig, lay.sigma_ws, stream, it == 0);
        if (st) return st;
        CDS_CUDA_TRY(cudaMemsetAsync(lay.nactive, 0, sizeof(int32_t), stream));
        k_qp_step_bracketed<<<nb, 128, 0, stream>>>(eps, orb, np, lay.sig, lay.dsig, conv, omega,
                                                    pole, bracket, iters, status, lay.active,
                                                    lay.nactive);
        CDS_LAUNCH_CHECK();
        CDS_CUDA_TRY(cudaMemcpyAsync(&h_active, lay.nactive, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    return h_active > 0 ? CDS_ERR_NO_CONVERGENCE : CDS_OK;
}

extern "C" int cds_qp_solve_bracketed_cached(int32_t nmo, int32_t nocc, int32_t np,
                                             const int32_t* orb, const double* eps, double conv,
                                             int32_t max_iter, const void* cache,
                                             size_t cache_bytes, int32_t precision,
                                             double* omega, double* pole,
                                             int32_t* iters, int32_t* status, double* bracket,
                                             void* workspace, size_t workspace_bytes,
                                             cudaStream_t stream) {
    if (nmo <= 0 || nocc < 0 || nocc > nmo || np < 0 || np > 65535 || max_iter < 1 ||
        !(conv >= 0.0))
        return CDS_ERR_ARG;
    if (np == 0) return CDS_OK;
    if (!orb || !eps || !omega || !pole || !iters || !status || !bracket || !cache)
        return CDS_ERR_ARG;
    if (precision != CDS_PREC_FP64 && !is_split_tc(precision)) return CDS_ERR_UNSUPPORTED;
    if (cache_bytes < cds_sigma2_cache_bytes(nmo, nocc, np, precision)) return CDS_ERR_ARG;
    QpLayout lay = qp_cached_layout(workspace, nmo, nocc, np);
    if (!workspace || workspace_bytes < lay.bytes) return CDS_ERR_WORKSPACE;
    // brackets on the host from the orbital energies
    int st0 = upload_brackets(nmo, nocc, np, orb, eps, bracket, stream);
    if (st0) return st0;
    const int nb = (np + 127) / 128;
    k_qp_init<<<nb, 128, 0, stream>>>(eps, orb, np, nmo, omega, pole, iters, status, lay.active,
                                      lay.nactive);
    CDS_LAUNCH_CHECK();
    int32_t h_active = np;
    for (int32_t it = 0; it < max_iter && h_active > 0; ++it) {
        int st = sigma_from_cache(precision, nmo, nocc, np, eps, omega, lay, cache, stream,
                                  it == 0);
        if (st) return st;
        CDS_CUDA_TRY(cudaMemsetAsync(lay.nactive, 0, sizeof(int32_t), stream));
        k_qp_step_bracketed<<<nb, 128, 0, stream>>>(eps, orb, np, lay.sig, lay.dsig, conv, omega,
                                                    pole, bracket, iters, status, lay.active,
                                                    lay.nactive);
        CDS_LAUNCH_CHECK();
        CDS_CUDA_TRY(cudaMemcpyAsync(&h_active, lay.nactive, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, stream));
        CDS_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    return h_active > 0 ? CDS_ERR_NO_CONVERGENCE : CDS_OK;
}
