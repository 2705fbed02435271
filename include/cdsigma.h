/*
 * cdsigma -- Cholesky-factorised second-order electron propagator on one GPU.
 *
 * C ABI of the GPU library (libcdsigma.so, sm_103a).  Every call takes plain
 * pointers and sizes; "device" arrays live in GPU memory owned by the caller,
 * "host" arrays in host memory owned by the caller.  The library never frees
 * or keeps caller memory.  Where a call needs scratch memory the caller passes
 * a device workspace whose size the matching *_workspace_bytes() reports.
 *
 * Errors: every call returns a cds_status (0 = success).  Argument errors are
 * detected before any launch and leave outputs untouched.  CUDA launch errors
 * return CDS_ERR_CUDA.  Nothing is signalled by exceptions, traps or device
 * asserts; device-side failures are written to status words the caller reads.
 *
 * Streams: calls enqueue work on the given stream.  Calls documented as
 * "blocking" synchronise that stream before returning because their control
 * flow depends on device results (the Cholesky rank, Newton convergence).
 *
 * Conventions shared by all calls
 *  - Basis: N normalised s-type Gaussians; xyz[N][3] (bohr), alpha[N],
 *    atom[N] (centre index of each function).
 *  - Product densities I = (mu, nu), mu <= nu (paper Sec. II.A), packed as
 *    I = nu*(nu+1)/2 + mu; npair = N*(N+1)/2.
 *  - Cholesky vectors L[K][I], K = 0..M-1, row-major (vector-major).
 *  - MO coefficients C[N][nmo] row-major, column p = MO p; eps[nmo] ascending,
 *    the first nocc orbitals occupied.
 *  - MO factors (paper Eq. transformation): Lov[i][a][K] = B^K_{i,nocc+a}
 *    and Lp[t][r][K] = B^K_{orb[t], r}; K is the innermost (contiguous) index.
 */
#ifndef CDSIGMA_H
#define CDSIGMA_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CDS_OK = 0,
    CDS_ERR_ARG = 1,            /* invalid argument (size, null pointer, range) */
    CDS_ERR_CUDA = 2,           /* a CUDA runtime call or launch failed */
    CDS_ERR_NOT_PD = 3,         /* residual diagonal below -1e-10 * max initial diagonal */
    CDS_ERR_RANK_CAP = 4,       /* more than max_rank Cholesky vectors needed */
    CDS_ERR_NO_CONVERGENCE = 5, /* a Newton solve did not converge in max_iter */
    CDS_ERR_WORKSPACE = 6,      /* workspace smaller than *_workspace_bytes() */
    CDS_ERR_UNSUPPORTED = 7,    /* device or precision mode not supported */
    CDS_ERR_TIMEOUT = 8,        /* a bounded device-side wait gave up */
    CDS_ERR_CAPACITY = 9        /* a fixed-capacity output or static scratch is too small */
} cds_status;

typedef enum { CDS_SCHEME_FULL = 0, CDS_SCHEME_ATOMIC = 1 } cds_scheme;

/* Arithmetic of the J-contractions in sigma2 / qp_solve.
 * FP64: binary64 throughout (CUDA cores).
 * BF16X3 / FP16X3 / TF32X3: each factor split s*x = hi + lo with hi, lo bf16
 *   (s = 1), fp16 (s = a power of two with max|s x| <= 1024) or tf32 (s = 1,
 *   FP32 containers); the products hi*hi + hi*lo + lo*hi run on tcgen05
 *   tensor cores with fp32 accumulation.  Denominators are double-fp32
 *   pairs, per-element sums fp32, cross-tile sums and the Newton step fp64.
 *   FP16X3 carries ~22 significant bits per factor, BF16X3 ~17, TF32X3 ~22.
 *   TF32X3 serves the single-molecule self-energy, Newton and adjoint calls
 *   and the transform; MP2 and the batched calls take BF16X3 / FP16X3. */
typedef enum {
    CDS_PREC_FP64 = 0,
    CDS_PREC_BF16X3 = 2,
    CDS_PREC_FP16X3 = 3,
    CDS_PREC_F32X2 = 4,  /* decomposition and transform: (hi, lo) float pairs with exact
                            product and sum errors, ~2^-44 relative per operation, on the
                            FP32 units */
    CDS_PREC_TF32X3 = 5, /* self-energy, Newton, adjoint and transform: tcgen05 tensor
                            cores, each operand split into TF32 hi + lo, hi.hi + hi.lo +
                            lo.hi with FP32 accumulation, ~2^-21 relative per product
                            (BF16X3: ~2^-17) */
    CDS_PREC_OZAKI = 6   /* transform: tcgen05 tensor cores with exact slice products
                            (rows cut into six 7-bit BF16 digits below a power-of-two
                            scale, 21 slice pairs, exact FP32 sums for nbf <= 1040):
                            ~2^-42 of the row scales, for ill-conditioned C */
} cds_precision;

/* Newton status per orbital (paper Eq. NR). */
enum { CDS_QP_OK = 0, CDS_QP_NO_CONVERGENCE = 1, CDS_QP_NONFINITE = 2 };

/* Library version (major*10000 + minor*100 + patch). */
int cds_version(void);

/* Static description of a status code; never NULL. */
const char* cds_errstr(int status);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all streams); monotone, thread-safe. */
unsigned long long cds_launch_count(void);

/* Check of the bounded device-side wait (no counterpart in the paper).  Every
 * wait of the tensor-core kernels on an mbarrier gives up after a limit (2 s)
 * and writes CDS_ERR_TIMEOUT to the call's error word instead of hanging or
 * trapping.  This call runs that same wait on a barrier phase that nothing
 * completes, with a limit of `seconds` (0 < seconds <= 2), so that it must
 * give up; the kernel then returns normally.  err: device int32 error word
 * (caller-owned).  Blocking; returns the word (CDS_ERR_TIMEOUT when the wait
 * gave up as designed), or CDS_ERR_ARG / CDS_ERR_CUDA. */
int cds_wait_check(double seconds, int32_t* err, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Electron-repulsion integrals over s-type Gaussians (paper Sec. II.A,
 * Eq. integral):  (rho_I|rho_J) = 2 pi^(5/2)/(p q sqrt(p+q)) K_I K_J F0(T).
 * ---------------------------------------------------------------------- */

/* D[I] = (rho_I|rho_I) for all npair pairs.
 * xyz, alpha: device, as above.  D: device [npair] fp64 output. */
int cds_eri_diag(int32_t nbf, const double* xyz, const double* alpha, double* D,
                 cudaStream_t stream);

/* cols[c][I] = (rho_I|rho_{piv[c]}) for c < ncol and all I.
 * piv: device [ncol] int32 packed indices in [0, npair).  cols: device
 * [ncol][npair] fp64 output.  Out-of-range pivots return CDS_ERR_ARG only when
 * detectable on the host (ncol < 0); the kernel writes NaN columns for
 * out-of-range device indices. */
int cds_eri_columns(int32_t nbf, const double* xyz, const double* alpha,
                    const int32_t* piv, int32_t ncol, double* cols, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Threshold-delta diagonal-pivoted incomplete Cholesky decomposition of the
 * ERI supermatrix (paper Sec. II.A, Eq. gs_coulomb, Eq. CD, Eq. stricterr),
 * ERI columns generated on the fly.
 *   pivot: largest residual diagonal D_I over the candidate set; candidates
 *          within 1e-12 * max(initial D) of it (and above delta_eff) are tied
 *          and the lowest packed index wins;
 *   stop:  when every candidate residual is <= delta_eff,
 *          delta_eff = max(delta, npair * 2^-52 * max(initial D));
 *   the chosen pair's residual is then set to exactly 0;
 *   scheme FULL: all pairs are candidates; ATOMIC: only pairs with
 *          atom[mu] == atom[nu] (atomic-CD pivot restriction, paper Sec. II.A).
 * ---------------------------------------------------------------------- */

/* Workspace needed by cds_cd_decompose for a basis of nbf functions. */
size_t cds_cd_workspace_bytes(int32_t nbf);

/* Blocking.  precision: CDS_PREC_FP64 (binary64 throughout) or CDS_PREC_F32X2
 * (the projections sum_K L^K_I L^K_P in float-pair arithmetic, ~2^-44 relative
 * per step, with the vectors held as float pairs while the decomposition runs;
 * integral columns, L^k, the residual diagonal and the pivot search stay FP64;
 * L is returned in FP64 either way).  F32X2 also speculates: one streaming
 * pass forms the projections of the step's pivot and of a few likely next
 * pivots (the largest residuals of other blocks; cds_cd_candidates() in all),
 * and the following steps
 * whose pivots are among them reuse those projections plus the few vectors
 * made since.  The pivot rule and the result are those of the plain
 * algorithm; only the grouping of each sum differs (see cds_cd_stats).
 * CDS_PREC_OZAKI: the F32X2 decomposition whose streaming passes run on the
 * tcgen05 tensor cores for 32 candidates at once (a pass serves up to 64
 * steps): each stored element is also kept as a 56-bit fixed-point number
 * below its pair's power-of-two scale (> sqrt of the initial diagonal), in
 * eight exact BF16 slices of 7 bits, and the pass multiplies these slices
 * with exact products and exact FP32 sums (36 slice pairs; at most 2048 x 512
 * pairs after screening, the candidate search holding the block maxima in
 * shared memory, else CDS_ERR_UNSUPPORTED); the steps
 * in between add the vectors made since in float pairs.  Pairs whose initial
 * diagonal is below 1e-40 of the largest are screened out (Schwarz: each of
 * their vector elements is below 1e-20 of the square root of the largest
 * diagonal); they return L = 0 and D = D0, and the steps run on the other
 * pairs only.  The pivot sequence is the FP64 one (tested at C60 size).  Its
 * workspace is cds_cd_workspace_bytes_prec (the slice store takes 16 bytes
 * and the compact vectors 8 bytes per pair and vector of max_rank).
 * Inputs (device): xyz, alpha, atom.  Outputs (device, caller-owned):
 *   L     [max_rank][npair] fp64, rows 0..M-1 written;
 *   piv   [max_rank] int32 packed pivot index of each vector;
 *   D     [npair] fp64 residual diagonal after the last step (the error
 *         diagonal D_II of Eq. error_approx).
 * Outputs (host): *M_out = number of vectors, *delta_eff_out (may be NULL).
 * Returns CDS_ERR_RANK_CAP if max_rank vectors did not reach delta (L, piv
 * then hold the first max_rank vectors and *M_out = max_rank), CDS_ERR_NOT_PD
 * on a negative residual beyond roundoff. */
int cds_cd_decompose(int32_t nbf, const double* xyz, const double* alpha,
                     const int32_t* atom, double delta, int32_t scheme, int32_t max_rank,
                     int32_t precision, double* L, int32_t* piv, double* D, int32_t* M_out,
                     double* delta_eff_out, void* workspace, size_t workspace_bytes,
                     cudaStream_t stream);

/* Work counters of the last cds_cd_decompose that used this workspace
 * (blocking; reads the workspace's control block).  passes = steps that
 * streamed the stored vectors, streamed = vectors read by those passes in
 * total, extra = vectors added to a candidate projection by the steps in
 * between (F32X2 speculative projections: a pass forms the projections of
 * the pivot and of a few likely next pivots; a later step whose pivot is
 * among them adds only the vectors made since).  FP64 streams at every step:
 * passes = M, streamed = M(M-1)/2, extra = 0. */
int cds_cd_stats(int32_t nbf, const void* workspace, int32_t precision, int32_t* passes,
                 int64_t* streamed, int64_t* extra, cudaStream_t stream);

/* Pairs the last cds_cd_decompose in this workspace kept after screening
 * (blocking): CDS_PREC_OZAKI leaves out pairs whose initial diagonal is below
 * 1e-40 of the largest; FP64 and F32X2 keep all npair. */
int cds_cd_live_pairs(int32_t nbf, const void* workspace, int32_t precision, int64_t* nlive,
                      cudaStream_t stream);

/* Candidate pivots whose projections one streaming pass of the given
 * precision forms (host only; a later step continues the pass while its
 * pivot is among them and the pass is not full -- 4 steps for F32X2, 64 for
 * OZAKI): 4 for F32X2, 32 for OZAKI, 1 for FP64 (every step streams). */
int cds_cd_candidates(int32_t precision);

/* Workspace of cds_cd_decompose for one precision and max_rank (OZAKI holds a
 * slice store of max_rank columns; cds_cd_workspace_bytes covers FP64 and
 * F32X2 for any max_rank). */
size_t cds_cd_workspace_bytes_prec(int32_t nbf, int32_t max_rank, int32_t precision);

/* Kernel timing of the OZAKI decomposition's projection GEMM (the tcgen05
 * kernel that forms a pass's candidate projections; Eq. gs_coulomb).  While
 * enabled, every cds_cd_decompose / cds_cd_decompose_to_mo with
 * CDS_PREC_OZAKI records a CUDA event pair around each GEMM launch on the
 * stream the launch uses (not under stream capture) and adds the elapsed
 * times of the steps that ran to process-wide totals.  The GEMM is enqueued
 * at every step and returns at once unless the step starts a pass, so the
 * totals include those early returns.  cds_cd_gemm_timing(enable) switches it
 * and clears the totals; cds_cd_gemm_time reads them (*ms summed, *launches
 * counted).  Host only; not for concurrent decompositions.  Returns CDS_OK
 * (CDS_ERR_ARG on a NULL pointer). */
int cds_cd_gemm_timing(int32_t enable);
int cds_cd_gemm_time(double* ms, int64_t* launches);

/* ------------------------------------------------------------------------
 * The decomposition over contracted Cartesian Gaussian shells (the paper's
 * basis sets are contracted shells with higher angular momentum, Sec. III;
 * Eq. integral is the same Coulomb integral over their products).  Basis
 * function f (device arrays): centre xyz[f][3], Cartesian exponents
 * lmn[f][3] with l + m + n <= 2 (s, p, Cartesian d), primitives
 * [start[f], start[f+1]) of exps[] / coefs[] (the coefficients carry the
 * function's normalisation): chi_f = sum_k coefs[k] x^l y^m z^n exp(-exps[k] r^2)
 * about its centre.  Integrals: McMurchie-Davidson (Hermite expansion and
 * Hermite Coulomb integrals) in FP64, one thread per pair; the pivot rule,
 * stop rule, candidate sets, outputs and errors are those of
 * cds_cd_decompose (precision FP64; workspace cds_cd_workspace_bytes).
 * CDS_ERR_UNSUPPORTED for a function beyond d.  Blocking.
 * ---------------------------------------------------------------------- */
int cds_cd_decompose_shells(int32_t nbf, const double* xyz, const int32_t* lmn,
                            const int32_t* start, const double* exps, const double* coefs,
                            const int32_t* atom, double delta, int32_t scheme, int32_t max_rank,
                            double* L, int32_t* piv, double* D, int32_t* M_out,
                            double* delta_eff_out, void* workspace, size_t workspace_bytes,
                            cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Allocation-free Cholesky decomposition.  The paper has no counterpart: this
 * is a service for callers that cannot allocate device memory where they call
 * (GPU memory owned by another runtime or pool they cannot reach, a plugin
 * that must not grow the device footprint).  Same arguments, semantics and
 * results as cds_cd_decompose, without the workspace: the scratch is a fixed
 * device array inside the library (CDS_CD_STATIC_SCRATCH_BYTES, held on every
 * GPU that loads the library until the process exits).  The call allocates
 * nothing (no cudaMalloc, no library allocator).  Every call made outside a
 * stream capture resolves the array's device address with the device current;
 * a call inside a capture reuses the last one resolved on that device
 * (CDS_ERR_UNSUPPORTED if none), so make the first call on a device before
 * any stream capture.  Calls share the array: two calls
 * whose GPU work overlaps race.  Returns CDS_ERR_CAPACITY when the basis needs
 * more scratch than the array holds (nbf > cds_cd_static_max_nbf()).
 * ---------------------------------------------------------------------- */

#define CDS_CD_STATIC_SCRATCH_BYTES (4u << 20)

/* Blocking; see cds_cd_decompose for the arguments. */
int cds_cd_decompose_static(int32_t nbf, const double* xyz, const double* alpha,
                            const int32_t* atom, double delta, int32_t scheme, int32_t max_rank,
                            double* L, int32_t* piv, double* D, int32_t* M_out,
                            double* delta_eff_out, cudaStream_t stream);

/* Largest basis the allocation-free entry point accepts (host only). */
int cds_cd_static_max_nbf(void);

/* ------------------------------------------------------------------------
 * AO -> MO transform of the Cholesky vectors (paper Eq. transformation):
 *   B^K_pq = sum_{mu,nu} C_{mu p} L^K_{mu nu} C_{nu q},  fp64.
 * ---------------------------------------------------------------------- */

/* Host only.  Workspace of cds_cd_to_mo for M vectors.  The tensor-core forms
 * transform the vectors in batches of max(32, about 65,536 / nbf rounded up
 * to 32) vectors, at most M, so the workspace grows with M up to that batch;
 * a workspace sized for a larger M serves any smaller one. */
size_t cds_cd_to_mo_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc, int32_t M, int32_t np);

/* Asynchronous (FP64, F32X2) or blocking (TF32X3, BF16X3: the tensor-core
 * kernels' error word is read at the end, CDS_ERR_TIMEOUT if a bounded wait
 * gave up).  L: device [M][npair]; C: device [nbf][nmo]; orb: device [np]
 * int32 MO indices in [0, nmo).  precision: CDS_PREC_FP64, CDS_PREC_F32X2,
 * CDS_PREC_TF32X3, CDS_PREC_BF16X3 or CDS_PREC_OZAKI (the last three on sm_103
 * only, OZAKI for nbf <= 1040; else CDS_ERR_UNSUPPORTED).  TF32X3 / BF16X3
 * accumulate in FP32 and lose ~u |C_p|_1 |C_q|_1 of each element (u = 2^-21
 * / 2^-17): they return CDS_ERR_UNSUPPORTED when u max_q |C_q|_1^2 > 2^-8
 * (ill-conditioned C; use CDS_PREC_OZAKI or CDS_PREC_F32X2 there).  Outputs (device, fp64): Lov [nocc][nmo-nocc][M],
 * Lp [np][nmo][M] (Lp may be NULL when np == 0). */
int cds_cd_to_mo(int32_t nbf, int32_t nmo, int32_t nocc, int32_t M, const double* L,
                 const double* C, const int32_t* orb, int32_t np, int32_t precision,
                 double* Lov, double* Lp, void* workspace, size_t workspace_bytes,
                 cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Atomic Cholesky basis and the V-approximation (paper Sec. II.A, atomic CD;
 * Eq. int_approx, Eq. error_approx).  For every unique atom (the exponents
 * of the functions on one centre, in basis order) the isolated atom's one-
 * centre ERI matrix is decomposed by the pivot rule of cds_cd_decompose at
 * delta; its pivots, on every atom of that type, are the basis densities
 * rho~_K.  With the metric V_KL = (rho~_K|rho~_L) = L_m L_m^T,
 *   B = L_m^-1 (rho~|rho_I),  (rho_I|rho_J) ~ sum_K B^K_I B^K_J,
 * the factor form of Eq. CD: B goes to cds_cd_to_mo in place of L (M = naux).
 * ---------------------------------------------------------------------- */

/* Workspace of cds_acd_aux_pairs for atoms of at most max_atom_funcs functions. */
size_t cds_acd_workspace_bytes(int32_t max_atom_funcs);

/* Blocking.  Inputs (device): alpha [nbf], atom [nbf] (centre of each
 * function).  Output (host, caller-owned): aux [capacity] packed pair indices
 * of the basis densities, centres ascending, each centre's in its type's
 * pivot order; *naux their number.  CDS_ERR_CAPACITY if more than capacity
 * (*naux still set).  Each isolated atom is decomposed in the caller's
 * workspace (cds_acd_workspace_bytes of the largest atom), so calls on
 * different workspaces may overlap. */
int cds_acd_aux_pairs(int32_t nbf, const double* alpha, const int32_t* atom, double delta,
                      int32_t* aux, int32_t capacity, int32_t* naux, void* workspace,
                      size_t workspace_bytes, cudaStream_t stream);

size_t cds_ri_workspace_bytes(int32_t nbf, int32_t naux, int32_t precision);

/* Blocking.  Inputs (device): xyz, alpha as cds_cd_decompose; aux [naux]
 * packed pair indices of the basis densities.  Output (device, caller-
 * owned): B [naux][npair].  The factors come from forward substitution with
 * the basis as fixed pivots (B restricted to the basis' columns is L_m^T, so
 * the metric factor is formed on the way).  precision: CDS_PREC_FP64, or
 * CDS_PREC_F32X2 (integrals and the substitution in float pairs; B ~1e-9 of
 * max|B| from the FP64 result; workspace holds naux x npair float pairs).
 * CDS_ERR_NOT_PD if the metric is not positive definite to working precision
 * (a Cholesky pivot at or below 1e-12 x its diagonal, e.g. a density listed
 * twice); CDS_ERR_ARG on an index outside the basis. */
int cds_ri_factors(int32_t nbf, const double* xyz, const double* alpha, const int32_t* aux,
                   int32_t naux, int32_t precision, double* B, void* workspace,
                   size_t workspace_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Decomposition and transform in one call.  Runs cds_cd_decompose
 * (cd_precision: CDS_PREC_F32X2 or CDS_PREC_OZAKI) and cds_cd_to_mo
 * (tr_precision: CDS_PREC_F32X2, CDS_PREC_TF32X3, CDS_PREC_BF16X3 or
 * CDS_PREC_OZAKI) with the transform of each batch of 32 finished vectors
 * overlapped with the decomposition of the next ones, on two library streams
 * (the decomposition's at the highest priority), joined to `stream` on
 * return.  The results are those of the two calls in sequence.
 * Inputs and outputs as cds_cd_decompose and cds_cd_to_mo, except:
 *   Lov  [nocc][nmo-nocc][M] and Lp [np][nmo][M] are written compact for the
 *        final rank M, into caller buffers of room for max_rank in place of M;
 *   the workspace (cds_cd_decompose_to_mo_workspace_bytes) holds both calls'
 *        workspaces and max_rank-strided staging copies of Lov and Lp.
 * Blocking, like cds_cd_decompose.  The two library streams belong to the
 * device, so calls from several host threads share them (their work
 * interleaves in stream order).  On the library stream the tensor-core
 * decomposition replays its 32-step chunks as a CUDA graph (CDS_TUNE_CD_GRAPH);
 * CDS_TUNE_PIPE_SPLIT divides the SMs between the two streams.
 * ---------------------------------------------------------------------- */
size_t cds_cd_decompose_to_mo_workspace_bytes(int32_t nbf, int32_t nmo, int32_t nocc,
                                              int32_t max_rank, int32_t np, int32_t cd_precision);
int cds_cd_decompose_to_mo(int32_t nbf, const double* xyz, const double* alpha,
                           const int32_t* atom, double delta, int32_t scheme, int32_t max_rank,
                           const double* C, int32_t nmo, int32_t nocc, const int32_t* orb,
                           int32_t np, int32_t tr_precision, int32_t cd_precision, double* L,
                           int32_t* piv, double* D,
                           int32_t* M_out,
                           double* delta_eff_out, double* Lov, double* Lp, void* workspace,
                           size_t workspace_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Diagonal second-order self-energy (paper Eq. SE) and its energy derivative
 * for np orbitals orb[t] at nE energies each:
 *   sigma[t][e]  = Sigma_qq(E[t][e]),  dsigma[t][e] = dSigma_qq/dE (analytic),
 * MO integrals recomputed tile by tile from the factors and never stored.
 * Inputs are the outputs of cds_cd_to_mo plus eps (device [nmo]).
 * ---------------------------------------------------------------------- */

size_t cds_sigma2_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np,
                                  int32_t nE, int32_t precision);

/* Asynchronous.  Lp holds the factor rows of the np orbitals (Sigma_qq
 * depends on q only through them); E: device [np][nE]; sigma, dsigma: device
 * [np][nE] outputs (dsigma may be NULL).  precision: cds_precision.
 * 1 <= nE <= 4096, np <= 65535. */
int cds_sigma2_diag(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                    const double* Lp, int32_t np, const double* eps, const double* E,
                    int32_t nE, int32_t precision, double* sigma, double* dsigma,
                    void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Newton quasiparticle solve (paper Eq. qpapp, Eq. iter, Eq. ps, Eq. NR):
 *   w <- w + (eps_q + Sigma(w) - w) P,  P = 1/(1 - dSigma/dw),  w0 = eps_q,
 *   stop at |dw| <= conv.  Each iteration recomputes Sigma from the factors.
 * ---------------------------------------------------------------------- */

size_t cds_qp_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np,
                              int32_t precision);

/* Blocking.  Outputs (device, [np]): omega (final iterate), pole (pole
 * strength of the last step), iters (Sigma evaluations), status (CDS_QP_*).
 * Returns CDS_ERR_NO_CONVERGENCE if any orbital did not converge (all outputs
 * are still written). */
int cds_qp_solve(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                 const double* Lp, const int32_t* orb, int32_t np, const double* eps,
                 double conv, int32_t max_iter, int32_t precision, double* omega,
                 double* pole, int32_t* iters, int32_t* status, void* workspace,
                 size_t workspace_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Cached numerators ("pole-cached" Newton).  In Eq. SE every element's
 * numerator (2 X_xy - X_yx) X_xy is independent of the energy; only the
 * denominator E + e_s - e_x - e_y moves.  cds_sigma2_diag_cache runs
 * cds_sigma2_diag and also stores the numerators of every work item, as the
 * kernel formed them, in a caller buffer of cds_sigma2_cache_bytes (split
 * precisions: FP32, 128 x 128 items, ~0.38 GB per orbital at C60 shapes;
 * FP64: 32 x 32 items, ~0.45 GB per orbital); cds_qp_solve_cached then runs
 * the Newton iteration of cds_qp_solve with each Sigma(w) evaluated from that
 * buffer, streaming it once per pass instead of recomputing the integrals.
 * Per element the arithmetic is the recomputing kernel's; in FP64 the order
 * of the sums too (equal results at equal energies), in the split precisions
 * only the order of the FP32 sums differs.
 * ---------------------------------------------------------------------- */

size_t cds_sigma2_cache_bytes(int32_t nmo, int32_t nocc, int32_t np, int32_t precision);

/* As cds_sigma2_diag (precision CDS_PREC_FP64, CDS_PREC_BF16X3, CDS_PREC_FP16X3
 * or CDS_PREC_TF32X3), plus cache (device, caller-owned, >=
 * cds_sigma2_cache_bytes of the same precision): the numerators of the
 * orbitals Lp[0..np).  Split precisions: the tensor-core pass evaluates each
 * orbital's first energy while storing the numerators; the other energies
 * are summed from the stored numerators by a second kernel, so they equal
 * cds_sigma2_diag's up to the order of the FP32 sums.  FP64: one pass
 * evaluates every energy and stores the numerators.  Asynchronous. */
int cds_sigma2_diag_cache(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                          const double* Lp, int32_t np, const double* eps, const double* E,
                          int32_t nE, int32_t precision, double* sigma, double* dsigma,
                          void* cache, size_t cache_bytes, void* workspace,
                          size_t workspace_bytes, cudaStream_t stream);

size_t cds_qp_cached_workspace_bytes(int32_t nmo, int32_t nocc, int32_t np);

/* As cds_qp_solve, with Sigma from a cache that cds_sigma2_diag_cache filled
 * for the same orbitals (orb[t] = the orbital of Lp[t]) in `precision` (the
 * cache's form).  Blocking. */
int cds_qp_solve_cached(int32_t nmo, int32_t nocc, int32_t np, const int32_t* orb,
                        const double* eps, double conv, int32_t max_iter, const void* cache,
                        size_t cache_bytes, int32_t precision, double* omega, double* pole,
                        int32_t* iters,
                        int32_t* status, void* workspace, size_t workspace_bytes,
                        cudaStream_t stream);

/* Safeguarded Newton recomputing Sigma from the factors (not in the paper; a
 * variant of Eq. iter): the bracket rule of cds_qp_solve_bracketed_cached
 * below with each Sigma(w) evaluated as in cds_qp_solve (precision
 * CDS_PREC_FP64, CDS_PREC_BF16X3, CDS_PREC_FP16X3 or CDS_PREC_TF32X3; workspace
 * cds_qp_workspace_bytes).  bracket (device, [np][2], caller-owned) receives
 * the final bracket.  Blocking. */
int cds_qp_solve_bracketed(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                           const double* Lp, const int32_t* orb, int32_t np, const double* eps,
                           double conv, int32_t max_iter, int32_t precision, double* omega,
                           double* pole, int32_t* iters, int32_t* status, double* bracket,
                           void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* Safeguarded Newton from cached numerators (not in the paper; a variant of
 * Eq. iter).  Every pole of Sigma_qq lies at e_i + e_j - e_a or e_a + e_b -
 * e_i, and between neighbouring poles f(w) = w - e_q - Sigma(w) rises from
 * -inf to +inf, so the interval around e_q holds exactly one root: the
 * quasiparticle solution connected to the orbital.  From w = e_q the Newton
 * step is kept while it stays inside the current bracket of that root and
 * replaced by the midpoint otherwise.  bracket (device, [np][2], caller-
 * owned) receives the final bracket; the initial one (the nearest poles, a
 * side without a pole taken 10 Ha away) is formed on the host.  Blocking;
 * otherwise as cds_qp_solve_cached. */
int cds_qp_solve_bracketed_cached(int32_t nmo, int32_t nocc, int32_t np, const int32_t* orb,
                                  const double* eps, double conv, int32_t max_iter,
                                  const void* cache, size_t cache_bytes, int32_t precision,
                                  double* omega,
                                  double* pole, int32_t* iters, int32_t* status,
                                  double* bracket, void* workspace, size_t workspace_bytes,
                                  cudaStream_t stream);

/* ------------------------------------------------------------------------
 * MP2 correlation energy (paper Eq. MP2), the ground-state companion of
 * Eq. SE on the same factors:
 *   E = sum_{i,j,a,b} (2 (ai|bj) - (aj|bi)) (ai|bj) / (e_i + e_j - e_a - e_b),
 *   (ai|bj) = sum_K Lov[i][a][K] Lov[j][b][K], recomputed tile by tile.
 * For each i the sum over j, a, b is the second sum of Eq. SE with q := i at
 * E = e_i, and the call runs on the self-energy kernels (FP64, or the
 * tensor-core split precisions).
 * ---------------------------------------------------------------------- */

size_t cds_mp2_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t precision);

/* Asynchronous.  Inputs (device): Lov [nocc][nmo-nocc][M] fp64, eps [nmo].
 * Outputs (device, caller-owned, either may be NULL but not both):
 * e_pair [nocc] = sum_{j,a,b} for each occupied i; e_total [1] = sum of
 * e_pair in a fixed order.  A tensor-core wait that gives up writes NaN.
 * precision: CDS_PREC_FP64, CDS_PREC_BF16X3 or CDS_PREC_FP16X3. */
int cds_mp2_energy(int32_t nmo, int32_t nocc, int32_t M, const double* Lov,
                   const double* eps, int32_t precision, double* e_pair, double* e_total,
                   void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Adjoint (no counterpart in the paper, which does not differentiate; the
 * derivative of Eq. SE, Eq. iter and Eq. transformation).  For a loss l of
 * converged quasiparticle energies w_t with upstream gradients g_t:
 *   dl/dtheta = sum_t g_t P_t (de_qt/dtheta + dSigma_t/dtheta),
 *   P_t = 1/(1 - dSigma_t/dw) at w_t (the implicit-function theorem),
 * with dSigma/dX_xy = (4 X_xy - 2 X_yx) / D_xy for the MO integrals
 * X = (qx|sy), recomputed from the factors for each orbital (never stored
 * for all orbitals at once).
 * ---------------------------------------------------------------------- */

size_t cds_qp_gradient_workspace_bytes(int32_t nmo, int32_t nocc, int32_t M, int32_t np,
                                       int32_t precision);

/* Asynchronous (FP64) or blocking (split precisions: the tensor-core error
 * word is read at the end, CDS_ERR_TIMEOUT if a bounded wait gave up).
 * Inputs as cds_qp_solve plus omega (device [np], converged roots) and g
 * (device [np] upstream gradients).  Outputs (device, fp64 arrays): d_eps
 * [nmo], d_Lov [nocc][nmo-nocc][M], d_Lp [np][nmo][M].  precision:
 *   CDS_PREC_FP64: X and dSigma/dX recomputed per orbital in FP64 on the CUDA
 *     cores, FP64 GEMMs; workspace holds one orbital's dSigma/dX
 *     (o*v*o + v*o*v doubles) plus copies of the factors;
 *   CDS_PREC_BF16X3 / CDS_PREC_TF32X3: X = (qx|sy) recomputed by split-
 *     precision tcgen05 GEMMs (hi.hi + hi.lo + lo.hi, FP32 accumulation), the
 *     factor gradients by the same GEMMs on split dSigma/dX, ~1e-5 relative
 *     (FP32-accumulation accuracy, stored in the fp64 outputs); orbitals go
 *     in chunks of at most 8, and the workspace holds one chunk's split
 *     dSigma/dX in two layouts (~0.8 GB per orbital at o = 180, v = 660).
 * Requires 0 < nocc < nmo. */
int cds_qp_gradient(int32_t nmo, int32_t nocc, int32_t M, const double* Lov, const double* Lp,
                    const int32_t* orb, int32_t np, const double* eps, const double* omega,
                    const double* g, int32_t precision, double* d_eps, double* d_Lov,
                    double* d_Lp, void* workspace, size_t workspace_bytes, cudaStream_t stream);

size_t cds_cd_to_mo_backward_workspace_bytes(int32_t nbf, int32_t nmo, int32_t np);

/* Asynchronous, FP64.  dl/dC [nbf][nmo] (device, overwritten) from dl/dLov
 * and dl/dLp through the transform of cds_cd_to_mo. */
int cds_cd_to_mo_backward(int32_t nbf, int32_t nmo, int32_t nocc, int32_t M, const double* L,
                          const double* C, const int32_t* orb, int32_t np, const double* dLov,
                          const double* dLp, double* dC, void* workspace, size_t workspace_bytes,
                          cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Batched form: many molecules of uneven size, orbital and energy counts in
 * one call per stage (not in the paper, which treats one molecule; each
 * molecule's results are those of the single-molecule calls above).
 * Molecule m is described by cds_mol; its arrays sit back to back in
 * concatenated buffers at the element offsets cds_batch_offsets returns,
 * offs[m * CDS_BATCH_NOFF + k], with k:
 *   0 basis functions (xyz uses 3x, alpha, atom)   1 pairs (D)
 *   2 L [max_rank][npair]                            3 piv [max_rank]
 *   4 C [nbf][nbf]                                   5 eps [nbf]
 *   6 orbitals: orb, omega, pole, iters, status [np] 7 energies: E, sigma, dsigma [np][nE]
 *   8 Lov [nocc][nbf-nocc][M]                        9 Lp [np][nbf][M]
 * (row nmol holds the totals).  Local MO indices in orb; atom indices are the
 * molecule's own.  The workspace (cds_batch_workspace_bytes) holds a
 * scratch part shared by the decomposition and the transform, a part
 * holding the self-energy / Newton state that a graph (below) refers to,
 * 8 worker slots: the library runs the per-molecule transforms on 8 host
 * threads, each with a library stream of its own, ordered after the
 * caller's stream and before its later work; and, sized for
 * CDS_PREC_OZAKI only, the region of the batched tensor-core decomposition
 * (every molecule's slice store [max_rank rounded up to 32][8][npair] BF16,
 * candidate projections and pair data).
 * ---------------------------------------------------------------------- */

typedef struct {
    int32_t nbf;       /* basis functions (= MOs) */
    int32_t nocc;      /* occupied orbitals */
    int32_t np;        /* orbitals whose Sigma / quasiparticle is wanted */
    int32_t nE;        /* energies per orbital on the Sigma grid (>= 1) */
    int32_t max_rank;  /* capacity of the molecule's Cholesky buffer */
} cds_mol;

#define CDS_BATCH_NOFF 10

/* Host only.  offs: host [(nmol + 1) * CDS_BATCH_NOFF]. */
int cds_batch_offsets(int32_t nmol, const cds_mol* mols, int64_t* offs);

/* Host only.  precision CDS_PREC_OZAKI adds the region of the batched
 * tensor-core decomposition after the worker slots; any other value leaves
 * it out.  The calls accept a workspace without the slots (the scratch and
 * state parts only); the transform then runs the molecules one after the
 * other on the caller's stream, and the tensor-core decomposition returns
 * CDS_ERR_WORKSPACE. */
size_t cds_batch_workspace_bytes(int32_t nmol, const cds_mol* mols, int32_t precision);

/* Blocking.  Per molecule as cds_cd_decompose (delta and scheme shared);
 * M_out: host [nmol].  precision: CDS_PREC_FP64, or CDS_PREC_F32X2 (float-pair
 * projections and vectors, FP64 integral column, residuals and pivot
 * decisions; L converted to FP64 at the end): one update and one
 * pivot-select launch per step for the whole batch.  CDS_PREC_OZAKI: the
 * tensor-core form of cds_cd_decompose for every molecule (the same
 * screening, pivots and arithmetic, so the same results bit for bit), its
 * steps batched: three launches per step (slicing, projection GEMM, update)
 * for up to 1024 molecules, larger batches in groups of 1024 (the workspace
 * needs the region of cds_batch_workspace_bytes(..., CDS_PREC_OZAKI)); a
 * molecule's compact vectors are held in its own rows of L during the
 * steps.  Returns the first non-OK molecule status (CDS_ERR_TIMEOUT first
 * when a bounded wait of the projection GEMM gave up). */
int cds_batch_cd_decompose(int32_t nmol, const cds_mol* mols, const double* xyz,
                           const double* alpha, const int32_t* atom, double delta,
                           int32_t scheme, int32_t precision, double* L, int32_t* piv, double* D,
                           int32_t* M_out, void* workspace, size_t workspace_bytes,
                           cudaStream_t stream);

/* Asynchronous (blocking while the worker threads enqueue and, for the
 * exact-slice form, read each molecule's error word).  M: host [nmol] ranks.
 * Per molecule as cds_cd_to_mo. */
int cds_batch_cd_to_mo(int32_t nmol, const cds_mol* mols, const int32_t* M, const double* L,
                       const double* C, const int32_t* orb, int32_t precision, double* Lov,
                       double* Lp, void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* Blocking (descriptor upload), then one persistent tensor-core launch over
 * the items of every molecule.  precision: BF16X3 or FP16X3.  stamps:
 * device [nmol + 1] or NULL (unused here). */
int cds_batch_sigma2(int32_t nmol, const cds_mol* mols, const int32_t* M, const double* Lov,
                     const double* Lp, const double* eps, const double* E, int32_t precision,
                     double* sigma, double* dsigma, unsigned long long* stamps, void* workspace,
                     size_t workspace_bytes, cudaStream_t stream);

/* Blocking.  Newton for every molecule's orbitals, one batched Sigma pass per
 * iteration.  stamps (device [nmol + 1], may be NULL): [0] = %globaltimer at
 * the start, [1 + m] = time the last orbital of molecule m retired. */
int cds_batch_qp_solve(int32_t nmol, const cds_mol* mols, const int32_t* M, const double* Lov,
                       const double* Lp, const int32_t* orb, const double* eps, double conv,
                       int32_t max_iter, int32_t precision, double* omega, double* pole,
                       int32_t* iters, int32_t* status, unsigned long long* stamps,
                       void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* A CUDA graph of the batched Sigma grid (sigma, dsigma) followed by the
 * Newton solve with exactly max_iter passes (converged orbitals skip their
 * work): captured by the library (blocking), replayed by cds_graph_launch
 * with one launch.  Every pointer and the workspace must stay valid, and
 * Lov/Lp/E/eps are re-read at each replay.  Library-owned; free with
 * cds_graph_destroy. */
typedef struct cds_graph cds_graph;
int cds_batch_graph_create(int32_t nmol, const cds_mol* mols, const int32_t* M, const double* Lov,
                           const double* Lp, const int32_t* orb, const double* eps,
                           const double* E, int32_t precision, double conv, int32_t max_iter,
                           double* sigma, double* dsigma, double* omega, double* pole,
                           int32_t* iters, int32_t* status, unsigned long long* stamps,
                           void* workspace, size_t workspace_bytes, cds_graph** out);
int cds_graph_launch(cds_graph* graph, cudaStream_t stream);
int cds_graph_destroy(cds_graph* graph);

/* ------------------------------------------------------------------------
 * Kernel configuration of the tensor-core self-energy, process-wide (no
 * counterpart in the paper; set by the autotuner, which times graph replays
 * of a batch and keeps the fastest choice).
 *   CDS_TUNE_ENERGY_CHUNK: energies per epilogue pass of the batched grid
 *     pass, 8 or 16 (default 16);
 *   CDS_TUNE_ITEM_ORDER: 0 = work items interleaved across the persistent
 *     CTAs (default), 1 = each CTA takes a contiguous range;
 *   CDS_TUNE_NEWTON_CACHE: 1 = the batched grid pass keeps the numerators
 *     and the batched Newton passes evaluate Sigma from them (default), 0 =
 *     each Newton pass recomputes the integrals;
 *   CDS_TUNE_CD_GRAPH: the tensor-core decomposition replays each chunk of
 *     32 steps as one CUDA graph (one launch instead of 96) when max_rank is
 *     at least this value and the stream is not a default stream (0 = never;
 *     default 512; the batched form launches step by step);
 *   CDS_TUNE_PIPE_SPLIT: in cds_cd_decompose_to_mo with a tensor-core
 *     transform, the transform's GEMMs take at most this many CTAs (one per
 *     SM) and the decomposition's projection GEMM the other SMs, so the two
 *     streams run side by side (0 = no split, default);
 *   CDS_TUNE_GRID_EC: energies per pass of the kernels that evaluate the
 *     Sigma grid from the kept numerators (the register tile: 64 numerators x
 *     this many energies per thread), 2, 4 (default) or 8.
 * Graphs keep the configuration they were captured with.
 * ---------------------------------------------------------------------- */
enum { CDS_TUNE_ENERGY_CHUNK = 0, CDS_TUNE_ITEM_ORDER = 1, CDS_TUNE_NEWTON_CACHE = 2,
       CDS_TUNE_CD_GRAPH = 3, CDS_TUNE_PIPE_SPLIT = 4, CDS_TUNE_GRID_EC = 5 };
int cds_tune_set(int32_t knob, int32_t value);   /* CDS_ERR_ARG on an invalid pair */
int cds_tune_get(int32_t knob);                  /* -1 for an unknown knob */

#ifdef __cplusplus
}
#endif

#endif /* CDSIGMA_H */
