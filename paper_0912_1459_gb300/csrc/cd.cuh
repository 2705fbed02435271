// Shared declarations of the Cholesky decomposition kernels (cd.cu) and its
// exact-slice tensor-core projection GEMM (cd_tc.cu).
#pragma once

#include "common.cuh"

namespace cds {

constexpr int kCdThreads = 128;
constexpr int kUpdWarps = 8;                  // k_cd_update: warps splitting the K sum
constexpr int kUpdThreads = 32 * kUpdWarps;
constexpr int kUpdPairs = 64;                 // k_cd_project: pairs per projection tile
constexpr int kStepPer = 2;                   // k_cd_update: pairs per thread
constexpr int kStepChunk = kStepPer * kUpdThreads;   // k_cd_update: contiguous pairs per block
constexpr int kCdChunk = 2048;   // pivot row L^K_P staged in shared memory in chunks
constexpr double kTieRel = 1e-12;
constexpr double kNotPdRel = 1e-10;
constexpr int kHostCheckEvery = 32;
#ifndef CDS_KSPEC
#define CDS_KSPEC 4
#endif
#ifndef CDS_KSPEC_ROWS
#define CDS_KSPEC_ROWS 4
#endif
constexpr int kSpec = CDS_KSPEC;          // candidate pivots per speculative projection pass
constexpr int kSpecRows = CDS_KSPEC_ROWS; // rows of L in flight per thread and iteration
constexpr int kSpecChunk = 4096 / kSpec;   // pivot columns staged per shared-memory chunk (32 KB)
// Exact-slice tensor-core form (CDS_PREC_OZAKI): candidates per streaming
// pass, the longest batch of steps one pass serves, the column group of the
// slice store (one 64-byte TMA row of BF16), the slices per element and the
// bits per slice (56-bit fixed point below a per-pair power-of-two scale).
constexpr int kSpecTC = 32;
constexpr int kBatchTC = 64;
constexpr int kGroupTC = 32;
constexpr int kSlicesTC = 8;
constexpr int kBitsTC = 7;
constexpr int kMaxBlocksTC = 2048;   // update blocks the candidate search holds in shared memory

// Programmatic dependent launch of the per-step kernels of the tensor-core
// form: each kernel lets the next one be scheduled as soon as all its own
// blocks run (pdl_trigger) and waits for its predecessor's completion and
// memory before it reads anything (pdl_wait; a no-op in a normal launch), so
// the launch of step k+1's kernels overlaps the serial tail of step k's.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... K, typename... A>
inline cudaError_t launch_pdl(void (*kern)(K...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t stream, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

struct CdCtrl {
    double scale;      // max initial diagonal (all pairs)
    double delta_eff;  // max(delta, npair * 2^-52 * scale)
    double G;          // max candidate residual after the last update
    double Dmin;       // min residual after the last update
    double DP;         // residual of the current pivot
    double rDP;        // 1 / sqrt(DP)
    float2 rDPf;       // the same as a float pair
    int64_t P;         // current pivot
    int32_t done;      // decomposition stopped
    int32_t status;    // cds_status
    int32_t M;         // vectors produced
    int32_t _pad;
    unsigned int counter;  // last-block-done counter
    unsigned int _pad2;
    // speculative projections (float-pair mode): the pivots of the current
    // batch's candidate set, the batch's first step, the slot of the current
    // pivot in the set, and whether this step streams L (a new batch)
    long long S[kSpec];
    int32_t k0, slot, pass, passes;     // passes: batches started (streaming passes)
    long long streamed;                  // sum over passes of the vectors streamed (k0)
    long long extra;                     // sum over continued steps of the vectors added (k - k0)
    // exact-slice tensor-core form: its candidate set, and the step of the
    // previous pass (the slice store holds every row before it)
    long long STc[kSpecTC];
    int32_t kdone;
    int32_t nlive;     // tensor-core form: pairs kept after screening
    int32_t kstep;     // tensor-core form: the step the kernels run next
    int32_t _pad4;
};

// Tensor-core form: pairs whose initial diagonal is below kScreenRel of the
// largest are left out of the decomposition (Schwarz: every L^K_I of such a
// pair is below sqrt(D0_I), i.e. below 1e-20 sqrt(max D0); their vectors are
// returned as 0 and their residual as D0_I, and no other pair's arithmetic
// involves them).
constexpr double kScreenRel = 1e-40;
constexpr int kScanPer = 4;                        // pairs per thread in the compaction
constexpr int kScanThreads = 256;
constexpr int kScanChunk = kScanPer * kScanThreads;   // pairs per compaction block

// The exact-slice projection GEMM of one step (cd_tc.cu).  Enqueued at every
// step of the tensor-core form; it returns at once unless the step starts a
// streaming pass (ctrl->pass), and then forms, for the pass's candidate set,
//   G[c][I] = sum_{K < k0} L^K_I L^K_{S_c}     (float pairs, [kSpecTC][n]),
// from the slice store (A: [kcap / kGroupTC][kSlicesTC][n][kGroupTC], pair
// rows blocked by 32-column groups) and the candidate rows (B: the same with
// kSpecTC rows), both scaled by
// the per-row powers of two sigA / sigB.
struct CdTcGemm;
int cd_tc_gemm_setup(CdTcGemm** out, int64_t n, int32_t kcap, const void* a_planes,
                     const void* b_planes, const float* sigA, const float* sigB, float2* G,
                     const CdCtrl* ctrl, int32_t* err);
int cd_tc_gemm_launch(const CdTcGemm* g, cudaStream_t stream);
void cd_tc_gemm_free(CdTcGemm* g);

// Batched form: one launch per step for up to kMaxMolsTC molecules, each with
// its own two tensor maps (cd_tc_maps_bytes() bytes per molecule, 64-byte
// aligned, in device memory) and this table entry; the tiles of the
// molecules that start a pass at the step are spread over one CTA per SM.
constexpr int kMaxMolsTC = 1024;
struct CdTcMolGemm {
    int64_t n;            // pair rows (the live pairs)
    const float* sa;      // [n] pair scales
    const float* sb;      // [kSpecTC] candidate scales
    float2* G;            // [kSpecTC][n]
    const CdCtrl* ctrl;
};
// Inclusive prefix, in place, of pre[1 .. nmol] (shared memory), and pre[0] = 0;
// run by the 32 threads of one warp.
template <typename T>
__device__ __forceinline__ void warp_prefix_smem(T* pre, int nmol) {
    const int lane = threadIdx.x & 31;
    T run = 0;
    for (int c0 = 0; c0 < nmol; c0 += 32) {
        const int c = c0 + lane;
        T x = c < nmol ? pre[c + 1] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (c < nmol) pre[c + 1] = run + x;
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) pre[0] = 0;
}
size_t cd_tc_maps_bytes();
int cd_tc_maps_encode(void* out, int64_t n, int32_t kcap, const void* a_planes,
                      const void* b_planes);
int cd_tc_batch_gemm_launch(const CdTcMolGemm* mols, const void* maps, int32_t nmol,
                            int32_t* err, cudaStream_t stream);

}  // namespace cds
