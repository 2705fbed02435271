// Allocation-free variant of the Cholesky decomposition entry point.
//
// Some callers cannot allocate device memory at the point where they want a
// decomposition: a host program whose GPU memory is owned by another runtime
// or memory pool it cannot reach from this call site, a plugin that must not
// grow the device footprint, or a code path where a cudaMalloc would
// synchronise the device at an inconvenient moment.  cds_cd_decompose needs
// a caller-provided workspace; this entry point instead uses a fixed scratch
// array that lives in the library's own device image, so the caller passes
// only the inputs and the outputs.
//
// The scratch is a file-scope __device__ array of CDS_CD_STATIC_SCRATCH_BYTES
// (4 MiB); every GPU that loads the library holds it until the process exits.
// Host code may not use the array's name as a device address (on the host it
// is only a stand-in symbol), so the device address is looked up with
// cudaGetSymbolAddress, with the device current, at every call made outside a
// stream capture; a call inside a capture reuses the address of the last
// uncaptured call on that device, so the first call on a device should come
// before any stream capture.  All calls share the one array and it keeps the
// previous call's contents: the decomposition re-initialises everything it
// reads (pair data, candidate mask, control block) at the start of each call,
// and two calls whose GPU work overlaps in time race on the array.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kStaticBytes = CDS_CD_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_cd_scratch[kStaticBytes];

std::mutex g_lock;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Outside a
// stream capture it is looked up at every call (the lookup allocates
// nothing), so a context that was destroyed and re-created since the last
// call, which reloads the module at a new address, never leaves a stale
// address behind.  During a capture the address of the last uncaptured call
// on this device is used; with none yet the call is refused.
int scratch_address(cudaStream_t stream, void** out) {
    int dev = 0;
    CDS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CDS_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CDS_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
    std::lock_guard<std::mutex> guard(g_lock);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        CDS_CUDA_TRY(cudaGetSymbolAddress(&p, g_cd_scratch));
        if (!p) return CDS_ERR_CUDA;
        g_addr[dev] = p;
    }
    if (!g_addr[dev]) return CDS_ERR_UNSUPPORTED;
    *out = g_addr[dev];
    return CDS_OK;
}

}  // namespace

extern "C" int cds_cd_decompose_static(int32_t nbf, const double* xyz, const double* alpha,
                                       const int32_t* atom, double delta, int32_t scheme,
                                       int32_t max_rank, double* L, int32_t* piv, double* D,
                                       int32_t* M_out, double* delta_eff_out,
                                       cudaStream_t stream) {
    if (nbf <= 0) return CDS_ERR_ARG;
    const size_t need = cds::cd_workspace_bytes_for(nbf, false);
    if (need == 0) return CDS_ERR_ARG;
    if (need > kStaticBytes) return CDS_ERR_CAPACITY;
    void* ws = nullptr;
    int st = scratch_address(stream, &ws);
    if (st) return st;
    return cds_cd_decompose(nbf, xyz, alpha, atom, delta, scheme, max_rank, CDS_PREC_FP64, L, piv,
                            D, M_out, delta_eff_out, ws, kStaticBytes, stream);
}

extern "C" int cds_cd_static_max_nbf(void) {
    int32_t lo = 1, hi = 1 << 16;
    while (lo < hi) {   // largest nbf whose workspace fits the static scratch
        int32_t mid = lo + (hi - lo + 1) / 2;
        if (cds::cd_workspace_bytes_for(mid, false) <= kStaticBytes) lo = mid; else hi = mid - 1;
    }
    return lo;
}
