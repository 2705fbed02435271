// Library identity, status strings and the launch counter.
#include <atomic>

#include "common.cuh"

namespace cds {
static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace cds

extern "C" unsigned long long cds_launch_count(void) { return cds::g_launches.load(); }

extern "C" int cds_version(void) { return 100; }

extern "C" const char* cds_errstr(int status) {
    switch (status) {
        case CDS_OK: return "success";
        case CDS_ERR_ARG: return "invalid argument";
        case CDS_ERR_CUDA: return "CUDA runtime error";
        case CDS_ERR_NOT_PD: return "residual diagonal negative beyond roundoff";
        case CDS_ERR_RANK_CAP: return "Cholesky rank cap reached before delta";
        case CDS_ERR_NO_CONVERGENCE: return "Newton iteration did not converge";
        case CDS_ERR_WORKSPACE: return "workspace too small";
        case CDS_ERR_UNSUPPORTED: return "unsupported device or precision";
        case CDS_ERR_TIMEOUT: return "bounded device wait gave up";
        case CDS_ERR_CAPACITY: return "problem exceeds the allocation-free scratch array";
        default: return "unknown status";
    }
}
