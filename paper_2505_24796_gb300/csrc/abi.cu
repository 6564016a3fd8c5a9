// abi.cu -- status strings and version of the C ABI (include/tcgs.h).
#include <atomic>

#include "common.cuh"

namespace tcgs {
static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace tcgs

extern "C" const char* tcgs_status_string(int status) {
    switch (status) {
        case TCGS_OK: return "ok";
        case TCGS_ERR_INVALID: return "invalid argument";
        case TCGS_ERR_CUDA: return "CUDA error";
        case TCGS_ERR_CAPACITY: return "splat capacity exceeded";
        case TCGS_ERR_TIMEOUT: return "device wait timed out";
        case TCGS_ERR_UNSUPPORTED: return "unsupported device (needs sm_103a)";
        case TCGS_ERR_SCRATCH_LIMIT: return "request exceeds the built-in scratch array";
        default: return "unknown status";
    }
}

extern "C" int tcgs_version(void) { return 100; }

extern "C" uint64_t tcgs_kernel_launches(void) { return tcgs::g_launches.load(std::memory_order_relaxed); }
