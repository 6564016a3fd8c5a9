// abi.cu -- status strings and version of the C ABI (include/tcgs.h).
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace tcgs {
static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::mutex g_info_mutex;
static DeviceInfo g_info[kMaxDevices];
static bool g_info_set[kMaxDevices] = {};

bool current_device_info(DeviceInfo* out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
    std::lock_guard<std::mutex> lock(g_info_mutex);
    if (!g_info_set[dev]) {
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return false;
        g_info[dev] = DeviceInfo{dev, sms, major == 10 && minor == 3};
        g_info_set[dev] = true;
    }
    *out = g_info[dev];
    return true;
}
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
