// abi.cu -- status strings and version of the C ABI (include/tcgs.h).
#include "common.cuh"

extern "C" const char* tcgs_status_string(int status) {
    switch (status) {
        case TCGS_OK: return "ok";
        case TCGS_ERR_INVALID: return "invalid argument";
        case TCGS_ERR_CUDA: return "CUDA error";
        case TCGS_ERR_CAPACITY: return "splat capacity exceeded";
        case TCGS_ERR_TIMEOUT: return "device wait timed out";
        case TCGS_ERR_UNSUPPORTED: return "unsupported device (needs sm_103a)";
        default: return "unknown status";
    }
}

extern "C" int tcgs_version(void) { return 100; }
