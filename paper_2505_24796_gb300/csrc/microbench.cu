// microbench.cu -- throughput of the special-function unit's base-2 exponential (PTX
// ex2.approx.ftz.f32), the one transcendental the tensor-core renderer evaluates per walked
// (pixel, Gaussian) slot; measured rather than taken from a datasheet, as the denominator of the
// renderer's SFU figure.
#include "common.cuh"

namespace tcgs {
namespace {

constexpr int kEx2Chains = 8;   // independent chains per thread, so the unit, not latency, bounds it

// Each thread runs kEx2Chains chains x <- -2^x for `iters` steps (x stays in [-1, -0.5]) and writes
// the chains' sum, so no step can be dropped.
__global__ void __launch_bounds__(256) k_ex2_rate(float* __restrict__ out, int iters) {
    float x[kEx2Chains];
#pragma unroll
    for (int c = 0; c < kEx2Chains; ++c) x[c] = -0.5f - 0.0625f * (float)c - 1e-6f * (float)(threadIdx.x & 31);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kEx2Chains; ++c) x[c] = -ex2_approx(x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kEx2Chains; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace tcgs

extern "C" tcgs_status tcgs_microbench_ex2(float* out, int32_t blocks, int32_t iters, tcgs_stream stream) {
    using namespace tcgs;
    if (!out || blocks <= 0 || iters <= 0) return TCGS_ERR_INVALID;
    k_ex2_rate<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, iters);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}
