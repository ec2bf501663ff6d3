// FP32 kernels: shifted populations g = f - w rho0 and theta = T - T_sat,
// FP32 arithmetic; FP16 storage of g as a probe.
#include "lbm_device.cuh"

namespace lbmgb {
namespace {
template <class P>
struct Set {
    using Flow = FlowShape<P, 32, 8, 4>;
    using Heat = HeatShape<P, 32, 16, 256>;
    static cudaError_t flow(const DevParams &p, const StepBuffers &b, cudaStream_t s) { return Flow::launch(p, b, s); }
    static cudaError_t heat(const DevParams &p, const StepBuffers &b, cudaStream_t s) { return Heat::launch(p, b, s); }
    static cudaError_t diag(const DevParams &p, const StepBuffers &b, cudaStream_t s) { return launch_diag<P, 512>(p, b, Flow::blocks(p), s); }
    static int blocks(const DevParams &p) { return Flow::blocks(p); }
};
const KernelSet ks32 = {"fp32", sizeof(float), sizeof(float), sizeof(float), Set<PolicyF32>::flow,
                        Set<PolicyF32>::heat, Set<PolicyF32>::diag, launch_init<PolicyF32>,
                        launch_import<PolicyF32>, launch_export<PolicyF32>, Set<PolicyF32>::blocks,
                        Set<PolicyF32>::Heat::prepare};
const KernelSet ks16 = {"fp16", sizeof(__half), sizeof(float), sizeof(float), Set<PolicyF16>::flow,
                        Set<PolicyF16>::heat, Set<PolicyF16>::diag, launch_init<PolicyF16>,
                        launch_import<PolicyF16>, launch_export<PolicyF16>, Set<PolicyF16>::blocks,
                        Set<PolicyF16>::Heat::prepare};
}  // namespace
const KernelSet *kernels_fp32() { return &ks32; }
const KernelSet *kernels_fp16() { return &ks16; }
}  // namespace lbmgb
