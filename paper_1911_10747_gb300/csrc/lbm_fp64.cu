// FP64 kernels: the oracle-parity path.  Compiled with -fmad=false so that
// every product and sum is rounded on its own, as in a plain evaluation of
// the formulas.
#include "lbm_device.cuh"

namespace lbmgb {
namespace {
using P = PolicyF64;
using Flow = FlowShape<P, 32, 8, 2>;
using Heat = HeatShape<P, 32, 16, 256>;
cudaError_t diag(const DevParams &p, const StepBuffers &b, int nblk, cudaStream_t s) {
    return launch_diag<P, 512>(p, b, nblk, s);
}
cudaError_t no_prepare() { return cudaSuccess; }
const FlowVariant flows[] = {{"flow64_32x8x2", Flow::launch, Flow::blocks, no_prepare}};
const HeatVariant heats[] = {{"heat64_32x16_t256", Heat::launch, Heat::prepare}};
const KernelSet ks = {"fp64", sizeof(double), sizeof(double), sizeof(double), 1, flows, 1, heats, diag,
                      launch_init<P>, launch_import<P>, launch_export<P>, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                      launch_import32<P>};
}  // namespace
const KernelSet *kernels_fp64() { return &ks; }
}  // namespace lbmgb
