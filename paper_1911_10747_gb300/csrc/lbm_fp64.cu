// FP64 kernels: the oracle-parity path.  Compiled with -fmad=false so that
// every product and sum is rounded on its own, as in a plain evaluation of
// the formulas.
#include "lbm_device.cuh"

namespace lbmgb {
namespace {
using P = PolicyF64;
using Flow = FlowShape<P, 32, 8, 2>;
using Heat = HeatShape<P, 32, 16, 256>;
cudaError_t flow(const DevParams &p, const StepBuffers &b, cudaStream_t s) { return Flow::launch(p, b, s); }
cudaError_t heat(const DevParams &p, const StepBuffers &b, cudaStream_t s) { return Heat::launch(p, b, s); }
cudaError_t diag(const DevParams &p, const StepBuffers &b, cudaStream_t s) { return launch_diag<P, 512>(p, b, Flow::blocks(p), s); }
int blocks(const DevParams &p) { return Flow::blocks(p); }
const KernelSet ks = {"fp64", sizeof(double), sizeof(double), sizeof(double), flow, heat, diag,
                      launch_init<P>, launch_import<P>, launch_export<P>, blocks, Heat::prepare};
}  // namespace
const KernelSet *kernels_fp64() { return &ks; }
}  // namespace lbmgb
