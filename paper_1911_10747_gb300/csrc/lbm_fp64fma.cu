// FP64 kernels compiled with fused multiply-add contraction (-fmad=true): the
// same source as lbm_fp64.cu, but the compiler may fuse a product into the
// following sum.  Results are no longer bit-identical to the oracle (which
// rounds every product and sum on its own); they are checked against it to
// a relative 1e-12 per site.  A policy type of this unit's own keeps its
// kernel instantiations apart from the -fmad=false ones.
#include "lbm_device.cuh"

namespace lbmgb {
namespace {
struct PolicyF64Fma : PolicyF64 {};
using P = PolicyF64Fma;
using Flow = FlowShape<P, 32, 8, 2>;
using Heat = HeatShape<P, 32, 16, 256>;
cudaError_t diag(const DevParams &p, const StepBuffers &b, int nblk, cudaStream_t s) {
    return launch_diag<P, 512>(p, b, nblk, s);
}
cudaError_t no_prepare() { return cudaSuccess; }
const FlowVariant flows[] = {{"flow64fma_32x8x2", Flow::launch, Flow::blocks, no_prepare}};
const HeatVariant heats[] = {{"heat64fma_32x16_t256", Heat::launch, Heat::prepare}};
const KernelSet ks = {"fp64fma", sizeof(double), sizeof(double), sizeof(double), 1, flows, 1, heats, diag,
                      launch_init<P>, launch_import<P>, launch_export<P>, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                      launch_import32<P>};
}  // namespace
const KernelSet *kernels_fp64_fma() { return &ks; }
}  // namespace lbmgb
