// FP32 kernels: shifted populations g = f - w rho0 and theta = T - T_sat,
// FP32 arithmetic; FP16 storage of g as a probe.  Several launch shapes of
// the flow and heat kernels are compiled; lbm_autotune picks among them.
#include "lbm_fast.cuh"
#include "lbm_tma.cuh"
#include "lbm_heatwave.cuh"
#include "lbm_flowwave.cuh"
#include "lbm_multi.cuh"

namespace lbmgb {
namespace {
template <class P>
cudaError_t diag(const DevParams &p, const StepBuffers &b, int nblk, cudaStream_t s) {
    return launch_diag_flat<P, 1024>(p, b, nblk, s);
}
#define FLOWV(P, BX, BY, RY, MB)                                                                  \
    {"flow_" #BX "x" #BY "x" #RY "_b" #MB, FlowFastShape<P, BX, BY, RY, MB>::launch,                \
     FlowFastShape<P, BX, BY, RY, MB>::blocks, FlowFastShape<P, BX, BY, RY, MB>::prepare}
#define FLOWP(P, BX, BY, RY, MB)                                                                  \
    {"flowpers_" #BX "x" #BY "x" #RY "_b" #MB, FlowPersShape<P, BX, BY, RY, MB>::launch,            \
     FlowPersShape<P, BX, BY, RY, MB>::blocks, FlowPersShape<P, BX, BY, RY, MB>::prepare}
#define FLOWT(P, BY, RY, MB)                                                                      \
    {"flowtma_64x" #BY "x" #RY "_b" #MB, FlowTmaShape<P, BY, RY, MB>::launch, FlowTmaShape<P, BY, RY, MB>::blocks, \
     FlowTmaShape<P, BY, RY, MB>::prepare}
#define FLOWW(WPB, MB, U2)                                                                        \
    {"flowwave_w" #WPB "_b" #MB "_u" #U2, FlowWaveShape<WPB, MB, U2>::launch,                          \
     FlowWaveShape<WPB, MB, U2>::blocks, FlowWaveShape<WPB, MB, U2>::prepare}
#define FLOWWT(WPB, MB, SM, ST, TU)                                                               \
    {"flowwave_w" #WPB "_b" #MB "_s" #SM "t" #ST "x" #TU, FlowWaveShape<WPB, MB, 0, SM, ST, TU>::launch, \
     FlowWaveShape<WPB, MB, 0, SM, ST, TU>::blocks, FlowWaveShape<WPB, MB, 0, SM, ST, TU>::prepare}
#define HEATP16D(P, BY, R, MB)                                                                    \
    {"heatpair16_64x" #BY "x" #R "_down", HeatPairShape<P, BY, R, MB, true, true>::launch,              \
     HeatPairShape<P, BY, R, MB, true, true>::prepare}
#define HEATS(P, BW, BY, R, MB) \
    {"heatrows_" #BW "x" #BY "x" #R, HeatRowsShape<P, BW, BY, R, MB>::launch, HeatRowsShape<P, BW, BY, R, MB>::prepare}
#define HEATSD(P, BW, BY, R, MB)                                                                 \
    {"heatrows_" #BW "x" #BY "x" #R "_dfsrc", HeatRowsShape<P, BW, BY, R, MB, true>::launch,          \
     HeatRowsShape<P, BW, BY, R, MB, true>::prepare}
#define HEATP(P, BY, R, MB) \
    {"heatpair_64x" #BY "x" #R, HeatPairShape<P, BY, R, MB>::launch, HeatPairShape<P, BY, R, MB>::prepare}
#define HEATP16(P, BY, R, MB)                                                                     \
    {"heatpair16_64x" #BY "x" #R, HeatPairShape<P, BY, R, MB, true>::launch,                           \
     HeatPairShape<P, BY, R, MB, true>::prepare}
#define HEATW(P, CL, WPB, MB, RS) \
    {"heatwave_c" #CL "_w" #WPB "_b" #MB "_r" #RS, HeatWaveShape<P, CL, WPB, MB, RS>::launch, \
     HeatWaveShape<P, CL, WPB, MB, RS>::prepare}
#define FLOWM(P) {"flowmulti_32x8x2", MultiKernels<P>::flow, MultiKernels<P>::flow_blocks, MultiKernels<P>::prepare}
#define FLOWWM(P) {"flowwavemulti_w4_b4", MultiKernels<P>::wave, MultiKernels<P>::wave_blocks, MultiKernels<P>::prepare}
#define HEATM(P) {"heatmulti_64x12x4", MultiKernels<P>::heat, MultiKernels<P>::prepare}
#define MULTI(P) sizeof(MultiRun), fill_multi<P>, multi_flow_items<P>, multi_heat_tiles, multi_mode<P>, MultiKernels<P>::launch, \
    launch_import32<P>
#define NOMULTI(P) 0, nullptr, nullptr, nullptr, nullptr, nullptr, launch_import32<P>
#define HEATV(P, TX, TY, BX, BY) \
    {"heat_" #TX "x" #TY "_t" #BX "x" #BY, HeatFastShape<P, TX, TY, BX, BY>::launch, HeatFastShape<P, TX, TY, BX, BY>::prepare}

const FlowVariant flows32[] = {
    FLOWT(PolicyF32, 4, 2, 3), FLOWP(PolicyF32, 64, 4, 2, 2), FLOWP(PolicyF32, 32, 8, 2, 2),
    FLOWP(PolicyF32, 32, 8, 1, 3), FLOWV(PolicyF32, 32, 8, 2, 3), FLOWV(PolicyF32, 64, 4, 2, 3),
    FLOWW(4, 3, 8), FLOWW(4, 4, 8),
    FLOWWT(4, 3, 16, 4, 4),
    FLOWWM(PolicyF32), FLOWM(PolicyF32),
};
const HeatVariant heats32[] = {
    HEATS(PolicyF32, 64, 6, 5, 1), HEATS(PolicyF32, 64, 8, 4, 1), HEATS(PolicyF32, 64, 10, 3, 1),
    HEATS(PolicyF32, 64, 6, 6, 1),
    HEATS(PolicyF32, 32, 8, 4, 2),
    HEATP(PolicyF32, 12, 4, 1), HEATP(PolicyF32, 8, 4, 1), HEATP16(PolicyF32, 12, 4, 1), HEATP16D(PolicyF32, 12, 4, 1),
    HEATW(PolicyF32, 2, 2, 4, 8), HEATM(PolicyF32),
    HEATV(PolicyF32, 32, 16, 32, 8), HEATV(PolicyF32, 64, 32, 32, 16),
};
// the Eq. 24 source in double-float arithmetic (precision LBM_FP32_DFSRC)
const HeatVariant heats32df[] = {HEATSD(PolicyF32, 64, 8, 4, 1), HEATSD(PolicyF32, 64, 6, 5, 1)};
const FlowVariant flows16[] = {FLOWP(PolicyF16, 32, 8, 2, 2), FLOWV(PolicyF16, 32, 8, 2, 3), FLOWM(PolicyF16)};
const HeatVariant heats16[] = {HEATS(PolicyF16, 64, 10, 3, 1), HEATS(PolicyF16, 64, 8, 4, 1), HEATP(PolicyF16, 12, 4, 1),
                               HEATP16(PolicyF16, 12, 4, 1), HEATP16D(PolicyF16, 12, 4, 1),
                               HEATV(PolicyF16, 32, 32, 32, 16), HEATM(PolicyF16)};

const KernelSet ks32 = {"fp32", sizeof(float), sizeof(float), sizeof(float),
                        (int)(sizeof(flows32) / sizeof(flows32[0])), flows32,
                        (int)(sizeof(heats32) / sizeof(heats32[0])), heats32, diag<PolicyF32>,
                        launch_init<PolicyF32>, launch_import<PolicyF32>, launch_export<PolicyF32>, MULTI(PolicyF32)};
// (the two multi-run flow variants, listed last, need a run descriptor this set does not keep)
const KernelSet ks32df = {"fp32dfsrc", sizeof(float), sizeof(float), sizeof(float),
                          (int)(sizeof(flows32) / sizeof(flows32[0])) - 2, flows32,
                          (int)(sizeof(heats32df) / sizeof(heats32df[0])), heats32df, diag<PolicyF32>,
                          launch_init<PolicyF32>, launch_import<PolicyF32>, launch_export<PolicyF32>, NOMULTI(PolicyF32)};
const KernelSet ks16 = {"fp16", sizeof(__half), sizeof(float), sizeof(float),
                        (int)(sizeof(flows16) / sizeof(flows16[0])), flows16,
                        (int)(sizeof(heats16) / sizeof(heats16[0])), heats16, diag<PolicyF16>,
                        launch_init<PolicyF16>, launch_import<PolicyF16>, launch_export<PolicyF16>, MULTI(PolicyF16)};
}  // namespace
const KernelSet *kernels_fp32() { return &ks32; }
const KernelSet *kernels_fp16() { return &ks16; }
const KernelSet *kernels_fp32_dfsrc() { return &ks32df; }
}  // namespace lbmgb
