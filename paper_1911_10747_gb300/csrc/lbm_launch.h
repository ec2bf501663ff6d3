// Internal interface between the host runtime (lbm_runtime.cu) and the
// per-precision kernel translation units (lbm_fp64.cu, lbm_fp32.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace lbmgb {

// FLAG_MODEL_A is set by the library (heater.ny_solid = 0), never by callers
enum { FLAG_PERIODIC_Y = 1, FLAG_ISOTHERMAL = 2, FLAG_FROZEN_FLOW = 4, FLAG_MODEL_A = 8 };
enum { TOP_WALL = 0, TOP_OUTFLOW = 1 };
enum { BCM_SPOTS = 0, BCM_NOISE = 1, BCM_SINE = 2 };
// ERRW_TIMEOUT: a staged-copy wait ran out (100 ms).  The block stops, then
// waits once more (bounded) for each stage with copies outstanding before it
// exits.  If the copy engine itself has stalled, copies can still be in flight
// when those waits also run out, and could land in shared memory that a later
// block owns: the step's results are invalid either way, and the host reports
// LBM_E_TIMEOUT.
// ERRW_DESC: a multi-run kernel block found a descriptor it cannot trust
// (not filled, or its tile outside its run) and skipped its tile.
enum { ERRW_PSI = 1, ERRW_NONFINITE_RHO = 2, ERRW_NONFINITE_T = 4, ERRW_TIMEOUT = 8, ERRW_DESC = 16 };
enum { TAG_INIT_NOISE = 1, TAG_BOTTOM_NOISE = 2 };
enum { SERIES_WIDTH = 4 };

// Everything a kernel needs about the run, precomputed on the host in FP64.
struct DevParams {
    int nx, nf, ns, nt;           // columns, fluid rows, heater rows, nt = ns + nf
    int flags, top_mode, bc_mode;
    int liquid_rows;
    double a, b, R, G, kappa, Tc; // Peng-Robinson constants
    double T_sat, T_b;
    double rho_L, rho_V, rho_mean, rho_shift;
    double drho_LV, dtau_LV;      // rho_L - rho_V, tau_L - tau_V (Eq. 5)
    double g, c_v, cv_chi, lambda_s, rho_c_s;
    double tau_L, tau_V;
    double s[9];                  // MRT rates; s7, s8 unused (per-site)
    double hs[9];                 // 1 - s_k / 2
    double tau_e_m, tau_s_m;      // 1/s1 - 1/2, 1/s2 - 1/2
    double varpi12;               // 12 varpi
    double sign_eps;
    double c_w_top;
    double bc_noise, sine_amp, sine_wl;
    long long sine_t0, sine_t1;
    double init_noise;
    double vap_threshold;         // (rho_L + rho_V) / 2
    unsigned long long seed;
    unsigned tx_pad;              // test hook: extra bytes the staged-copy waits expect (0)
};

// Device buffers of one run touched by a step (types erased; the kernel
// translation unit casts them to its storage types).
struct StepBuffers {
    const void *f_in;
    void *f_out;
    const void *T_in;
    void *T_out;
    void *rho, *ux, *uy;     // moments of this step (real type of the path)
    const double *cw;        // [nx] heater-surface wettability coefficients
    double *part;            // [2 * lbm blocks] per-block mass and vapour count
    unsigned *err;           // latched fault bits
    long long *step;         // device step counter
    double *series;          // [cap][SERIES_WIDTH]
    int series_cap;
    double *q_top;           // [nx] local interface flux of the last step
    double *last;            // [SERIES_WIDTH] diagnostics of the last step
    double *scratch;         // reduction scratch for init (>= 1024 doubles)
    const void *mdesc;       // the run's own multi-run descriptor for this parity (kernel sets that have one)
    unsigned *wq;            // 2 words, zero between launches: work counter of the wavefront flow kernel
};

// One launch shape of the flow or heat kernel.  Every variant of a kernel
// does the same per-site arithmetic; only tiling and occupancy differ.
struct FlowVariant {
    const char *name;
    cudaError_t (*launch)(const DevParams &, const StepBuffers &, cudaStream_t);
    int (*blocks)(const DevParams &);   // blocks of one launch (= per-block partials)
    cudaError_t (*prepare)();           // per-device set-up (persistent grid size)
};
struct HeatVariant {
    const char *name;
    cudaError_t (*launch)(const DevParams &, const StepBuffers &, cudaStream_t);
    cudaError_t (*prepare)();           // per-device kernel attributes
};

struct KernelSet {
    const char *name;
    size_t f_elem, T_elem, m_elem;      // storage bytes per population, T, moment
    int n_flow;
    const FlowVariant *flow;
    int n_heat;
    const HeatVariant *heat;
    cudaError_t (*diag)(const DevParams &, const StepBuffers &, int nblk, cudaStream_t);
    // Initial state (Sec. 3.1).  phase 0: initial densities into rho and
    // their sum into scratch[0]; phase 1 (after the host has fixed rho_mean
    // and rho_shift): populations into f_out, T_sat into T_out.
    cudaError_t (*init)(const DevParams &, const StepBuffers &, int phase, cudaStream_t);
    // float64 post-stream f / T (device) -> storage (f_out / T_out).
    cudaError_t (*import_state)(const DevParams &, const double *f, const double *T,
                                const StepBuffers &, cudaStream_t);
    // storage -> float64 device arrays (any pointer may be NULL).
    cudaError_t (*export_fields)(const DevParams &, const StepBuffers &, double *rho, double *ux,
                                 double *uy, double *T, double *f, cudaStream_t);
    // Multi-run launches (one launch per kernel kind steps many runs over a
    // work list of (run, item)); multi_desc_bytes = 0 if the set has none.
    size_t multi_desc_bytes;
    // a run's descriptor (host memory `out`) for its buffers of parity 0 / 1,
    // the parity of its state at phase 0 of the launches, its launch mode (bit
    // 0: wavefront flow units instead of 32 x 16-site tiles; bit 1: heat tiles
    // staged as whole rows; multi_mode gives the bits a run can take) and its
    // first flow items and heat tiles in the launches
    void (*multi_fill)(const DevParams &, const StepBuffers &b0, const StepBuffers &b1, int parity, int mode,
                       int flow0, int heat_tile0, void *out);
    int (*multi_flow_items)(const DevParams &, int mode);
    int (*multi_heat_tiles)(const DevParams &);
    int (*multi_mode)(const DevParams &);
    // kind 0 flow (tiles), 1 heat, 2 diagnostics, 3 flow (wavefront units),
    // 4 heat (whole-row staging; every run of the launch must take it) over
    // nruns descriptors (device), items of that kind in total; errw: the
    // launches' error word; wq: two words, zero between launches, for the
    // wavefront launches' work counter
    cudaError_t (*multi_launch)(int kind, const void *desc, int nruns, int items, int phase, unsigned *errw,
                                unsigned *wq, cudaStream_t);
    // float32 post-stream f / T (device) -> storage, as import_state
    cudaError_t (*import_state32)(const DevParams &, const float *f, const float *T, const StepBuffers &,
                                  cudaStream_t);
};

// Message returned by lbm_last_error(NULL) (thread-local).
void set_global_error(const std::string &msg);

const KernelSet *kernels_fp64();
const KernelSet *kernels_fp32();
const KernelSet *kernels_fp16();
const KernelSet *kernels_fp32_dfsrc();
const KernelSet *kernels_fp64_fma();

}  // namespace lbmgb
