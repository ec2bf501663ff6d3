// Host runtime behind the C ABI of include/lbm.h: configuration checks,
// device allocation, the per-step launch sequence (flow kernel, heat kernel,
// diagnostics kernel), CUDA-graph replay, state import/export and read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_launch.h"

using namespace lbmgb;

namespace {
thread_local std::string g_create_error;

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};
}  // namespace

struct lbm_run {
    DevParams p{};
    const KernelSet *ks = nullptr;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool use_graphs = true;
    int parity = 0;                 // 0: state in buffers [0], 1: in [1]
    int64_t steps = 0;
    int64_t series_from = 0;        // first step of the current trajectory (lbm_set_state restarts it)
    bool diag_stale = false;        // lbm_set_state since the last step: no diagnostics of this state yet
    void *f[2] = {nullptr, nullptr};
    void *T[2] = {nullptr, nullptr};
    // moments and per-block partials are double-buffered by parity, so the
    // diagnostics kernel of step n (side stream) can overlap the flow kernel
    // of step n + 1
    void *rho[2] = {nullptr, nullptr}, *ux[2] = {nullptr, nullptr}, *uy[2] = {nullptr, nullptr};
    double *part[2] = {nullptr, nullptr};
    double *cw = nullptr, *series = nullptr, *q_top = nullptr, *last = nullptr;
    cudaStream_t dstream = nullptr;  // diagnostics stream
    cudaEvent_t ev_heat = nullptr, ev_diag = nullptr;    // plain launches
    cudaEvent_t cev_heat = nullptr, cev_diag = nullptr;  // inside stream captures
    double *scratch = nullptr;
    void *mdesc = nullptr;          // two multi-run descriptors (state parity 0, 1), kernel sets that have them
    double *stage = nullptr;        // float64 staging for read-back / import
    size_t stage_elems = 0;
    unsigned *err = nullptr;
    long long *dstep = nullptr;
    int series_cap = 4096;
    int nblk = 0;                   // blocks of the selected flow variant
    int fv = 0, hv = 0;             // selected flow / heat variants
    int version = 0;                // bumped when captured launch parameters change
    cudaGraphExec_t graph = nullptr;   // two steps
    cudaGraphExec_t graph8 = nullptr;  // eight steps
    bool timing = false;
    std::vector<EventPair> ev[3];
    double t_ms[3] = {0, 0, 0};
    int64_t t_count = 0;
    // optional device allocator (lbm_opts_t.dev_alloc / dev_free)
    void *(*dev_alloc)(size_t, void *) = nullptr;
    void (*dev_free)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    bool bounds_check = false;
    std::string msg;
};

void lbmgb::set_global_error(const std::string &msg) { g_create_error = msg; }

static int fail(lbm_run *h, int code, const std::string &m) {
    if (h) h->msg = m; else g_create_error = m;
    return code;
}
static int cuda_fail(lbm_run *h, cudaError_t e, const char *where) {
    return fail(h, LBM_E_CUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}
#define CK(h, call)                                     \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

static StepBuffers buffers(lbm_run *h, int par) {
    StepBuffers b{};
    b.f_in = h->f[par];
    b.f_out = h->f[par ^ 1];
    b.T_in = h->T[par];
    b.T_out = h->T[par ^ 1];
    b.rho = h->rho[par];
    b.ux = h->ux[par];
    b.uy = h->uy[par];
    b.cw = h->cw;
    b.part = h->part[par];
    b.err = h->err;
    b.wq = h->err + 2;  // words 2, 3 of the run's error-word block
    b.step = h->dstep;
    b.series = h->series;
    b.series_cap = h->series_cap;
    b.q_top = h->q_top;
    b.last = h->last;
    b.scratch = h->scratch;
    b.mdesc = h->mdesc ? static_cast<const char *>(h->mdesc) + par * h->ks->multi_desc_bytes : nullptr;
    return b;
}
// Buffers describing the current state as the "output" side (init / import)
// and as the "input" side (export).
static StepBuffers state_as_out(lbm_run *h) { return buffers(h, h->parity ^ 1); }
static StepBuffers state_as_in(lbm_run *h) {
    StepBuffers b = buffers(h, h->parity);
    // the moments of the last step were written with the other parity
    b.rho = h->rho[h->parity ^ 1];
    b.ux = h->ux[h->parity ^ 1];
    b.uy = h->uy[h->parity ^ 1];
    return b;
}

// Device memory of a run: cudaMalloc / cudaFree, or the caller's allocator.
static cudaError_t dalloc(lbm_run *h, void **p, size_t bytes) {
    if (!h->dev_alloc) return cudaMalloc(p, bytes);
    *p = h->dev_alloc(bytes, h->alloc_ctx);
    if (!*p) return cudaErrorMemoryAllocation;
    if ((reinterpret_cast<uintptr_t>(*p) & 255u) != 0) {  // TMA and vector loads need aligned bases
        h->dev_free(*p, h->alloc_ctx);
        *p = nullptr;
        return cudaErrorMisalignedAddress;
    }
    return cudaSuccess;
}
static void dfree(lbm_run *h, void *p) {
    if (!p) return;
    if (h->dev_free) h->dev_free(p, h->alloc_ctx);
    else cudaFree(p);
}
// cudaFree waits for the device; a caller's allocator may not, so the run's
// queued work is finished first
static void quiesce(lbm_run *h) {
    if (!h->dev_free) return;
    if (h->dstream) cudaStreamSynchronize(h->dstream);
    if (h->stream) cudaStreamSynchronize(h->stream);
}

static void free_all(lbm_run *h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->graph8) cudaGraphExecDestroy(h->graph8);
    quiesce(h);
    for (int k = 0; k < 2; k++) {
        dfree(h, h->f[k]);
        dfree(h, h->T[k]);
    }
    for (int k = 0; k < 2; k++) {
        dfree(h, h->rho[k]); dfree(h, h->ux[k]); dfree(h, h->uy[k]); dfree(h, h->part[k]);
    }
    dfree(h, h->cw); dfree(h, h->series); dfree(h, h->q_top); dfree(h, h->last);
    for (cudaEvent_t ev : {h->ev_heat, h->ev_diag, h->cev_heat, h->cev_diag})
        if (ev) cudaEventDestroy(ev);
    if (h->dstream) cudaStreamDestroy(h->dstream);
    dfree(h, h->scratch); dfree(h, h->stage); dfree(h, h->err); dfree(h, h->dstep); dfree(h, h->mdesc);
    for (auto &v : h->ev)
        for (auto &e : v) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Host-side constants, evaluated in FP64 in the order the formulas are written
// (the library is built with -ffp-contract=off).
static int fill_params(const lbm_domain_t *d, const lbm_heater_t *ht, const lbm_eos_t *eo, const lbm_bc_t *bc,
                       DevParams &p, std::string &why) {
    if (d->nx < 1) { why = "domain.nx must be >= 1"; return 0; }
    if (d->ny_fluid < 2) { why = "domain.ny_fluid must be >= 2"; return 0; }
    if (d->liquid_rows < 0 || d->liquid_rows > d->ny_fluid) { why = "domain.liquid_rows out of range"; return 0; }
    if (d->top_mode != LBM_TOP_WALL && d->top_mode != LBM_TOP_OUTFLOW) { why = "domain.top_mode invalid"; return 0; }
    if (d->flags & ~7) { why = "domain.flags has unknown bits"; return 0; }
    const bool py = (d->flags & LBM_PERIODIC_Y) != 0;
    if (py && ht->ny_solid != 0) { why = "periodic-y test mode needs heater.ny_solid = 0"; return 0; }
    const bool model_a = !py && ht->ny_solid == 0;  // Fig. 1a: no heater
    if (!py && !model_a && ht->ny_solid < 3) {
        why = "heater.ny_solid must be 0 (Model A) or >= 3 (bottom flux uses rows 0..2)";
        return 0;
    }
    if ((double)d->nx * (double)(d->ny_fluid + ht->ny_solid + 1) > 2.0e9) { why = "domain too large for 32-bit row indexing"; return 0; }
    if (!(eo->G < 0)) { why = "eos.G must be negative (psi real for p_EOS < rho/3)"; return 0; }
    if (!(eo->a > 0 && eo->b > 0 && eo->R > 0)) { why = "eos.a, eos.b, eos.R must be positive"; return 0; }
    if (!(eo->rho_L > eo->rho_V && eo->rho_V > 0)) { why = "eos needs rho_L > rho_V > 0"; return 0; }
    if (!(d->nu_L > 0 && d->nu_V > 0)) { why = "viscosities must be positive"; return 0; }
    for (int k = 0; k < 9; k++)
        if (!(d->s[k] > 0 && d->s[k] < 2)) { why = "MRT rates must lie in (0, 2)"; return 0; }
    if (!(d->c_v > 0 && d->cv_chi > 0)) { why = "c_v and cv_chi must be positive"; return 0; }
    if (!py && !model_a && !(ht->lambda_s > 0 && ht->rho_c_s > 0)) { why = "heater lambda_s and rho_c_s must be positive"; return 0; }
    if (bc->mode < 0 || bc->mode > 2) { why = "bc.mode invalid"; return 0; }
    if (bc->n_spots < 0 || bc->n_spots > 8) { why = "bc.n_spots must be in 0..8"; return 0; }
    if (bc->mode == LBM_BC_SINE && !(bc->sine_wavelength > 0)) { why = "bc.sine_wavelength must be positive"; return 0; }
    p.nx = d->nx;
    p.nf = d->ny_fluid;
    // Model A: temperature row 0 is the wall's Dirichlet row (T_b), coupled to
    // the first fluid row with the fluid's conductivity
    p.ns = model_a ? 1 : ht->ny_solid;
    p.nt = p.ns + p.nf;
    p.flags = d->flags | (model_a ? FLAG_MODEL_A : 0);
    p.top_mode = d->top_mode;
    p.bc_mode = bc->mode;
    p.liquid_rows = d->liquid_rows;
    p.a = eo->a; p.b = eo->b; p.R = eo->R; p.G = eo->G;
    p.Tc = (0.0778 * eo->a) / ((0.45724 * eo->b) * eo->R);
    p.kappa = 0.37464 + 1.54226 * eo->omega - 0.26992 * eo->omega * eo->omega;
    p.T_sat = eo->T_sat_over_Tc * p.Tc;
    p.T_b = bc->T_b_over_Tc * p.Tc;
    p.rho_L = eo->rho_L; p.rho_V = eo->rho_V;
    p.rho_mean = d->rho_mean;
    p.g = d->g; p.c_v = d->c_v; p.cv_chi = d->cv_chi;
    p.lambda_s = ht->lambda_s; p.rho_c_s = ht->rho_c_s;
    p.tau_L = 3.0 * d->nu_L + 0.5;
    p.tau_V = 3.0 * d->nu_V + 0.5;
    p.drho_LV = eo->rho_L - eo->rho_V;
    p.dtau_LV = p.tau_L - p.tau_V;
    for (int k = 0; k < 9; k++) {
        p.s[k] = d->s[k];
        p.hs[k] = 1.0 - 0.5 * d->s[k];
    }
    p.tau_e_m = 1.0 / d->s[1] - 0.5;
    p.tau_s_m = 1.0 / d->s[2] - 0.5;
    p.varpi12 = 12.0 * d->varpi;
    p.sign_eps = d->sign_eps;
    p.c_w_top = bc->c_w_top;
    p.bc_noise = bc->noise_amp;
    p.sine_amp = bc->sine_amp_over_Tc * p.Tc;
    p.sine_wl = bc->sine_wavelength;
    p.sine_t0 = bc->sine_t0;
    p.sine_t1 = bc->sine_t1;
    p.init_noise = d->init_noise;
    p.vap_threshold = 0.5 * (eo->rho_L + eo->rho_V);
    p.seed = d->seed;
    // Test hook for the bounded waits of the staged-copy flow kernel: a
    // positive LBM_TEST_TX_PAD makes its stages expect more bytes than the
    // copies deliver, so every wait runs out and the step reports
    // LBM_E_TIMEOUT.  Unset in normal use.
    const char *pad = std::getenv("LBM_TEST_TX_PAD");
    p.tx_pad = pad ? (unsigned)std::strtoul(pad, nullptr, 10) : 0u;
    return 1;
}

// Device address of page-locked host memory mapped for the current device,
// or nullptr (pageable memory, or not a host pointer).
template <class V>
static const V *host_alias(const V *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? static_cast<const V *>(a.devicePointer) : nullptr;
}

static int ensure_stage(lbm_run *h, size_t elems) {
    if (h->stage_elems >= elems) return LBM_OK;
    quiesce(h);
    dfree(h, h->stage);
    h->stage = nullptr;
    h->stage_elems = 0;
    if (dalloc(h, (void **)&h->stage, elems * sizeof(double)) != cudaSuccess)
        return fail(h, LBM_E_NOMEM, "staging allocation failed");
    h->stage_elems = elems;
    return LBM_OK;
}

static int check_err_word(lbm_run *h) {
    unsigned e = 0;
    CK(h, cudaMemcpyAsync(&e, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (e & ERRW_TIMEOUT)
        return fail(h, LBM_E_TIMEOUT, "a kernel's wait for its staged data ran out (the step's results are invalid)");
    if (e & ERRW_DESC)
        return fail(h, LBM_E_STATE, "a multi-run kernel found a descriptor it could not trust and skipped its tile");
    if (e) {
        std::string m = "numerical fault latched by the kernels:";
        if (e & ERRW_PSI) m += " negative pseudopotential radicand;";
        if (e & ERRW_NONFINITE_RHO) m += " non-finite density;";
        if (e & ERRW_NONFINITE_T) m += " non-finite temperature;";
        return fail(h, LBM_E_NUMERIC, m);
    }
    return LBM_OK;
}

extern "C" {

const char *lbm_status_string(int s) {
    switch (s) {
        case LBM_OK: return "LBM_OK";
        case LBM_E_INVAL: return "LBM_E_INVAL";
        case LBM_E_NOMEM: return "LBM_E_NOMEM";
        case LBM_E_CUDA: return "LBM_E_CUDA";
        case LBM_E_NUMERIC: return "LBM_E_NUMERIC";
        case LBM_E_TIMEOUT: return "LBM_E_TIMEOUT";
        case LBM_E_STATE: return "LBM_E_STATE";
        default: return "unknown status";
    }
}

const char *lbm_last_error(lbm_handle h) { return h ? h->msg.c_str() : g_create_error.c_str(); }

int lbm_create(const lbm_domain_t *domain, const lbm_heater_t *heater, const lbm_eos_t *eos, const lbm_bc_t *bc,
               const lbm_opts_t *opts, lbm_handle *out) {
    if (!out) return fail(nullptr, LBM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!domain || !heater || !eos || !bc || !opts) return fail(nullptr, LBM_E_INVAL, "a configuration struct is NULL");
    lbm_run *h = new (std::nothrow) lbm_run();
    if (!h) return fail(nullptr, LBM_E_NOMEM, "host allocation failed");
    std::string why;
    if (!fill_params(domain, heater, eos, bc, h->p, why)) {
        delete h;
        return fail(nullptr, LBM_E_INVAL, why);
    }
    switch (opts->precision) {
        case LBM_FP64: h->ks = kernels_fp64(); break;
        case LBM_FP32: h->ks = kernels_fp32(); break;
        case LBM_FP16: h->ks = kernels_fp16(); break;
        case LBM_FP32_DFSRC: h->ks = kernels_fp32_dfsrc(); break;
        case LBM_FP64_FMA: h->ks = kernels_fp64_fma(); break;
        default: delete h; return fail(nullptr, LBM_E_INVAL, "opts.precision invalid");
    }
    if ((opts->dev_alloc == nullptr) != (opts->dev_free == nullptr)) {
        delete h;
        return fail(nullptr, LBM_E_INVAL, "opts.dev_alloc and opts.dev_free must be set together");
    }
    h->dev_alloc = opts->dev_alloc;
    h->dev_free = opts->dev_free;
    h->alloc_ctx = opts->alloc_ctx;
    h->bounds_check = opts->bounds_check != 0;
    h->device = opts->device;
    h->use_graphs = opts->use_graphs != 0;
    if (opts->series_capacity < 0) { delete h; return fail(nullptr, LBM_E_INVAL, "opts.series_capacity negative"); }
    if (opts->series_capacity > 0) h->series_cap = opts->series_capacity;
    int rc = LBM_OK;
    auto bad = [&](int code) { rc = code; free_all(h); std::string m = h->msg; delete h; g_create_error = m; return rc; };
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) { cuda_fail(h, e, "cudaSetDevice"); return bad(LBM_E_CUDA); }
    if (opts->stream) {
        h->stream = (cudaStream_t)opts->stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { cuda_fail(h, e, "cudaStreamCreate"); return bad(LBM_E_CUDA); }
        h->own_stream = true;
    }
    if ((e = cudaStreamCreateWithFlags(&h->dstream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_heat, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_diag, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->cev_heat, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->cev_diag, cudaEventDisableTiming)) != cudaSuccess) {
        cuda_fail(h, e, "diagnostics stream");
        return bad(LBM_E_CUDA);
    }
    for (int v = 0; v < h->ks->n_heat; v++)
        if ((e = h->ks->heat[v].prepare()) != cudaSuccess) { cuda_fail(h, e, "kernel attributes"); return bad(LBM_E_CUDA); }
    for (int v = 0; v < h->ks->n_flow; v++)
        if ((e = h->ks->flow[v].prepare()) != cudaSuccess) { cuda_fail(h, e, "kernel attributes"); return bad(LBM_E_CUDA); }
    const DevParams &p = h->p;
    const size_t nfl = (size_t)p.nx * p.nf, ntl = (size_t)p.nx * p.nt;
    int max_blocks = 0;
    for (int v = 0; v < h->ks->n_flow; v++) max_blocks = std::max(max_blocks, h->ks->flow[v].blocks(p));
    h->nblk = h->ks->flow[0].blocks(p);
    struct A { void **ptr; size_t bytes; } allocs[] = {
        {&h->f[0], 9 * nfl * h->ks->f_elem}, {&h->f[1], 9 * nfl * h->ks->f_elem},
        {&h->T[0], ntl * h->ks->T_elem}, {&h->T[1], ntl * h->ks->T_elem},
        {&h->rho[0], nfl * h->ks->m_elem}, {&h->ux[0], nfl * h->ks->m_elem}, {&h->uy[0], nfl * h->ks->m_elem},
        {&h->rho[1], nfl * h->ks->m_elem}, {&h->ux[1], nfl * h->ks->m_elem}, {&h->uy[1], nfl * h->ks->m_elem},
        {(void **)&h->cw, (size_t)p.nx * sizeof(double)},
        {(void **)&h->part[0], 2 * (size_t)max_blocks * sizeof(double)},
        {(void **)&h->part[1], 2 * (size_t)max_blocks * sizeof(double)},
        {(void **)&h->series, (size_t)h->series_cap * SERIES_WIDTH * sizeof(double)},
        {(void **)&h->q_top, (size_t)p.nx * sizeof(double)}, {(void **)&h->last, SERIES_WIDTH * sizeof(double)},
        {(void **)&h->scratch, 1024 * sizeof(double)}, {(void **)&h->err, 4 * sizeof(unsigned)},
        {(void **)&h->dstep, sizeof(long long)},
        {&h->mdesc, 2 * h->ks->multi_desc_bytes},
    };
    for (auto &a : allocs) {
        if (a.bytes == 0) continue;
        e = dalloc(h, a.ptr, a.bytes);
        if (e != cudaSuccess) {
            fail(h, LBM_E_NOMEM, std::string("device allocation of ") + std::to_string(a.bytes) + " bytes failed: " +
                                     (e == cudaErrorMisalignedAddress ? "opts.dev_alloc returned memory not aligned to 256 bytes"
                                                                      : cudaGetErrorString(e)));
            return bad(LBM_E_NOMEM);
        }
    }
    // heater-surface wettability per column (nucleate spots: columns within
    // spot_half_width periodic distance of a spot centre, Sec. 4.1)
    std::vector<double> cwh(p.nx);
    for (int x = 0; x < p.nx; x++) {
        double c = bc->c_w_base;
        for (int k = 0; k < bc->n_spots; k++) {
            int dx = ((x - bc->spot_x[k]) % p.nx + p.nx) % p.nx;
            if (dx > p.nx - dx) dx = p.nx - dx;
            if (dx <= bc->spot_half_width) c = bc->c_w_spot[k];
        }
        cwh[x] = c;
    }
    long long zero = 0;
    if ((e = cudaMemcpyAsync(h->cw, cwh.data(), p.nx * sizeof(double), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h->dstep, &zero, sizeof(zero), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->err, 0, 4 * sizeof(unsigned), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->last, 0, SERIES_WIDTH * sizeof(double), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->q_top, 0, p.nx * sizeof(double), h->stream)) != cudaSuccess) {
        cuda_fail(h, e, "initial copies");
        return bad(LBM_E_CUDA);
    }
    // initial state (Sec. 3.1): densities, their mean, then populations and T
    StepBuffers b = state_as_out(h);
    if ((e = h->ks->init(h->p, b, 0, h->stream)) != cudaSuccess) { cuda_fail(h, e, "init kernels"); return bad(LBM_E_CUDA); }
    double sum = 0;
    if ((e = cudaMemcpyAsync(&sum, h->scratch, sizeof(double), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
        cuda_fail(h, e, "initial density read-back");
        return bad(LBM_E_CUDA);
    }
    if (!(h->p.rho_mean > 0)) h->p.rho_mean = sum / (double)nfl;
    h->p.rho_shift = (opts->rho_shift > 0) ? opts->rho_shift : h->p.rho_mean;
    if ((e = h->ks->init(h->p, b, 1, h->stream)) != cudaSuccess) { cuda_fail(h, e, "init kernels"); return bad(LBM_E_CUDA); }
    if (h->mdesc) {
        // the run's own multi-run descriptors (for the "multi" launch-shape
        // variants), one per state parity, now that rho_mean is fixed
        const size_t db = h->ks->multi_desc_bytes;
        std::vector<char> hd(2 * db);
        for (int par = 0; par < 2; par++)
            h->ks->multi_fill(h->p, buffers(h, 0), buffers(h, 1), par, 0, 0, 0, hd.data() + par * db);
        if ((e = cudaMemcpyAsync(h->mdesc, hd.data(), 2 * db, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
            cuda_fail(h, e, "run descriptors");
            return bad(LBM_E_CUDA);
        }
    }
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { cuda_fail(h, e, "init sync"); return bad(LBM_E_CUDA); }
    *out = h;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h) {
    if (!h) return LBM_OK;
    cudaSetDevice(h->device);
    if (h->dstream) cudaStreamSynchronize(h->dstream);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return LBM_OK;
}

static cudaError_t launch_kernel(lbm_run *h, int k, const StepBuffers &b) {
    if (k == 0) return h->ks->flow[h->fv].launch(h->p, b, h->stream);
    if (k == 1) return h->ks->heat[h->hv].launch(h->p, b, h->stream);
    // per-kernel timing runs the diagnostics on the main stream, so its events
    // time the kernel itself rather than its wait behind an overlapping kernel
    return h->ks->diag(h->p, b, h->nblk, h->timing ? h->stream : h->dstream);
}

// Make the main stream wait for the last queued diagnostics kernel.  Events
// recorded inside a stream capture cannot be waited on outside it, so
// captures use their own pair.
static cudaError_t join_diag(lbm_run *h, bool capturing = false) {
    return cudaStreamWaitEvent(h->stream, capturing ? h->cev_diag : h->ev_diag, 0);
}

// One step: flow and heat on the main stream, diagnostics on the side
// stream after the heat kernel.  The next step's flow kernel does not wait
// for the diagnostics (moments and partials are double-buffered); its heat
// kernel does (it reads the step counter the diagnostics kernel advances).
// wait_prev_diag is false for the first step of a stream capture, which is
// ordered after earlier work by the graph launch itself.
static int launch_step(lbm_run *h, bool timed, bool wait_prev_diag = true, bool capturing = false) {
    StepBuffers b = buffers(h, h->parity);
    cudaError_t e;
    cudaEvent_t eh = capturing ? h->cev_heat : h->ev_heat, ed = capturing ? h->cev_diag : h->ev_diag;
    // The heat kernel reads the step counter the previous diagnostics kernel
    // advanced, so it waits for it; the flow kernel overlaps that kernel,
    // except with FP16 storage, whose store dither is keyed by the counter.
    const int first_reader = h->ks->f_elem == 2 ? 0 : 1;
    for (int k = 0; k < 3; k++) {
        cudaStream_t st = (k == 2 && !h->timing) ? h->dstream : h->stream;
        if (k == first_reader && wait_prev_diag) CK(h, cudaStreamWaitEvent(h->stream, ed, 0));
        if (k == 2 && !h->timing) {
            CK(h, cudaEventRecord(eh, h->stream));
            CK(h, cudaStreamWaitEvent(h->dstream, eh, 0));
        }
        EventPair ep;
        if (timed) {
            CK(h, cudaEventCreate(&ep.a));
            CK(h, cudaEventCreate(&ep.b));
            CK(h, cudaEventRecord(ep.a, st));
        }
        if ((e = launch_kernel(h, k, b)) != cudaSuccess) return cuda_fail(h, e, k == 0 ? "flow kernel" : (k == 1 ? "heat kernel" : "diagnostics kernel"));
        if (timed) {
            CK(h, cudaEventRecord(ep.b, st));
            h->ev[k].push_back(ep);
        }
        if (k == 2) CK(h, cudaEventRecord(ed, st));
    }
    h->parity ^= 1;
    return LBM_OK;
}

static int build_graph(lbm_run *h, int nsteps, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    for (int i = 0; i < nsteps && rc == LBM_OK; i++) rc = launch_step(h, false, i > 0, true);
    cudaError_t ej = (rc == LBM_OK) ? join_diag(h, true) : cudaSuccess;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc != LBM_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (ej != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(h, ej, "graph join"); }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { *out = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
    return LBM_OK;
}

int lbm_step(lbm_handle h, int64_t n) {
    if (!h) return LBM_E_INVAL;
    if (n < 0) return fail(h, LBM_E_INVAL, "negative step count");
    CK(h, cudaSetDevice(h->device));
    if (n > 0) h->diag_stale = false;  // the diagnostics kernel of these steps runs before any read-back
    int rc;
    if (h->bounds_check) {  // one step at a time, each waited for and checked
        while (n > 0) {
            if ((rc = launch_step(h, h->timing)) != LBM_OK) return rc;
            n -= 1;
            h->steps += 1;
            CK(h, join_diag(h));
            CK(h, cudaStreamSynchronize(h->dstream));
            CK(h, cudaStreamSynchronize(h->stream));
            CK(h, cudaGetLastError());
            if ((rc = check_err_word(h)) != LBM_OK) return rc;
        }
        return LBM_OK;
    }
    const bool graphs = h->use_graphs && !h->timing && h->stream != nullptr;
    while (n > 0) {
        if (graphs && n >= 8 && h->parity == 0) {
            if (!h->graph8 && (rc = build_graph(h, 8, &h->graph8)) != LBM_OK) return rc;
            CK(h, join_diag(h));  // the graph's first heat kernel reads the step counter
            CK(h, cudaGraphLaunch(h->graph8, h->stream));
            n -= 8;
            h->steps += 8;
            continue;
        }
        if (graphs && n >= 2 && h->parity == 0) {
            if (!h->graph && (rc = build_graph(h, 2, &h->graph)) != LBM_OK) return rc;
            CK(h, join_diag(h));
            CK(h, cudaGraphLaunch(h->graph, h->stream));
            n -= 2;
            h->steps += 2;
            continue;
        }
        if ((rc = launch_step(h, h->timing)) != LBM_OK) return rc;
        n -= 1;
        h->steps += 1;
    }
    // later work on the main stream sees this call's diagnostics
    CK(h, join_diag(h));
    return LBM_OK;
}

int lbm_sync(lbm_handle h) {
    if (!h) return LBM_E_INVAL;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->dstream));
    CK(h, cudaStreamSynchronize(h->stream));
    return check_err_word(h);
}

int64_t lbm_step_count(lbm_handle h) { return h ? h->steps : -1; }

int lbm_get_state(lbm_handle h, double *f, double *T, int64_t *step, int dst_is_device) {
    if (!h) return LBM_E_INVAL;
    double *dst[2] = {nullptr, nullptr};
    unsigned mask = 0;
    int j = 0;
    if (T) { mask |= LBM_FIELD_T; dst[j++] = T; }  // lbm_fields takes T before F
    if (f) { mask |= LBM_FIELD_F; dst[j++] = f; }
    const int rc = mask ? lbm_fields(h, mask, dst, dst_is_device) : LBM_OK;
    if (rc == LBM_OK && step) *step = h->steps;
    return rc;
}

int lbm_fields(lbm_handle h, unsigned mask, double *const *dst, int dst_is_device) {
    if (!h) return LBM_E_INVAL;
    if (mask & ~31u) return fail(h, LBM_E_INVAL, "unknown field bits");
    if (mask && !dst) return fail(h, LBM_E_INVAL, "dst is NULL");
    CK(h, cudaSetDevice(h->device));
    const size_t nfl = (size_t)h->p.nx * h->p.nf, ntl = (size_t)h->p.nx * h->p.nt;
    const size_t sizes[5] = {nfl, nfl, nfl, ntl, 9 * nfl};
    double *dptr[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t off[5] = {0, 0, 0, 0, 0}, total = 0;
    int j = 0;
    for (int k = 0; k < 5; k++) {
        if (!(mask & (1u << k))) continue;
        if (!dst[j]) return fail(h, LBM_E_INVAL, "a destination pointer is NULL");
        off[k] = total;
        total += sizes[k];
        j++;
    }
    int rc;
    if (!dst_is_device && total) {
        if ((rc = ensure_stage(h, total)) != LBM_OK) return rc;
    }
    j = 0;
    for (int k = 0; k < 5; k++) {
        if (!(mask & (1u << k))) continue;
        dptr[k] = dst_is_device ? dst[j] : h->stage + off[k];
        j++;
    }
    StepBuffers b = state_as_in(h);
    cudaError_t e = h->ks->export_fields(h->p, b, dptr[0], dptr[1], dptr[2], dptr[3], dptr[4], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "export kernel");
    if (!dst_is_device) {
        j = 0;
        for (int k = 0; k < 5; k++) {
            if (!(mask & (1u << k))) continue;
            CK(h, cudaMemcpyAsync(dst[j], dptr[k], sizes[k] * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            j++;
        }
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return check_err_word(h);
}

// lbm_set_state / lbm_set_state_f32: V is the arrays' type.
extern "C++" {
template <class V>
static int set_state(lbm_handle h, const V *f, const V *T, int64_t step, int src_is_device) {
    if (!h) return LBM_E_INVAL;
    if (step < 0) return fail(h, LBM_E_INVAL, "negative step");
    CK(h, cudaSetDevice(h->device));
    const size_t nfl = (size_t)h->p.nx * h->p.nf, ntl = (size_t)h->p.nx * h->p.nt;
    const V *df = f, *dT = T;
    int rc;
    if (!src_is_device && (f || T)) {
        // Page-locked host memory the device can address is read by the
        // import kernel itself (over NVLink-C2C on Grace: copy and conversion
        // in one pass); other host memory is staged with an async copy (the
        // stage holds 9 NF NX + NT NX doubles, room for either type).
        const V *af = host_alias(f), *aT = host_alias(T);
        if ((f && !af) || (T && !aT)) {
            if ((rc = ensure_stage(h, 9 * nfl + ntl)) != LBM_OK) return rc;
        }
        V *stage = reinterpret_cast<V *>(h->stage);
        if (f) {
            if (af) {
                df = af;
            } else {
                CK(h, cudaMemcpyAsync(stage, f, 9 * nfl * sizeof(V), cudaMemcpyHostToDevice, h->stream));
                df = stage;
            }
        }
        if (T) {
            if (aT) {
                dT = aT;
            } else {
                CK(h, cudaMemcpyAsync(stage + 9 * nfl, T, ntl * sizeof(V), cudaMemcpyHostToDevice, h->stream));
                dT = stage + 9 * nfl;
            }
        }
    }
    // write into the current state buffers
    StepBuffers b = buffers(h, h->parity ^ 1);
    b.f_out = h->f[h->parity];
    b.T_out = h->T[h->parity];
    if (df || dT) {
        cudaError_t e;
        if constexpr (sizeof(V) == sizeof(double)) e = h->ks->import_state(h->p, (const double *)df, (const double *)dT, b, h->stream);
        else e = h->ks->import_state32(h->p, (const float *)df, (const float *)dT, b, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "import kernel");
    }
    long long s = step;
    CK(h, cudaMemcpyAsync(h->dstep, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));  // host sources may be freed after return
    h->steps = step;
    // the diagnostics ring and the last-step values describe the previous
    // trajectory: rows before `step` are no longer served, and the scalar
    // readers refuse until a step of the new state has run
    h->series_from = step;
    h->diag_stale = true;
    return LBM_OK;
}
}  // extern "C++"

int lbm_set_state(lbm_handle h, const double *f, const double *T, int64_t step, int src_is_device) {
    return set_state(h, f, T, step, src_is_device);
}

int lbm_set_state_f32(lbm_handle h, const float *f, const float *T, int64_t step, int src_is_device) {
    return set_state(h, f, T, step, src_is_device);
}

static const char *kStaleDiag = "no step has run since lbm_set_state: the diagnostics describe the previous state";

int lbm_wall_heat_flux(lbm_handle h, double *q_bottom_mean, double *q_top_local) {
    if (!h) return LBM_E_INVAL;
    if (h->diag_stale) return fail(h, LBM_E_STATE, kStaleDiag);
    CK(h, cudaSetDevice(h->device));
    double last[SERIES_WIDTH];
    CK(h, cudaMemcpyAsync(last, h->last, sizeof(last), cudaMemcpyDeviceToHost, h->stream));
    if (q_top_local) CK(h, cudaMemcpyAsync(q_top_local, h->q_top, h->p.nx * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (q_bottom_mean) *q_bottom_mean = last[0];
    return check_err_word(h);
}

static int read_last(lbm_run *h, int k, double *out) {
    if (!h || !out) return LBM_E_INVAL;
    if (h->diag_stale) return fail(h, LBM_E_STATE, kStaleDiag);
    CK(h, cudaSetDevice(h->device));
    double last[SERIES_WIDTH];
    CK(h, cudaMemcpyAsync(last, h->last, sizeof(last), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *out = last[k];
    return check_err_word(h);
}

int lbm_vapour_fraction(lbm_handle h, double *out) { return read_last(h, 2, out); }
int lbm_mass(lbm_handle h, double *out) { return read_last(h, 3, out); }

int lbm_series(lbm_handle h, int64_t first, int64_t count, double *out) {
    if (!h) return LBM_E_INVAL;
    if (count < 0 || (count > 0 && !out)) return fail(h, LBM_E_INVAL, "bad count or NULL out");
    if (count == 0) return LBM_OK;
    if (first < h->series_from || first + count > h->steps || h->steps - first > h->series_cap)
        return fail(h, LBM_E_INVAL, "requested steps are not in the diagnostics ring");
    CK(h, cudaSetDevice(h->device));
    for (int64_t k = 0; k < count;) {
        const int64_t slot = (first + k) % h->series_cap;
        const int64_t run = std::min<int64_t>(count - k, h->series_cap - slot);
        CK(h, cudaMemcpyAsync(out + k * SERIES_WIDTH, h->series + slot * SERIES_WIDTH, run * SERIES_WIDTH * sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
        k += run;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return check_err_word(h);
}

int lbm_set_timing(lbm_handle h, int enable) {
    if (!h) return LBM_E_INVAL;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto &v : h->ev) {
        for (auto &e : v) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
        v.clear();
    }
    for (double &t : h->t_ms) t = 0;
    h->t_count = 0;
    h->timing = enable != 0;
    return LBM_OK;
}

int lbm_kernel_times(lbm_handle h, double *avg_ms, int64_t *launches) {
    if (!h || !avg_ms) return LBM_E_INVAL;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 3; k++) {
        for (auto &e : h->ev[k]) {
            float ms = 0;
            CK(h, cudaEventElapsedTime(&ms, e.a, e.b));
            h->t_ms[k] += ms;
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
        if (k == 0) h->t_count += (int64_t)h->ev[0].size();
        h->ev[k].clear();
    }
    for (int k = 0; k < 3; k++) avg_ms[k] = h->t_count ? h->t_ms[k] / (double)h->t_count : 0.0;
    if (launches) *launches = h->t_count;
    return LBM_OK;
}

int lbm_kernels_per_step(lbm_handle h) { return h ? 3 : 0; }

}  // extern "C"

// ---- batches of runs ---------------------------------------------------------
// Runs of one kernel set that has multi-run kernels are stepped together:
// per step one flow, one heat and one diagnostics launch over all their
// work items -- one group per launch mode (wavefront flow or tiles, heat
// tiles staged as whole rows or cell by cell).  The other runs of a batch are stepped by their
// own kernels, one concurrent branch per run.
struct MultiGroup {
    const KernelSet *ks = nullptr;
    int mode = 0;                   // launch mode: bit 0 wavefront flow units, bit 1 whole-row heat staging
    unsigned *wq = nullptr;         // 2 words: the wavefront launches' work counter
    std::vector<int> idx;           // positions in the batch's run list
    void *desc = nullptr;           // device descriptors, in idx order
    std::vector<char> host;         // their host image
    int flow_tiles = 0, heat_tiles = 0;
    cudaStream_t gs = nullptr, gd = nullptr;       // kernel and diagnostics streams
    cudaEvent_t ev_heat = nullptr, ev_diag = nullptr;    // inside graph captures
    cudaEvent_t xev_heat = nullptr, xev_diag = nullptr;  // plain launches
};

struct lbm_batch_s {
    std::vector<lbm_run *> runs;
    std::vector<int> versions;
    std::vector<int> parities;      // each run's buffer parity when the graph was captured
    std::vector<cudaEvent_t> join;
    std::vector<bool> in_group;     // stepped by a multi-run group
    std::vector<MultiGroup> groups;
    unsigned *errw = nullptr;       // error word of the groups' launches (ERRW_DESC)
    cudaEvent_t fork = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int device = 0;
    std::string msg;
};

static int bfail(lbm_batch_s *b, int code, const std::string &m) {
    if (b) b->msg = m; else g_create_error = m;
    return code;
}

static void batch_free(lbm_batch_s *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto &g : b->groups) {
        if (g.desc) cudaFree(g.desc);
        if (g.wq) cudaFree(g.wq);
        for (cudaEvent_t ev : {g.ev_heat, g.ev_diag, g.xev_heat, g.xev_diag})
            if (ev) cudaEventDestroy(ev);
        for (cudaStream_t st : {g.gs, g.gd})
            if (st) cudaStreamDestroy(st);
    }
    if (b->errw) cudaFree(b->errw);
    if (b->stream) cudaStreamDestroy(b->stream);
}

// Descriptors of every group's runs for their current state parities
// (phase 0 of the next launches), uploaded before any launch that uses them.
static int batch_fill_groups(lbm_batch_s *b) {
    // launches queued earlier may still read the descriptors: they all end
    // up on the batch stream
    if (!b->groups.empty()) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("batch sync: ") + cudaGetErrorString(e));
    }
    for (auto &g : b->groups) {
        const size_t db = g.ks->multi_desc_bytes;
        int f0 = 0, h0 = 0;
        for (size_t k = 0; k < g.idx.size(); k++) {
            lbm_run *h = b->runs[g.idx[k]];
            g.ks->multi_fill(h->p, buffers(h, 0), buffers(h, 1), h->parity, g.mode, f0, h0, g.host.data() + k * db);
            f0 += g.ks->multi_flow_items(h->p, g.mode);
            h0 += g.ks->multi_heat_tiles(h->p);
        }
        g.flow_tiles = f0;
        g.heat_tiles = h0;
        // ordered on the batch stream and waited for: a plain cudaMemcpy from
        // pageable memory may return before its data lands, and it is not
        // ordered with the non-blocking streams the kernels run on
        cudaError_t e = cudaMemcpyAsync(g.desc, g.host.data(), g.host.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("batch descriptors: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}

// One step (phase 0 or 1 of the current descriptors) of every group, ordered
// after `from` and joined back into it.  As for a single run, the
// diagnostics run on their own stream under the next step's flow kernel; the
// heat kernel (and with FP16 storage also the flow kernel) waits for the
// previous step's diagnostics, which advance the step counters.
static cudaError_t batch_groups_step(lbm_batch_s *b, int phase, bool first, bool captured, cudaEvent_t fork) {
    cudaError_t e = cudaSuccess;
    for (auto &g : b->groups) {
        cudaEvent_t ev_heat = captured ? g.ev_heat : g.xev_heat, ev_diag = captured ? g.ev_diag : g.xev_diag;
        const int n = (int)g.idx.size();
        const bool fp16 = g.ks->f_elem == 2;
        if (first) {
            if ((e = cudaStreamWaitEvent(g.gs, fork, 0)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(g.gd, fork, 0)) != cudaSuccess) return e;
        } else if (fp16 && (e = cudaStreamWaitEvent(g.gs, ev_diag, 0)) != cudaSuccess) {
            return e;
        }
        if ((e = g.ks->multi_launch((g.mode & 1) ? 3 : 0, g.desc, n, g.flow_tiles, phase, b->errw, g.wq, g.gs)) !=
            cudaSuccess)
            return e;
        if (!first && !fp16 && (e = cudaStreamWaitEvent(g.gs, ev_diag, 0)) != cudaSuccess) return e;
        if ((e = g.ks->multi_launch((g.mode & 2) ? 4 : 1, g.desc, n, g.heat_tiles, phase, b->errw, g.wq, g.gs)) !=
            cudaSuccess)
            return e;
        if ((e = cudaEventRecord(ev_heat, g.gs)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(g.gd, ev_heat, 0)) != cudaSuccess) return e;
        if ((e = g.ks->multi_launch(2, g.desc, n, 0, phase, b->errw, g.wq, g.gd)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ev_diag, g.gd)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}
static cudaError_t batch_groups_join(lbm_batch_s *b, bool captured, cudaStream_t into) {
    cudaError_t e = cudaSuccess;
    for (auto &g : b->groups) {
        cudaEvent_t ev_heat = captured ? g.ev_heat : g.xev_heat, ev_diag = captured ? g.ev_diag : g.xev_diag;
        if ((e = cudaEventRecord(ev_heat, g.gs)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(into, ev_heat, 0)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(into, ev_diag, 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Capture two steps of every run: the batch stream forks to each run's
// stream (runs outside a multi-run group: each queues its own kernels) and
// to the groups' streams (one launch per kernel kind and step for all the
// group's runs), and the branches join back.
static int batch_build_graph(lbm_batch_s *b) {
    int rc = batch_fill_groups(b);
    if (rc != LBM_OK) return rc;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess) rc = LBM_E_CUDA;
    for (size_t i = 0; i < b->runs.size() && rc == LBM_OK; i++) {
        if (b->in_group[i]) continue;
        lbm_run *h = b->runs[i];
        if ((e = cudaStreamWaitEvent(h->stream, b->fork, 0)) != cudaSuccess) { rc = LBM_E_CUDA; break; }
        if ((rc = launch_step(h, false, false, true)) != LBM_OK || (rc = launch_step(h, false, true, true)) != LBM_OK) {
            b->msg = h->msg;
            break;
        }
        if ((e = join_diag(h, true)) != cudaSuccess || (e = cudaEventRecord(b->join[i], h->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(b->stream, b->join[i], 0)) != cudaSuccess) { rc = LBM_E_CUDA; break; }
    }
    if (rc == LBM_OK && !b->groups.empty()) {
        if ((e = batch_groups_step(b, 0, true, true, b->fork)) != cudaSuccess ||
            (e = batch_groups_step(b, 1, false, true, b->fork)) != cudaSuccess ||
            (e = batch_groups_join(b, true, b->stream)) != cudaSuccess)
            rc = LBM_E_CUDA;
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (rc != LBM_OK || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (rc == LBM_E_CUDA) return bfail(b, rc, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return rc != LBM_OK ? rc : bfail(b, LBM_E_CUDA, std::string("batch capture: ") + cudaGetErrorString(e2));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return bfail(b, LBM_E_CUDA, std::string("batch graph: ") + cudaGetErrorString(e)); }
    for (size_t i = 0; i < b->runs.size(); i++) {
        b->versions[i] = b->runs[i]->version;
        b->parities[i] = b->runs[i]->parity;
    }
    return LBM_OK;
}

extern "C" {

int lbm_batch_create(const lbm_handle *runs, int32_t n, lbm_batch *out) {
    if (!out) return bfail(nullptr, LBM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!runs || n < 1) return bfail(nullptr, LBM_E_INVAL, "a batch needs at least one run");
    lbm_batch_s *b = new (std::nothrow) lbm_batch_s();
    if (!b) return bfail(nullptr, LBM_E_NOMEM, "host allocation failed");
    b->device = runs[0] ? runs[0]->device : 0;
    for (int i = 0; i < n; i++) {
        if (!runs[i]) { delete b; return bfail(nullptr, LBM_E_INVAL, "NULL run in batch"); }
        if (runs[i]->device != b->device) { delete b; return bfail(nullptr, LBM_E_INVAL, "runs of a batch must share a device"); }
        for (int j = 0; j < i; j++)
            if (runs[j] == runs[i]) { delete b; return bfail(nullptr, LBM_E_INVAL, "a run appears twice in the batch"); }
        b->runs.push_back(runs[i]);
        b->versions.push_back(-1);
        b->parities.push_back(-1);
        b->in_group.push_back(false);
    }
    // runs whose kernel set has multi-run kernels are stepped per kernel set
    // and flow mode in one launch per kernel kind
    for (int i = 0; i < n; i++) {
        const KernelSet *ks = b->runs[i]->ks;
        if (ks->multi_desc_bytes == 0) continue;
        const int mode = ks->multi_mode(b->runs[i]->p);
        MultiGroup *g = nullptr;
        for (auto &q : b->groups)
            if (q.ks == ks && q.mode == mode) g = &q;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->ks = ks;
            g->mode = mode;
        }
        g->idx.push_back(i);
        b->in_group[i] = true;
    }
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !b->groups.empty()) {
        e = cudaMalloc(&b->errw, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemsetAsync(b->errw, 0, sizeof(unsigned), b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    for (auto &g : b->groups) {
        g.host.resize(g.idx.size() * g.ks->multi_desc_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&g.desc, g.host.size());
        if (e == cudaSuccess) e = cudaMalloc(&g.wq, 2 * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemsetAsync(g.wq, 0, 2 * sizeof(unsigned), b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.gs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.gd, cudaStreamNonBlocking);
        for (cudaEvent_t *ev : {&g.ev_heat, &g.ev_diag, &g.xev_heat, &g.xev_diag})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    for (int i = 0; i < n && e == cudaSuccess; i++) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        b->join.push_back(ev);
    }
    if (e != cudaSuccess) {
        std::string m = std::string("batch set-up: ") + cudaGetErrorString(e);
        batch_free(b);
        delete b;
        return bfail(nullptr, LBM_E_CUDA, m);
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b) {
    if (!b) return LBM_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int64_t n) {
    if (!b) return LBM_E_INVAL;
    if (n < 0) return bfail(b, LBM_E_INVAL, "negative step count");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
    for (auto h : b->runs)
        if (h->timing) return bfail(b, LBM_E_STATE, "a run of the batch has per-kernel timing enabled");
    int rc;
    while (n >= 2) {
        // a captured graph bakes in every run's buffer parity and launch shape
        bool stale = !b->graph;
        for (size_t i = 0; i < b->runs.size(); i++)
            stale = stale || b->versions[i] != b->runs[i]->version || b->parities[i] != b->runs[i]->parity;
        if (stale) {
            if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
            // order the capture after everything already queued on the runs' streams
            for (size_t i = 0; i < b->runs.size(); i++) {
                if ((e = cudaEventRecord(b->join[i], b->runs[i]->stream)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(b->stream, b->join[i], 0)) != cudaSuccess)
                    return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
            }
            if ((rc = batch_build_graph(b)) != LBM_OK) return rc;
        }
        // the graph starts after the runs' queued work and the runs' streams
        // wait for the graph before any later work of their own
        for (size_t i = 0; i < b->runs.size(); i++) {
            if ((e = cudaEventRecord(b->join[i], b->runs[i]->stream)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(b->stream, b->join[i], 0)) != cudaSuccess)
                return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
        }
        if ((e = cudaGraphLaunch(b->graph, b->stream)) != cudaSuccess) return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
        if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess) return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
        for (auto h : b->runs) {
            if ((e = cudaStreamWaitEvent(h->stream, b->fork, 0)) != cudaSuccess) return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
            h->steps += 2;
            h->diag_stale = false;
        }
        n -= 2;
    }
    if (n == 1) {
        // odd remainder: one step; runs outside the groups on their own
        // streams, the groups by one plain launch per kernel kind
        for (size_t i = 0; i < b->runs.size(); i++)
            if (!b->in_group[i] && (rc = lbm_step(b->runs[i], 1)) != LBM_OK) return bfail(b, rc, b->runs[i]->msg);
        if (!b->groups.empty()) {
            if ((rc = batch_fill_groups(b)) != LBM_OK) return rc;
            for (size_t i = 0; i < b->runs.size(); i++) {
                if (!b->in_group[i]) continue;
                if ((e = cudaEventRecord(b->join[i], b->runs[i]->stream)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(b->stream, b->join[i], 0)) != cudaSuccess)
                    return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
            }
            if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess ||
                (e = batch_groups_step(b, 0, true, false, b->fork)) != cudaSuccess ||
                (e = batch_groups_join(b, false, b->stream)) != cudaSuccess ||
                (e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess)
                return bfail(b, LBM_E_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
            for (size_t i = 0; i < b->runs.size(); i++) {
                if (!b->in_group[i]) continue;
                lbm_run *h = b->runs[i];
                if ((e = cudaStreamWaitEvent(h->stream, b->fork, 0)) != cudaSuccess)
                    return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
                h->parity ^= 1;
                h->steps += 1;
                h->diag_stale = false;
            }
        }
    }
    return LBM_OK;
}

int lbm_batch_query(lbm_batch b, int32_t *done) {
    if (!b || !done) return LBM_E_INVAL;
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
    *done = 0;
    std::vector<cudaStream_t> streams{b->stream};
    for (auto h : b->runs) {
        streams.push_back(h->stream);
        streams.push_back(h->dstream);
    }
    for (cudaStream_t st : streams) {
        if (!st) continue;
        e = cudaStreamQuery(st);
        if (e == cudaErrorNotReady) {
            cudaGetLastError();  // not an error: clear it
            return LBM_OK;
        }
        if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
    }
    *done = 1;
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch b) {
    if (!b) return LBM_E_INVAL;
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
    if (b->errw) {
        unsigned w = 0;
        if ((e = cudaMemcpyAsync(&w, b->errw, sizeof(w), cudaMemcpyDeviceToHost, b->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
            return bfail(b, LBM_E_CUDA, cudaGetErrorString(e));
        if (w & ERRW_DESC)
            return bfail(b, LBM_E_STATE, "a multi-run kernel found a descriptor it could not trust and skipped its tile");
    }
    for (auto h : b->runs) {
        int rc = lbm_sync(h);
        if (rc != LBM_OK) return bfail(b, rc, h->msg);
    }
    return LBM_OK;
}

const char *lbm_batch_last_error(lbm_batch b) { return b ? b->msg.c_str() : g_create_error.c_str(); }

int lbm_device_bytes(const lbm_domain_t *domain, const lbm_heater_t *heater, const lbm_opts_t *opts, uint64_t *bytes) {
    if (!domain || !heater || !opts || !bytes) return fail(nullptr, LBM_E_INVAL, "NULL argument");
    const KernelSet *ks = opts->precision == LBM_FP64 ? kernels_fp64()
                          : opts->precision == LBM_FP32 ? kernels_fp32()
                          : opts->precision == LBM_FP16 ? kernels_fp16()
                          : opts->precision == LBM_FP32_DFSRC ? kernels_fp32_dfsrc()
                          : opts->precision == LBM_FP64_FMA ? kernels_fp64_fma() : nullptr;
    if (!ks) return fail(nullptr, LBM_E_INVAL, "opts.precision invalid");
    if (domain->nx < 1 || domain->ny_fluid < 1 || heater->ny_solid < 0) return fail(nullptr, LBM_E_INVAL, "bad sizes");
    const uint64_t nfl = (uint64_t)domain->nx * domain->ny_fluid;
    const bool model_a = heater->ny_solid == 0 && !(domain->flags & LBM_PERIODIC_Y);
    const uint64_t ntl = (uint64_t)domain->nx * (domain->ny_fluid + (model_a ? 1 : heater->ny_solid));
    const uint64_t cap = opts->series_capacity > 0 ? (uint64_t)opts->series_capacity : 4096;
    // populations x2, temperature x2, moments x3 for each step parity,
    // per-column arrays, per-block partials for each parity (at most one
    // block per 32 sites), series ring, small words
    *bytes = 2 * 9 * nfl * ks->f_elem + 2 * ntl * ks->T_elem + 6 * nfl * ks->m_elem + 2 * 8 * (uint64_t)domain->nx +
             2 * 2 * 8 * (nfl / 32 + 1) + cap * SERIES_WIDTH * 8 + 1024 * 8 + 4096 + 2 * ks->multi_desc_bytes;
    return LBM_OK;
}

int lbm_variants(lbm_handle h, int kind, int *count, int *selected) {
    if (!h || (kind != 0 && kind != 1)) return h ? fail(h, LBM_E_INVAL, "kind must be 0 (flow) or 1 (heat)") : LBM_E_INVAL;
    if (count) *count = kind == 0 ? h->ks->n_flow : h->ks->n_heat;
    if (selected) *selected = kind == 0 ? h->fv : h->hv;
    return LBM_OK;
}

const char *lbm_variant_name(lbm_handle h, int kind, int index) {
    if (!h) return "";
    if (kind == 0 && index >= 0 && index < h->ks->n_flow) return h->ks->flow[index].name;
    if (kind == 1 && index >= 0 && index < h->ks->n_heat) return h->ks->heat[index].name;
    return "";
}

int lbm_select_variants(lbm_handle h, int flow, int heat) {
    if (!h) return LBM_E_INVAL;
    if (flow < 0 || flow >= h->ks->n_flow || heat < 0 || heat >= h->ks->n_heat)
        return fail(h, LBM_E_INVAL, "variant index out of range");
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    if (h->graph8) { cudaGraphExecDestroy(h->graph8); h->graph8 = nullptr; }
    h->fv = flow;
    h->hv = heat;
    h->version++;
    h->nblk = h->ks->flow[flow].blocks(h->p);
    return LBM_OK;
}

// Time every flow and heat variant on the current state (outputs go to the
// buffers the next step overwrites; the diagnostics kernel and the step
// counter are not touched), keep the fastest pair.
int lbm_autotune(lbm_handle h, int iters, double *best_ms) {
    if (!h) return LBM_E_INVAL;
    if (iters < 1) return fail(h, LBM_E_INVAL, "iters must be >= 1");
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    StepBuffers b = buffers(h, h->parity);
    cudaEvent_t a, z;
    CK(h, cudaEventCreate(&a));
    CK(h, cudaEventCreate(&z));
    double best[2] = {1e300, 1e300};
    int pick[2] = {h->fv, h->hv};
    const int saved[2] = {h->fv, h->hv};
    for (int kind = 0; kind < 2; kind++) {
        const int nv = kind == 0 ? h->ks->n_flow : h->ks->n_heat;
        for (int v = 0; v < nv; v++) {
            if (kind == 0) h->fv = v; else h->hv = v;
            // each candidate is timed inside a flow + heat pair, as in a step:
            // the flow kernel's traffic leaves L2 in the state the heat
            // kernel meets there (alone, the heat inputs would stay cached)
            cudaError_t e = launch_kernel(h, 0, b);  // warm-up
            if (e == cudaSuccess) e = launch_kernel(h, 1, b);
            if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
            for (int it = 0; it < iters && e == cudaSuccess; it++) {
                e = launch_kernel(h, 0, b);
                if (e == cudaSuccess) e = launch_kernel(h, 1, b);
            }
            if (e == cudaSuccess) e = cudaEventRecord(z, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(z);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
            if (e != cudaSuccess) {
                h->fv = saved[0]; h->hv = saved[1];
                cudaEventDestroy(a); cudaEventDestroy(z);
                return cuda_fail(h, e, "autotune launch");
            }
            if (ms / iters < best[kind]) { best[kind] = ms / iters; pick[kind] = v; }
        }
        if (kind == 0) h->fv = pick[0];  // heat variants read the moments of the chosen flow
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    h->fv = saved[0];
    h->hv = saved[1];
    if (best_ms) { best_ms[0] = best[0]; best_ms[1] = best[1]; }
    int rc = lbm_select_variants(h, pick[0], pick[1]);
    if (rc != LBM_OK) return rc;
    return check_err_word(h);
}

}  // extern "C"
