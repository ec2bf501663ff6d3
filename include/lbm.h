/*
 * lbm.h -- C ABI of the GB300 boiling time-step library (liblbm_gb300.so).
 *
 * One run = one 2-D domain of NX periodic columns: NS solid heater rows
 * (row 0 = heater bottom) under NF fluid rows (model B of Fig. 1b), or with
 * NS = 0 the fluid alone on a heated wall (model A of Fig. 1a).  Each time
 * step advances
 *   - the flow: D2Q9 multiple-relaxation-time lattice Boltzmann collision with
 *     the pseudopotential force of a Peng-Robinson fluid and Li's improved
 *     forcing, fused with streaming and halfway bounce-back
 *     (arXiv:1911.10747 Sec. 2.1, Eq. 1-15);
 *   - the heat: the temperature equation of Eq. 24 (advection, conduction
 *     with the solid/fluid conductivity jump, phase-change source) by one RK4
 *     step (Eq. 25-26) with the isotropic differences of Eq. 27-28;
 *   - the diagnostics: heater-bottom flux (Eq. 36/39), heater-top local flux,
 *     vapour fraction and mass.
 *
 * Conventions for every entry point:
 *   - Return value: LBM_OK (0) or an lbm_status error code; the message of
 *     the last error on a handle is returned by lbm_last_error.
 *   - All structs passed in are copied; the caller keeps ownership.
 *   - The handle owns every device allocation it makes (by cudaMalloc, or by
 *     lbm_opts_t.dev_alloc when given); lbm_destroy frees them.  Pointers
 *     passed as "host" buffers must stay valid for the call
 *     only (calls that read back synchronise the handle's stream first).
 *   - Work is queued on the handle's CUDA stream (lbm_opts_t.stream, or a
 *     stream the library creates).  Numerical faults found by the kernels
 *     (negative pseudopotential radicand, non-finite density or temperature)
 *     are latched in a device word and reported as LBM_E_NUMERIC by the next
 *     call that synchronises (lbm_sync and every read-back); a staged-copy
 *     wait that ran out is reported the same way as LBM_E_TIMEOUT.
 *   - Page-locked host arrays given to lbm_set_state are read by the device
 *     directly; pageable ones are staged through a device buffer.
 *   - A handle is not thread-safe; distinct handles are independent.
 *
 * Layouts (row-major, x fastest): populations f[9][NF][NX] in the order of
 * Eq. 2; temperature T[NT][NX] with NT = NS + NF (model A: NT = 1 + NF, row
 * 0 being the heated wall's Dirichlet row); rho, ux, uy [NF][NX].  Values
 * crossing the ABI are always float64, whatever the internal storage
 * precision.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 3

enum lbm_status {
    LBM_OK = 0,
    LBM_E_INVAL = 1,   /* invalid argument or configuration */
    LBM_E_NOMEM = 2,   /* device or host allocation failed */
    LBM_E_CUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error) */
    LBM_E_NUMERIC = 4, /* the kernels latched a numerical fault */
    LBM_E_TIMEOUT = 5, /* a kernel's bounded wait for its staged data ran out (100 ms);
                          the step's results are invalid, the context stays usable */
    LBM_E_STATE = 6    /* call not valid in the handle's current state */
};

enum lbm_top_mode { LBM_TOP_WALL = 0, LBM_TOP_OUTFLOW = 1 };
enum lbm_bc_mode { LBM_BC_SPOTS = 0, LBM_BC_NOISE = 1, LBM_BC_SINE = 2 };
/* LBM_FP32_DFSRC: LBM_FP32 with the phase-change source of Eq. 24
 * (-(T / rho C_V)(dp/dT)_rho div u) evaluated in double-float arithmetic
 * (pairs of FP32 numbers, about 48 significand bits) instead of FP32: the
 * rho-only EOS factors, 1 / (rho C_V) and div u once per step, C1 T +
 * C2 sqrt(T) at every RK stage.  Everything else as LBM_FP32. */
/* LBM_FP64_FMA: the FP64 path compiled with fused multiply-add contraction;
 * faster, no longer bit-identical to a plain evaluation of the formulas
 * (LBM_FP64), and held to a relative 1e-12 per site of it. */
enum lbm_precision { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16 = 2, LBM_FP32_DFSRC = 3, LBM_FP64_FMA = 4 };
enum lbm_flags { LBM_PERIODIC_Y = 1, LBM_ISOTHERMAL = 2, LBM_FROZEN_FLOW = 4 };
enum lbm_field_mask {
    LBM_FIELD_RHO = 1, LBM_FIELD_UX = 2, LBM_FIELD_UY = 4, LBM_FIELD_T = 8, LBM_FIELD_F = 16
};

typedef struct lbm_run *lbm_handle;
typedef struct lbm_batch_s *lbm_batch;

/* Fluid domain and flow model (Sec. 2.1, 3.1). */
typedef struct {
    int32_t nx;          /* periodic columns, >= 1 */
    int32_t ny_fluid;    /* fluid rows NF, >= 2 */
    int32_t liquid_rows; /* initial liquid layer (rows 0..liquid_rows-1 at rho_L) */
    int32_t top_mode;    /* lbm_top_mode: no-slip wall (Sec. 3.1) or zero-gradient outflow */
    int32_t flags;       /* lbm_flags test modes: periodic in y (needs ny_solid = 0),
                            temperature frozen, flow frozen (u = 0) */
    int32_t pad0;
    double g;            /* gravity magnitude, F_g = (rho - rho_mean)(0, -g), Eq. 15 */
    double nu_L, nu_V;   /* kinematic viscosities; tau = 3 nu + 1/2 (Eq. 4), Eq. 5 blend */
    double c_v;          /* specific heat C_V */
    double cv_chi;       /* lambda = rho * cv_chi in the fluid (Sec. 3.1) */
    double s[9];         /* MRT rates s0..s8 (Eq. 3); s7, s8 are replaced by 1/tau(rho) */
    double varpi;        /* weight of the |F_m|^2 term of Eq. 9 */
    double sign_eps;     /* sign of that term in entry 2 of Eq. 9 (-1 in the cited scheme) */
    double init_noise;   /* relative amplitude of the seeded initial density noise */
    double rho_mean;     /* buoyancy reference density; <= 0: the initial fluid mean */
    uint64_t seed;       /* seed of the counter-based draws (initial noise, noisy bottom) */
} lbm_domain_t;

/* Solid heater for conjugate heat transfer (Fig. 1b, Sec. 3.1).  Heater rows
 * conduct only: dT/dt = div(lambda_s grad T) / rho_c_s.
 * ny_solid = 0 on a domain that is not periodic in y selects model A
 * (Fig. 1a, Sec. 4.1): no heater; the bottom temperature T_b(x, n) of
 * lbm_bc_t is held in T row 0, one lattice spacing below the first fluid
 * row and coupled to it with the fluid's conductivity (the mirror of the
 * top row's coupling to T_sat); lambda_s and rho_c_s are ignored and both
 * flux diagnostics report the wall flux -lambda_f (T(row 1) - T_b). */
typedef struct {
    int32_t ny_solid;    /* NS heater rows: >= 3, or 0 (model A; required when periodic in y) */
    int32_t pad0;
    double lambda_s;     /* heater conductivity */
    double rho_c_s;      /* heater volumetric heat capacity rho_S c_S */
} lbm_heater_t;

/* Peng-Robinson equation of state (Eq. 13) and pseudopotential (Eq. 12). */
typedef struct {
    double a, b, R, omega;  /* Tc = 0.0778 a / (0.45724 b R) */
    double G;               /* interaction strength (Eq. 11-12), negative */
    double T_sat_over_Tc;   /* saturation temperature: initial and top temperature */
    double rho_L, rho_V;    /* coexistence densities: initial phases, Eq. 5 blend,
                               vapour-fraction threshold (rho_L + rho_V) / 2 */
} lbm_eos_t;

/* Bottom temperature and heater-surface wettability (Sec. 3.2, 4.1). */
typedef struct {
    int32_t mode;           /* lbm_bc_mode: constant T_b (with spots), T_b (1 + A(2U-1))
                               per column and step, or the sine of Sec. 3.2 */
    int32_t n_spots;        /* nucleate spots, <= 8 */
    double T_b_over_Tc;     /* bottom temperature */
    double noise_amp;       /* A of the noisy bottom */
    double sine_amp_over_Tc, sine_wavelength;  /* T_b + amp Tc sin(2 pi (x - l/4) / l) */
    int64_t sine_t0, sine_t1;                  /* ... applied for t0 < step < t1 */
    int32_t spot_x[8];      /* spot centre columns */
    int32_t spot_half_width;/* a spot covers columns within this periodic distance */
    int32_t pad0;
    double c_w_base;        /* c_w = G_w psi(rho_w) of Eq. 14 along the heater surface */
    double c_w_spot[8];     /* c_w over each spot */
    double c_w_top;         /* c_w of the top wall */
} lbm_bc_t;

/* Library options. */
typedef struct {
    int32_t precision;      /* lbm_precision: FP64 (oracle parity), FP32 shifted
                               populations, FP16 population storage (probe),
                               FP32 with a double-float phase-change source,
                               FP64 with FMA contraction */
    int32_t use_graphs;     /* 1: lbm_step replays a captured two-step CUDA graph */
    void *stream;           /* cudaStream_t to queue work on; NULL: library-owned stream */
    double rho_shift;       /* reference density of the shifted populations; <= 0: rho_mean */
    int32_t series_capacity;/* per-step diagnostics ring length (0: 4096) */
    int32_t device;         /* CUDA device ordinal */
    /* Optional device allocator for the run's buffers (a framework's caching
     * allocator plugs in here).  Both NULL: cudaMalloc / cudaFree.  Both set:
     * dev_alloc(bytes, alloc_ctx) returns device memory of `device`, aligned to
     * 256 bytes, or NULL (then LBM_E_NOMEM); dev_free(ptr, alloc_ctx) releases
     * it.  The run synchronises its streams before it hands memory back, so a
     * stream-ordered allocator may reuse it at once.  One set, one NULL:
     * LBM_E_INVAL.  Called from the thread that calls lbm_create,
     * lbm_set_state (staging growth) and lbm_destroy. */
    void *(*dev_alloc)(size_t bytes, void *alloc_ctx);
    void (*dev_free)(void *ptr, void *alloc_ctx);
    void *alloc_ctx;
    int32_t bounds_check;   /* 1: debugging mode -- lbm_step runs its steps one at a
                               time and after each waits for the GPU and checks the
                               CUDA status and the device error word (numerical
                               faults, wait time-outs), so a fault is reported by
                               the call, at the step that caused it; no graphs.
                               lbm_batch_step does not check step by step */
    int32_t pad1;
} lbm_opts_t;

/* Create a run, allocate its device state and initialise it (Sec. 3.1):
 * liquid below, vapour above, at rest, T = T_sat everywhere.  Fails with
 * LBM_E_INVAL on an inconsistent configuration (message says which field). */
int lbm_create(const lbm_domain_t *domain, const lbm_heater_t *heater, const lbm_eos_t *eos,
               const lbm_bc_t *bc, const lbm_opts_t *opts, lbm_handle *out);

/* Free every resource of the run.  Accepts NULL. */
int lbm_destroy(lbm_handle h);

/* Queue n >= 0 time steps (asynchronous). */
int lbm_step(lbm_handle h, int64_t n);

/* Wait for queued work and report latched numerical faults. */
int lbm_sync(lbm_handle h);

/* Steps completed (including queued ones). */
int64_t lbm_step_count(lbm_handle h);

/* Copy fields out as float64.  For each bit set in mask, in the order RHO,
 * UX, UY, T, F, the next pointer of dst receives the field (rho/ux/uy:
 * NF*NX values, the moments of the last step; T: NT*NX; F: 9*NF*NX,
 * post-stream populations).  dst_is_device: 1 if the pointers are device
 * memory on the run's device, 0 for host memory.  Synchronises. */
int lbm_fields(lbm_handle h, unsigned mask, double *const *dst, int dst_is_device);

/* Replace the state: post-stream populations f (9*NF*NX) and temperature T
 * (NT*NX), float64, host or device; either may be NULL to keep it.
 * Sets the step counter to `step` (the counter keys the noisy bottom) and
 * starts a new trajectory there: lbm_series serves only steps >= `step`,
 * and lbm_wall_heat_flux, lbm_vapour_fraction and lbm_mass return
 * LBM_E_STATE until a step of the new state has run (their values would
 * describe the state before the import). */
int lbm_set_state(lbm_handle h, const double *f, const double *T, int64_t step,
                  int src_is_device);

/* lbm_set_state with float32 arrays (same layout, same semantics): half the
 * bytes to move when the state comes from host memory.  The values are
 * widened to float64 before the conversion to the run's storage, so a
 * float32 array and the same values given as float64 to lbm_set_state give
 * the same state bit for bit. */
int lbm_set_state_f32(lbm_handle h, const float *f, const float *T, int64_t step,
                      int src_is_device);

/* Checkpoint: the state lbm_set_state takes back -- post-stream populations
 * f (9*NF*NX) and temperature T (NT*NX) as float64, and the step counter.
 * Any of f, T, step may be NULL to skip it; dst_is_device as in lbm_fields.
 * Synchronises when f or T is requested.  lbm_set_state(h, f, T, step, ...)
 * on a run of the same configuration continues bit for bit (FP64 path;
 * reduced-precision storage converts through float64 both ways). */
int lbm_get_state(lbm_handle h, double *f, double *T, int64_t *step, int dst_is_device);

/* Heat flux of the last step: mean over x of -lambda_s dT/dy at the heater
 * bottom (Eq. 36 with rows 0-2, Eq. 39 without its scale factor) and, if
 * q_top_local is not NULL, the NX local fluxes -lambda_face dT/dy across the
 * heater/fluid interface.  Synchronises. */
int lbm_wall_heat_flux(lbm_handle h, double *q_bottom_mean, double *q_top_local);

/* Fraction of fluid sites with rho < (rho_L + rho_V) / 2 after the last step. */
int lbm_vapour_fraction(lbm_handle h, double *out);

/* Total fluid mass sum(rho) of the last step (float64 accumulation). */
int lbm_mass(lbm_handle h, double *out);

/* Per-step diagnostics ring: for steps first .. first+count-1 (each still in
 * the ring), 4 values each: q_bottom_mean, q_top_mean, vapour fraction, mass.
 * Synchronises.  LBM_E_INVAL if a step is not in the ring. */
int lbm_series(lbm_handle h, int64_t first, int64_t count, double *out);

/* Per-kernel timing with CUDA events on the run's stream: enable (1) or
 * disable (0).  While enabled, lbm_step launches kernel by kernel (no graph)
 * and accumulates the event time of each kernel. */
int lbm_set_timing(lbm_handle h, int enable);

/* Average milliseconds per launch of the flow kernel, the heat kernel and
 * the diagnostics kernel since timing was enabled, and the launches
 * averaged.  Synchronises. */
int lbm_kernel_times(lbm_handle h, double *avg_ms /* [3] */, int64_t *launches);

/* Kernels queued per time step (for launch accounting). */
int lbm_kernels_per_step(lbm_handle h);

/* Launch-shape variants.  The library compiles several tilings of the flow
 * kernel (kind 0) and the heat kernel (kind 1); every variant computes the
 * same per-site arithmetic.  lbm_variants reports how many there are and
 * which one is in use; lbm_variant_name returns a static name ("" for a bad
 * index); lbm_select_variants picks a pair (drops the captured graph). */
int lbm_variants(lbm_handle h, int kind, int *count, int *selected);
const char *lbm_variant_name(lbm_handle h, int kind, int index);
int lbm_select_variants(lbm_handle h, int flow, int heat);

/* Autotuner: on the run's current state, time `iters` flow + heat launch
 * pairs for every flow variant (with the heat variant in use), keep the
 * fastest, then the same for every heat variant, and keep that pair.  The
 * state, the step counter and the diagnostics are left unchanged (the
 * kernels write only buffers that the next step overwrites).  best_ms
 * (nullable, [2]) receives the winning average milliseconds per flow + heat
 * pair of each search.  Synchronises. */
int lbm_autotune(lbm_handle h, int iters, double *best_ms);

/* Batches of independent runs (the boiling-curve sweep, served requests).
 * A batch groups n >= 1 existing runs of one device (it does not own them;
 * destroy the batch before its runs).  lbm_batch_step advances every run by
 * n steps: pairs of steps are replayed from one captured CUDA graph whose
 * branches, one per run on that run's own stream, run concurrently on the
 * device, so small runs share the GPU instead of queueing behind each other.
 * The graph is re-captured when a run's launch shape changes
 * (lbm_select_variants, lbm_autotune).  Runs with per-kernel timing enabled
 * are rejected (LBM_E_STATE).  Work of a run issued through its own handle
 * before or after a batch step is ordered with it.  lbm_batch_sync waits and
 * reports the first latched fault; messages via lbm_batch_last_error
 * (NULL batch: the last failed lbm_batch_create). */
int lbm_batch_create(const lbm_handle *runs, int32_t n, lbm_batch *out);
int lbm_batch_step(lbm_batch b, int64_t n);
int lbm_batch_sync(lbm_batch b);
/* Non-blocking: *done = 1 when every kernel queued on the batch and on its
 * runs' streams has finished, else 0 (faults are reported by
 * lbm_batch_sync, not here). */
int lbm_batch_query(lbm_batch b, int32_t *done);
int lbm_batch_destroy(lbm_batch b);
const char *lbm_batch_last_error(lbm_batch b);

/* Device memory (bytes, upper estimate) a run of this configuration holds
 * from lbm_create on.  Not included: the float64 staging buffer that the
 * first read-back into host memory (lbm_fields, lbm_get_state) or import
 * from pageable memory (lbm_set_state) allocates, 8 bytes per value moved
 * (at most 9 NF NX + NT NX values), kept until lbm_destroy. */
int lbm_device_bytes(const lbm_domain_t *domain, const lbm_heater_t *heater, const lbm_opts_t *opts,
                     uint64_t *bytes);

/* Request loop with continuous batching (serving).  A server owns the runs
 * it creates.  lbm_server_submit queues a request (the five configuration
 * structs, copied; a step count; keep_fields = 1 to keep rho and T of the
 * final state) and returns its id.  Each lbm_server_tick admits queued
 * requests in arrival order while at most max_active runs are active and
 * their lbm_device_bytes sum stays within hbm_budget_bytes, advances every
 * active run by min(chunk_steps, the smallest remaining step count) through
 * one concurrent batch graph, waits for it, and retires finished runs (their
 * device memory is freed before the next admission).  A run whose kernels
 * latch a numerical fault is retired as failed alone.  lbm_server_status:
 * state 0 queued, 1 running, 2 done, 3 failed, and the submit / start /
 * finish times in seconds since the server was created.
 * lbm_server_result copies the final diagnostics (4 values, as one row of
 * lbm_series) and the kept fields (rho: NF*NX, T: NT*NX values, NT as in
 * lbm_fields).
 * lbm_server_poll is the non-blocking form of a tick: if the chunk in flight
 * has finished it retires finished runs; it admits queued requests (their
 * runs are created and initialised on their own streams while a chunk may
 * still be running); and if no chunk is in flight it launches the next one
 * over every active run, then returns without waiting.  Requests that
 * arrive during a chunk are thus admitted at once and join at the next chunk
 * boundary.  lbm_server_tick first completes a chunk in flight, admits,
 * launches the next chunk and waits for it (one whole chunk per call).
 * *finished counts the requests that reached state 2 or 3 in the call.
 * Not thread-safe. */
typedef struct lbm_server_s *lbm_server;
int lbm_server_create(uint64_t hbm_budget_bytes, int32_t max_active, int32_t chunk_steps, int32_t device,
                      lbm_server *out);
int lbm_server_submit(lbm_server s, const lbm_domain_t *domain, const lbm_heater_t *heater,
                      const lbm_eos_t *eos, const lbm_bc_t *bc, const lbm_opts_t *opts, int64_t steps,
                      int32_t keep_fields, int64_t *id);
int lbm_server_tick(lbm_server s, int32_t *finished);
int lbm_server_poll(lbm_server s, int32_t *finished);
int lbm_server_status(lbm_server s, int64_t id, int32_t *state, double *times /* [3] */);
int lbm_server_result(lbm_server s, int64_t id, double *diag4, double *rho, double *T);
int lbm_server_counts(lbm_server s, int32_t *queued, int32_t *active, uint64_t *bytes_in_use);
int lbm_server_destroy(lbm_server s);
const char *lbm_server_last_error(lbm_server s);

/* Diagnostics of one state without allocating device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc or cudaFree -- a host program whose device memory is owned by
 * another allocator (for instance a framework's caching allocator holding
 * the whole GPU), or a loop that must not risk the implicit device
 * synchronisation of those calls.
 *
 * Inputs (device pointers, float64, row-major as in lbm_fields): rho
 * [ny_fluid][nx] and T [NT][nx], NT as in lbm_fields: ny_solid + ny_fluid
 * with a heater (ny_solid >= 3), 1 + ny_fluid for model A (ny_solid = 0,
 * row 0 the wall's Dirichlet row), ny_fluid for a domain periodic in y
 * (ny_solid = 0 and LBM_PERIODIC_Y in flags; T is then not read).  Output:
 * out, a device pointer to 4 doubles receiving the same values as one row
 * of lbm_series for that configuration: mean heater-bottom flux (Eq. 36
 * with lambda_s), mean heater-surface face flux (harmonic-mean conductance,
 * cv_chi * rho in the fluid), vapour fraction (rho < (rho_L + rho_V) / 2)
 * and mass.  Model A reports its wall flux -cv_chi rho (T(row 1) - T_b) in
 * both flux slots; a domain periodic in y has no wall and reports 0 for
 * both.  flags: the lbm_flags of the run (only LBM_PERIODIC_Y is used).
 * Work is queued on `stream` (a cudaStream_t; NULL = legacy default
 * stream) and the call returns without waiting.
 *
 * Scratch: per-block partial sums go to a file-scope device array of
 * 16384 x 4 doubles (512 KiB) that every GPU loading the library keeps until
 * the process exits; inputs larger than 16,777,216 fluid sites (16384 blocks
 * of 1024 sites) are rejected with LBM_E_INVAL and a message.  No
 * cudaMalloc, cudaFree or allocating library routine is called.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.
 * All calls share the array and leave their partials in it (each call writes
 * every slot it reads, so nothing needs clearing): calls that overlap on the
 * GPU race, so serialise them (one stream, or events).
 * Errors: LBM_E_INVAL (NULL pointer, bad size, ny_solid of 1 or 2, a
 * periodic domain with ny_solid != 0, over capacity), LBM_E_CUDA (no current
 * device, symbol lookup or launch failed); the message is returned by
 * lbm_last_error(NULL). */
int lbm_diagnostics_static(const double *rho, const double *T, int32_t nx, int32_t ny_fluid,
                           int32_t ny_solid, int32_t flags, double lambda_s, double cv_chi, double rho_L,
                           double rho_V, double *out, void *stream);

/* Measured FMA throughput of one GPU, the peak against which the
 * arithmetic-bound kernels report their fraction.  The paper has no
 * counterpart (it reports no timings).  bits = 32 or 64 selects float or
 * double; device = CUDA ordinal (-1: the current device; the caller's current
 * device is restored).  Every thread of SMs x 8 blocks of 256 runs eight
 * independent chains of `iters` fused multiply-adds; one untimed launch, then
 * one launch timed with CUDA events on a private stream; *tflops receives
 * 2 x 8 x iters x threads / time in TFLOP/s.  Synchronous.  Allocates and
 * frees one small device buffer.  Errors: LBM_E_INVAL (bits not 32 / 64,
 * iters outside 1 .. 2^24, tflops NULL), LBM_E_CUDA; message via
 * lbm_last_error(NULL). */
int lbm_peak_fma(int32_t device, int32_t bits, int32_t iters, double *tflops);

/* Message of the last error on h (or of the last failed lbm_create when h is
 * NULL).  Valid until the next call on the same handle. */
const char *lbm_last_error(lbm_handle h);

/* Static name of a status code. */
const char *lbm_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
