// lbm_diagnostics_static: the end-of-step reductions (heater-bottom flux,
// heater-surface flux, vapour fraction, mass) of one state given as float64
// device arrays, computed without allocating any device memory.
//
// Who needs it: code that cannot call cudaMalloc / cudaFree -- for example a
// host application whose device memory is entirely owned by another
// allocator (a framework's caching allocator that has reserved the GPU), or a
// loop that must not risk the implicit device synchronisation those calls
// can cause.  The per-block partial sums live in a file-scope device array
// instead; every GPU that loads this library holds it until the process
// exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_launch.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSitesPerBlock = 4 * kThreads;              // fluid sites reduced by one block
constexpr int kMaxBlocks = 16384;                          // capacity of the static array
constexpr long long kMaxSites = (long long)kMaxBlocks * kSitesPerBlock;  // 16,777,216
constexpr int kMaxDevices = 64;

// [block][4]: mass, vapour count, heater-bottom flux sum, interface flux sum.
// 16384 x 4 x 8 B = 512 KiB per device.
static __device__ __align__(256) double g_partials[kMaxBlocks * 4];

std::mutex g_setup_mutex;
double *g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum(double v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Stage 1: block b reduces fluid sites [b K, (b + 1) K) and columns
// [b K, (b + 1) K) (when < nx) into partials[b][0..3].  Every slot that
// stage 2 reads is written here, so nothing has to start at zero.
// ns >= 3: heater rows 0..ns-1 (model B); ns = 0 without periodic rows:
// model A, T row 0 the wall's Dirichlet row, coupled to the first fluid row
// with the fluid's conductivity on both sides (the per-step diagnostics'
// rule); periodic in y: no wall, no flux.
__global__ void __launch_bounds__(kThreads)
k_static_partials(const double *__restrict__ rho, const double *__restrict__ T, int nx, int nf, int ns, int periodic,
                  double lambda_s, double cv_chi, double threshold, double *__restrict__ partials) {
    __shared__ double sh[4][kThreads / 32];
    const long long sites = (long long)nx * nf;
    const long long base = (long long)blockIdx.x * kSitesPerBlock;
    const bool model_a = ns == 0 && !periodic;
    double m = 0.0, v = 0.0, qb = 0.0, qt = 0.0;
    for (int j = threadIdx.x; j < kSitesPerBlock; j += kThreads) {
        const long long k = base + j;
        if (k < sites) {
            const double r = rho[k];
            m += r;
            v += (r < threshold) ? 1.0 : 0.0;
        }
        if (k < nx && !periodic && (ns >= 3 || model_a)) {
            const int x = (int)k;
            const int nsw = model_a ? 1 : ns;  // T row of the first fluid row
            // face flux through the heater surface or the model-A wall link
            // (harmonic-mean conductance)
            const double l1 = cv_chi * rho[x], l0 = model_a ? cv_chi * rho[x] : lambda_s;
            const double lf = (2.0 * (l0 * l1)) / (l0 + l1);
            const double q = (-lf) * (T[(size_t)nsw * nx + x] - T[(size_t)(nsw - 1) * nx + x]);
            qt += q;
            if (model_a) {
                qb += q;  // no heater: the wall flux stands for both
            } else {
                // Eq. 36 at the heater bottom, rows 0..2
                const double dTdy = ((4.0 * T[nx + x] - T[2 * nx + x]) - 3.0 * T[x]) / 2.0;
                qb += (-lambda_s) * dTdy;
            }
        }
    }
    m = warp_sum(m); v = warp_sum(v); qb = warp_sum(qb); qt = warp_sum(qt);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = m; sh[1][w] = v; sh[2][w] = qb; sh[3][w] = qt; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int i = 0; i < kThreads / 32; i++) s += sh[threadIdx.x][i];
        partials[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// Stage 2 (one block): fixed-order sum of the partials, scaled to the same
// four values as the per-step diagnostics series.
__global__ void __launch_bounds__(kThreads)
k_static_final(const double *__restrict__ partials, int nblk, int nx, int nf, int has_flux_i, double *__restrict__ out) {
    __shared__ double sh[4][kThreads / 32];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += kThreads)
        for (int c = 0; c < 4; c++) a[c] += partials[b * 4 + c];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int c = 0; c < 4; c++) {
        const double s = warp_sum(a[c]);
        if (l == 0) sh[c][w] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < 4; c++)
            for (int i = 0; i < kThreads / 32; i++) s[c] += sh[c][i];
        const double has_flux = has_flux_i ? 1.0 : 0.0;
        out[0] = has_flux * s[2] / (double)nx;        // mean heater-bottom flux
        out[1] = has_flux * s[3] / (double)nx;        // mean heater-surface flux
        out[2] = s[1] / ((double)nx * (double)nf);    // vapour fraction
        out[3] = s[0];                                // mass
    }
}

}  // namespace

extern "C" int lbm_diagnostics_static(const double *rho, const double *T, int32_t nx, int32_t ny_fluid,
                                      int32_t ny_solid, int32_t flags, double lambda_s, double cv_chi,
                                      double rho_L, double rho_V, double *out, void *stream) {
    if (!rho || !T || !out) {
        lbmgb::set_global_error("lbm_diagnostics_static: rho, T and out must be device pointers, not NULL");
        return LBM_E_INVAL;
    }
    if (nx < 1 || ny_fluid < 1 || ny_solid < 0) {
        lbmgb::set_global_error("lbm_diagnostics_static: nx, ny_fluid must be >= 1 and ny_solid >= 0");
        return LBM_E_INVAL;
    }
    const bool periodic = (flags & LBM_PERIODIC_Y) != 0;
    if (ny_solid == 1 || ny_solid == 2 || (periodic && ny_solid != 0)) {
        lbmgb::set_global_error("lbm_diagnostics_static: ny_solid must be >= 3 (heater), or 0 (model A, or a "
                                "domain periodic in y)");
        return LBM_E_INVAL;
    }
    const long long sites = (long long)nx * ny_fluid;
    if (sites > kMaxSites || nx > kMaxSites) {
        lbmgb::set_global_error("lbm_diagnostics_static: " + std::to_string(sites) +
                                " fluid sites exceed the static scratch capacity of " + std::to_string(kMaxSites) +
                                " (16384 blocks of 1024 sites)");
        return LBM_E_INVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        lbmgb::set_global_error(std::string("lbm_diagnostics_static: no usable current device: ") + cudaGetErrorString(e));
        return LBM_E_CUDA;
    }
    double *partials;
    {
        // one-time set-up per device, with that device current: the device
        // address of the static array (its host-side name is only a stand-in)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess || !p) {
                lbmgb::set_global_error(std::string("lbm_diagnostics_static: cudaGetSymbolAddress failed: ") +
                                        cudaGetErrorString(e));
                return LBM_E_CUDA;
            }
            g_partials_addr[dev] = static_cast<double *>(p);
        }
        partials = g_partials_addr[dev];
    }
    const int nblk = (int)((std::max<long long>(sites, nx) + kSitesPerBlock - 1) / kSitesPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    const double threshold = 0.5 * (rho_L + rho_V);
    k_static_partials<<<nblk, kThreads, 0, s>>>(rho, T, nx, ny_fluid, ny_solid, periodic ? 1 : 0, lambda_s, cv_chi,
                                                threshold, partials);
    k_static_final<<<1, kThreads, 0, s>>>(partials, nblk, nx, ny_fluid, periodic ? 0 : 1, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbmgb::set_global_error(std::string("lbm_diagnostics_static: launch failed: ") + cudaGetErrorString(e));
        return LBM_E_CUDA;
    }
    return LBM_OK;
}
