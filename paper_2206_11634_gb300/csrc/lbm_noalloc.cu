// lbm_flags_noalloc: node classification for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: a host application that owns the
// whole device memory pool and hands out no extra buffers, or a process with
// a strict no-allocation policy once its steady state has started.  This
// entry point classifies nodes for a set of particles with the same kernels
// as lbm_step() (k_bin + k_flags), but keeps their scratch (particle table,
// brick lists and work lists, counters, status) in one file-scope
// __device__ array of fixed size instead of a caller workspace.  The caller
// still passes the particles (host) and the output flag array (device).
//
// The array is reserved by the CUDA runtime when the library's device code
// is loaded on a device and stays reserved on every device that loads the
// library until the process exits.  The first call on each device looks up
// its device address (cudaGetSymbolAddress, with that device current); make
// that first call before any stream capture.
#include <cmath>
#include <cstring>
#include <mutex>

#include "lbm_internal.cuh"

using namespace lbmmb;

namespace {

constexpr int kMaxBricks = 1 << 16;   // e.g. 256 x 256 x 256 nodes (32x4x2-node bricks)
constexpr int kMaxParticles = 256;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffBin = 0;                                                    // bcount + step counters
constexpr size_t kOffList = align256(kOffBin + (size_t)(kMaxBricks + kStepCounters) * 4);  // brick lists
constexpr size_t kOffWork = align256(kOffList + (size_t)kMaxBricks * MAXPB * 4);  // work list ring, counts, stamps
constexpr size_t kWorkBytes = (size_t)kMaxBricks * 4 * 4 + 3 * 4;
constexpr size_t kOffStatus = align256(kOffWork + kWorkBytes);
constexpr size_t kOffParts = align256(kOffStatus + ST_SLOTS * 4);
constexpr size_t kScratchBytes = align256(kOffParts + (size_t)kMaxParticles * sizeof(DevParticle));

// Shared by every call on a device; holds the last call's contents.
__device__ __align__(256) unsigned char g_flags_scratch[kScratchBytes];

std::mutex g_mu;                       // serialises host calls (the host staging table below)
void *g_scratch_addr[kMaxDevices];     // device address of g_flags_scratch, per device
DevParticle g_host_parts[kMaxParticles];  // host staging of the particle table

}  // namespace

extern "C" int lbm_flags_noalloc(const lbm_config *cfg, const lbm_particle *host, int n, void *dev_flags,
                                 void *cuda_stream) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!cfg || !dev_flags || n < 0 || (n > 0 && !host)) return LBM_ERR_BAD_ARG;
    if (cfg->nx < 2 || cfg->ny < 2 || cfg->nz < 2) return LBM_ERR_BAD_ARG;
    if (cfg->lattice != 19 && cfg->lattice != 15) return LBM_ERR_BAD_ARG;
    if (cfg->storage < LBM_STORE_F64 || cfg->storage > LBM_STORE_BF16) return LBM_ERR_BAD_ARG;
    if (!(cfg->c0 > 0.0)) return LBM_ERR_BAD_ARG;
    const int nbx = (cfg->nx + BX - 1) / BX, nby = (cfg->ny + BY - 1) / BY, nbz = (cfg->nz + BZ - 1) / BZ;
    const long long nbricks = (long long)nbx * nby * nbz;
    if (nbricks > kMaxBricks) return LBM_ERR_CAPACITY;
    if (n > kMaxParticles) return LBM_ERR_CAPACITY;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_flags_scratch);
        if (e != cudaSuccess || !p) return LBM_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    char *base = static_cast<char *>(g_scratch_addr[dev]);

    // particle table: shape and pose only (classification needs no mass)
    for (int j = 0; j < n; j++) {
        const lbm_particle &p = host[j];
        if (p.n_cp < 1 || p.n_cp > LBM_MAX_CP) return LBM_ERR_BAD_ARG;
        DevParticle &d = g_host_parts[j];
        std::memset(&d, 0, sizeof(d));
        const double qn = std::sqrt(p.q[0] * p.q[0] + p.q[1] * p.q[1] + p.q[2] * p.q[2] + p.q[3] * p.q[3]);
        if (!(qn > 0.0)) return LBM_ERR_BAD_ARG;
        for (int a = 0; a < 4; a++) d.q[a] = p.q[a] / qn;
        for (int a = 0; a < 3; a++) { d.x[a] = p.x[a]; d.v[a] = p.v[a]; d.w[a] = p.w[a]; }
        d.ncp = p.n_cp;
        double Ks = 0.0, rmax = 0.0;
        for (int k = 0; k < p.n_cp; k++) {
            if (!(p.K[k] >= 0.0)) return LBM_ERR_BAD_ARG;
            for (int a = 0; a < 3; a++) d.cpb[k][a] = p.cp[k][a];
            d.K[k] = p.K[k];
            d.K_f[k] = (float)p.K[k];  // the sweeps' and flag pass's FP32 copy
            Ks += p.K[k];
            rmax = std::fmax(rmax, std::sqrt(p.cp[k][0] * p.cp[k][0] + p.cp[k][1] * p.cp[k][1] + p.cp[k][2] * p.cp[k][2]));
        }
        d.sumK = Ks;
        // bounding radius about x (the flag pass skips nodes outside it)
        d.brad = rmax + std::sqrt(Ks / cfg->c0) + p.Rs;
        d.brad_f = (float)d.brad;
    }

    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(base + kOffParts, g_host_parts, sizeof(DevParticle) * (size_t)n,
                                   cudaMemcpyHostToDevice, st);
    // what must start at zero: brick counts and counters, work lists and
    // stamps, status, and the output (bricks without particles are never
    // written)
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffBin, 0, (size_t)(nbricks + kStepCounters) * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffWork, 0, kWorkBytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffStatus, 0, ST_SLOTS * 4, st);
    const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
    if (e == cudaSuccess) e = cudaMemsetAsync(dev_flags, 0, (size_t)N * 2, st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;

    Params P;
    std::memset(&P, 0, sizeof(P));
    fill_scalar_params(*cfg, P);
    P.np = n;
    P.bcount = reinterpret_cast<int *>(base + kOffBin);
    P.counters = reinterpret_cast<int *>(base + kOffBin + (size_t)nbricks * 4);
    P.blist = reinterpret_cast<int *>(base + kOffList);
    P.step = 0;  // a single classification: only this step's list
    P.wl_list = reinterpret_cast<int *>(base + kOffWork);
    P.stamp = reinterpret_cast<int *>(base + kOffWork + (size_t)kMaxBricks * 3 * 4);
    P.wl_count = reinterpret_cast<int *>(base + kOffWork + (size_t)kMaxBricks * 4 * 4);
    P.status = reinterpret_cast<int *>(base + kOffStatus);
    P.parts = reinterpret_cast<DevParticle *>(base + kOffParts);
    // the output doubles as the "previous" flags: every node of it reads back
    // the value just written (or the cleared 0), so no node is refilled and no
    // population array is touched
    P.flag_new = static_cast<uint16_t *>(dev_flags);
    P.flag_old = static_cast<const uint16_t *>(dev_flags);

    launch_bin(P, st);
    switch (cfg->storage) {
        case LBM_STORE_F64: launch_flags_t<double>(P, st); break;
        case LBM_STORE_F32: launch_flags_t<float>(P, st); break;
        case LBM_STORE_F16: launch_flags_t<__half>(P, st); break;
        default: launch_flags_t<__nv_bfloat16>(P, st); break;
    }
    int status[ST_SLOTS];
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(status, base + kOffStatus, sizeof(status), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if (status[ST_ERR] & ERRB_BRICK_OVERFLOW) return LBM_ERR_CAPACITY;
    // the binning and the flag pass set no other bit; one would mean a fault
    // the result cannot be trusted after
    if (status[ST_ERR] != 0) return LBM_ERR_CUDA;
    return LBM_OK;
}
