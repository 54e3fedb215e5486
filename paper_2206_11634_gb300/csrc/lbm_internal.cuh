// Internal definitions shared by the kernels and the host side of the C ABI.
//
// Layout in HBM (all inside the caller's workspace, see lbm_api.cu):
//   populations  two arrays (read A, write B), structure of arrays
//                f[i][z][y][x] in the storage type, swapped every step;
//   node flags   two uint16 arrays (this step's and the previous step's),
//                0 = fluid, j+1 = solid node owned by particle j;
//   bricks       the lattice is tiled by 32x4x2-node bricks (one CTA of the
//                sweep each); per brick the ascending list of particles whose
//                search box meets it, and 6 FP64 force/torque partials per
//                listed particle written by the sweep;
//   particles    one DevParticle per particle (FP64 shape and state).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_metaball.h"

namespace lbmmb {

constexpr int BX = 32, BY = 4, BZ = 2;
constexpr int BRICK = BX * BY * BZ;  // nodes per brick = threads per sweep CTA
constexpr int MAXPB = LBM_MAX_PER_BRICK;
constexpr int MAXCP = LBM_MAX_CP;
constexpr int NWALL = 6;
constexpr int ROT_ITERS = 4;  // fixed-point sweeps of the implicit rotational half-kick

// Status words in the workspace.
enum StatusSlot { ST_ERR = 0, ST_SLOTS = 16 };
enum StepCounter { CNT_NREFILL = 0, CNT_NLINKS = 1 };
enum ErrBits { ERRB_BRICK_OVERFLOW = 1, ERRB_DIVERGED = 2, ERRB_TIMEOUT = 4 };

// ---------------------------------------------------------------------------
// Lattices.  D3Q19 (rest 1/3, axes 1/18, face diagonals 1/36) and the D3Q15
// of §2.2 (2/9, 1/9, 1/72).  Opposite directions are adjacent: i' = i+1 for
// odd i, i-1 for even i > 0.
// ---------------------------------------------------------------------------
template <int Q>
struct Lat;

template <>
struct Lat<19> {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int e(int i, int a) {
        constexpr int E[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return E[i][a];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
};

template <>
struct Lat<15> {
    static constexpr int Q = 15;
    __host__ __device__ static constexpr int e(int i, int a) {
        constexpr int E[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1}, {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                                  {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
        return E[i][a];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
};

// ---------------------------------------------------------------------------
// Storage codecs.  FP64/FP32 store f itself; FP16/BF16 store the offset
// s_i = f_i/w_i - rho0 (a few 1e-3 in magnitude), decoded as w_i (rho0 + s_i).
// ---------------------------------------------------------------------------
template <typename S>
struct Codec;

template <>
struct Codec<double> {
    using C = double;
    __device__ __forceinline__ static double ld(const double *p, double, double) { return __ldg(p); }
    __device__ __forceinline__ static void st(double *p, double f, double, double) { *p = f; }
    __device__ __forceinline__ static double ld_plain(const double *p, double, double) { return *p; }
};
template <>
struct Codec<float> {
    using C = float;
    __device__ __forceinline__ static float ld(const float *p, float, float) { return __ldg(p); }
    __device__ __forceinline__ static void st(float *p, float f, float, float) { *p = f; }
    __device__ __forceinline__ static float ld_plain(const float *p, float, float) { return *p; }
};
template <>
struct Codec<__half> {
    using C = float;
    __device__ __forceinline__ static float ld(const __half *p, float w, float rho0) {
        return w * (rho0 + __half2float(__ldg(p)));
    }
    __device__ __forceinline__ static float ld_plain(const __half *p, float w, float rho0) {
        return w * (rho0 + __half2float(*p));
    }
    __device__ __forceinline__ static void st(__half *p, float f, float w, float rho0) {
        *p = __float2half_rn(f * (1.0f / w) - rho0);
    }
};
template <>
struct Codec<__nv_bfloat16> {
    using C = float;
    __device__ __forceinline__ static float ld(const __nv_bfloat16 *p, float w, float rho0) {
        return w * (rho0 + __bfloat162float(__ldg(p)));
    }
    __device__ __forceinline__ static float ld_plain(const __nv_bfloat16 *p, float w, float rho0) {
        return w * (rho0 + __bfloat162float(*p));
    }
    __device__ __forceinline__ static void st(__nv_bfloat16 *p, float f, float w, float rho0) {
        *p = __float2bfloat16_rn(f * (1.0f / w) - rho0);
    }
};

// ---------------------------------------------------------------------------
// Particle table entry (device, FP64).
// ---------------------------------------------------------------------------
struct DevParticle {
    double x[3], q[4], v[3], w[3];
    double cpb[MAXCP][3];  // body frame
    double cpw[MAXCP][3];  // world, refreshed after every DEM phase
    double K[MAXCP];
    double mass, density, Rs, sumK;
    double I[9], Iinv[9];
    double lo[3], hi[3];   // search box: AABB(cpw) -+ sqrt(sum K / c0)
    double brad;           // bounding radius about x (DEM broad phase)
    int ncp, fixed, pad0, pad1;
};

// Everything a kernel needs, passed by value.
struct Params {
    int nx, ny, nz, Q;
    int per[3];
    long long N;
    int nbx, nby, nbz, nbricks;
    int np, n_sub, vibb, missing_force;
    double tau, rho0, c0;
    double F[3], g[3], u0[3];
    double kn, eta_n, kt, eta_t, mu_s, c_tol;
    void *fA;  // read (post-collision, time t)
    void *fB;  // write (post-collision, time t+1)
    uint16_t *flag_new;
    const uint16_t *flag_old;
    uint8_t *occ_new;  // bricks of flag_new that hold solid nodes
    const uint8_t *occ_old;
    int *bcount;       // [nbricks]
    int *blist;        // [nbricks][MAXPB]
    double *partial;   // [nbricks][MAXPB][6]
    DevParticle *parts;
    double *Fh, *Th;   // [np][3]
    double *Fc, *Tc;   // [np][3]
    double *pairF;     // [np*np][9]: F_i, T_i, T_j of pair (i<j)
    int *pair_on;      // [np*np]
    double *pair_xi, *pair_xm;   // [np*np][3]
    int *wall_on;      // [np*6]
    double *wall_xi, *wall_xcw;  // [np*6][3]
    int *status;       // [ST_SLOTS], sticky error bits
    int *counters;     // per-step counters, zeroed with the brick lists
};

__host__ __device__ __forceinline__ int dim_of(const Params &P, int a) { return a == 0 ? P.nx : (a == 1 ? P.ny : P.nz); }

__device__ __forceinline__ double minimg_d(const Params &P, int a, double d) {
    if (P.per[a]) {
        double L = (double)dim_of(P, a);
        d -= L * floor(d / L + 0.5);
    }
    return d;
}

// Brick index range of a particle's search box grown by one node on each side
// (the fluid neighbours whose links end inside it).  Along a periodic axis
// the range may wrap; `all` is set when it covers the axis.
struct BrickRange {
    int lo, hi;
    bool all;
};

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ BrickRange brick_range(const Params &P, const DevParticle &p, int a) {
    const int B = a == 0 ? BX : (a == 1 ? BY : BZ);
    const int nb = a == 0 ? P.nbx : (a == 1 ? P.nby : P.nbz);
    const int L = dim_of(P, a);
    int nlo = (int)floor(p.lo[a] - 1.0 - 1e-6);
    int nhi = (int)ceil(p.hi[a] + 1.0 + 1e-6);
    BrickRange r;
    r.all = false;
    if (P.per[a]) {
        if (nhi - nlo + 1 >= L) {
            r.lo = 0; r.hi = nb - 1; r.all = true;
            return r;
        }
        // wrap the start into [0, L) and keep the extent; the brick index
        // then runs from lo to hi (hi may exceed nb-1, taken modulo nb)
        int shift = floordiv(nlo, L) * L;
        nlo -= shift;
        nhi -= shift;
        r.lo = nlo / B;
        int hi_wrapped_nodes = nhi;  // may be >= L
        if (hi_wrapped_nodes >= L) {
            // nodes [nlo, L) then [0, nhi - L]
            r.hi = nb + (nhi - L) / B;
        } else {
            r.hi = nhi / B;
        }
        if (r.hi - r.lo + 1 >= nb) { r.lo = 0; r.hi = nb - 1; r.all = true; }
        return r;
    }
    if (nlo < 0) nlo = 0;
    if (nhi > L - 1) nhi = L - 1;
    r.lo = nlo / B;
    r.hi = nhi < nlo ? r.lo - 1 : nhi / B;
    return r;
}

__device__ __forceinline__ bool brick_in_range(const BrickRange &r, int b, int nb) {
    if (r.all) return true;
    if (r.hi < r.lo) return false;
    if (b >= r.lo && b <= r.hi) return true;
    return r.hi >= nb && b + nb <= r.hi;  // the wrapped tail
}

// ---------------------------------------------------------------------------
// Metaball function, Eq. (4).
// ---------------------------------------------------------------------------

// FP64, world coordinates (minimum image on periodic axes).
__device__ __forceinline__ double metaball64(const Params &P, const DevParticle &p, double x, double y, double z) {
    double M = 0.0;
    for (int k = 0; k < p.ncp; k++) {
        double dx = minimg_d(P, 0, x - p.cpw[k][0]);
        double dy = minimg_d(P, 1, y - p.cpw[k][1]);
        double dz = minimg_d(P, 2, z - p.cpw[k][2]);
        double r2 = dx * dx + dy * dy + dz * dz;
        M += p.K[k] / r2;
    }
    return M;
}

// Per-CTA copy of the listed particles in FP32, positions relative to the
// brick origin (so that node offsets are small exact integers).
struct SmemParticles {
    int n;
    int id[MAXPB];
    int ncp[MAXPB];
    float crel[MAXPB][MAXCP][3];
    float K[MAXPB][MAXCP];
    float prel[MAXPB][3];  // centroid relative to the brick origin
    float v[MAXPB][3], w[MAXPB][3];
};

// FP32 M of listed particle s at brick-local integer offset (lx,ly,lz) plus a
// fractional offset; `unsure` is set when the FP32 value cannot decide
// M >= c0 (inside the relative band 2^-12 around c0, or a control point
// closer than 1/2, where the rounding of its position dominates).
//
// Error budget: the control point's brick-relative position is rounded once
// to FP32 (|error| <= 2^-24 times its magnitude, < 2^-16 for magnitudes
// below 256), each difference along an axis is exact or rounded once, the
// square sum and the division add 4 roundings; for distances r >= 1/2 each
// term K/r^2 is off by at most 2^-13 relative, well inside the band.
__device__ __forceinline__ float metaball32(const Params &P, const SmemParticles &sp, int s, float lx, float ly,
                                            float lz, bool &unsure) {
    float M = 0.f;
    bool close = false;
    const float Lx = (float)P.nx, Ly = (float)P.ny, Lz = (float)P.nz;
    for (int k = 0; k < sp.ncp[s]; k++) {
        float dx = lx - sp.crel[s][k][0];
        float dy = ly - sp.crel[s][k][1];
        float dz = lz - sp.crel[s][k][2];
        if (P.per[0]) { if (dx > 0.5f * Lx) dx -= Lx; else if (dx < -0.5f * Lx) dx += Lx; }
        if (P.per[1]) { if (dy > 0.5f * Ly) dy -= Ly; else if (dy < -0.5f * Ly) dy += Ly; }
        if (P.per[2]) { if (dz > 0.5f * Lz) dz -= Lz; else if (dz < -0.5f * Lz) dz += Lz; }
        float r2 = dx * dx + dy * dy + dz * dz;
        close |= r2 < 0.25f;
        M += sp.K[s][k] / r2;
    }
    const float c0 = (float)P.c0;
    unsure = close || fabsf(M - c0) <= c0 * (1.0f / 4096.0f);
    return M;
}

// Load the listed particles of brick b into shared memory (called by the
// whole CTA; ends with __syncthreads()).
__device__ inline void load_smem_particles(const Params &P, SmemParticles &sp, int b, int bx0, int by0, int bz0) {
    const int cnt = min(P.bcount[b], MAXPB);
    if (threadIdx.x == 0) sp.n = cnt;
    for (int t = threadIdx.x; t < cnt * MAXCP; t += blockDim.x) {
        int s = t / MAXCP, k = t % MAXCP;
        const DevParticle &p = P.parts[P.blist[b * MAXPB + s]];
        if (k == 0) {
            sp.id[s] = P.blist[b * MAXPB + s];
            sp.ncp[s] = p.ncp;
            double org[3] = {(double)bx0, (double)by0, (double)bz0};
            double ctr[3] = {bx0 + 0.5 * BX, by0 + 0.5 * BY, bz0 + 0.5 * BZ};
            for (int a = 0; a < 3; a++) {
                sp.prel[s][a] = (float)(ctr[a] - org[a] + minimg_d(P, a, p.x[a] - ctr[a]));
                sp.v[s][a] = (float)p.v[a];
                sp.w[s][a] = (float)p.w[a];
            }
        }
        if (k < p.ncp) {
            double ctr[3] = {bx0 + 0.5 * BX, by0 + 0.5 * BY, bz0 + 0.5 * BZ};
            double org[3] = {(double)bx0, (double)by0, (double)bz0};
            for (int a = 0; a < 3; a++)
                sp.crel[s][k][a] = (float)(ctr[a] - org[a] + minimg_d(P, a, p.cpw[k][a] - ctr[a]));
            sp.K[s][k] = (float)p.K[k];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void brick_coords(const Params &P, int b, int &bx, int &by, int &bz) {
    bx = b % P.nbx;
    by = (b / P.nbx) % P.nby;
    bz = b / (P.nbx * P.nby);
}

// Launchers of the particle-side kernels (k_particles.cu).
void launch_bin(const Params &P, cudaStream_t st);
void launch_force_reduce(const Params &P, cudaStream_t st);
void launch_dem(const Params &P, cudaStream_t st);

// Launchers of the storage-templated kernels (launch_impl.cuh, one
// instantiation per storage type in sweep_<type>.cu).
template <typename S> void launch_init_t(const Params &P, void *f, cudaStream_t st);
template <typename S> void launch_flags_t(const Params &P, cudaStream_t st);
template <typename S> void launch_sweep_t(const Params &P, cudaStream_t st);
template <typename S>
void launch_fields_t(const Params &P, const void *f, const uint16_t *flags, double *rho, double *u, uint16_t *fl,
                     cudaStream_t st);
template <typename S> void launch_get_pop_t(const Params &P, const void *f, double *out, cudaStream_t st);
template <typename S> void launch_set_pop_t(const Params &P, void *f, const double *in, cudaStream_t st);
template <typename S> void launch_check_t(const Params &P, const void *f, const uint16_t *flags, cudaStream_t st);

}  // namespace lbmmb
