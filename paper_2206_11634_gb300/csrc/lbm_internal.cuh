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
constexpr int ROT_ITERS = 2;  // fixed-point sweeps of the implicit rotational half-kick

// Status words in the workspace.
enum StatusSlot { ST_ERR = 0, ST_SLOTS = 16 };
// CNT_NEAR_NEXT, CNT_FLAGS_NEXT: the brick queues of the near sweep and of
// the flag pass (next entry to hand out)
enum StepCounter { CNT_NREFILL = 0, CNT_NLINKS = 1, CNT_LISTED = 2, CNT_NEAR = 3, CNT_NEAR_NEXT = 4, CNT_FLAGS_NEXT = 5 };
constexpr int kStepCounters = 8;  // the slots above, rounded up (zeroed with the brick counts)
enum ErrBits { ERRB_BRICK_OVERFLOW = 1, ERRB_DIVERGED = 2, ERRB_TIMEOUT = 4, ERRB_DEM_CAPACITY = 8,
               ERRB_STATIC_CAPACITY = 16, ERRB_DEM_REACH = 32 };
// contact history flags (Params::pair_on per pair, wall_on per particle and
// wall): in contact at the last evaluation (the tangential spring carries
// over), and warm: the last evaluation of this potential collision (bounding
// spheres overlapping, or the plane within the bounding sphere) found a valid
// Newton solution, x_m or x_cw, which starts the next solve (§2.1.4)
enum ContactFlags { CONTACT_ON = 1, CONTACT_WARM = 2 };
// DEM kernels (lbm_config.dem_mode): the FP64 rigid-body integrator with the
// contact geometry in FP32 (k_dem64_plan + k_dem64_free + k_dem64c, lattices
// below FP64), the compensated-FP32 integrator (k_dem32), and everything in
// FP64 (k_dem, always on FP64 lattices).
enum DemKernel { DEM_FP64_INTEGRATOR = 0, DEM_FP32 = 1, DEM_FP64_ALL = 2 };

// A fluid node with particle links in a fixed geometry, and one of its links
// (geometry of Eq. (27): q, lever arm from the centroid to x_w, u_w).
struct StaticNode {
    int n;          // node index
    uint32_t mask;  // link directions (the unknowns)
    int base;       // its first StaticLink
};
struct StaticLink {
    float q, r[3], uw[3];
    int jf;  // particle index in bits 0-15; bit 31: x_ff is a fluid node in the box
};
// Link nodes per warp of the fixed-geometry link kernel: few, so that a
// warp's lanes evaluate its links in about one round (a link node has a few
// links) and small cases spread over many warps.
constexpr int kStaticNodesPerWarp = 8;

// Lattices stored below FP64 accumulate the per-particle force and torque
// totals in 64-bit fixed point with integer atomics: exact and independent of
// the order of the additions, without FP64 arithmetic.  Resolution 2^-40
// (~9e-13), range +-2^23 (~8e6) per component.
constexpr int kForceFixBits = 40;

// Default launch schedule: one plain-sweep CTA per brick, flags and near
// sweep persistent over 4 CTAs per SM (measured fastest on the settling
// metaball: persistent plain grids that leave CTA slots to the particle
// kernels ran 12-35 % slower per step).
constexpr int kDefaultPlainPerSm = 0;
// Batched lattices: CTAs per case of the flag and near sweeps, bricks per CTA
// of the plain sweep (lbm_batch_tune chooses them by measurement).
constexpr int kDefaultBatchChainCtas = 4;
constexpr int kDefaultBatchPlainChunk = 2;
constexpr int kDefaultChainPerSm = 0;

// FP32 DEM limits: its per-particle tables live in one CTA's shared memory.
constexpr int kDem32MaxParticles = 256;
constexpr int kDem32MaxCp = 2048;     // control points of all particles
constexpr int kDemMaxAdj = 16;        // candidate contact partners per particle and direction
constexpr int kSmallContactGroup = 32;  // contact groups up to this size run one 32-thread CTA each
constexpr int kTinyContactGroup = 4;    // ... up to this size one warp each, kTinyGroupsPerCta per CTA
constexpr int kTinyGroupsPerCta = 8;
// k_dem64_plan's group classes (dem_groups)
enum DemGroupClass { DEM_GROUP_TINY = 0, DEM_GROUP_SMALL = 1, DEM_GROUP_LARGE = 2 };

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

// Lattice entries for a direction known only at run time (out-of-line code):
// every component e+1 in {0,1,2} packed as 2 bits, 6 bits per direction,
// into two 64-bit constants, so no table has to be materialised.
template <int Q>
struct LatPack {
    static constexpr unsigned long long word(int half) {
        unsigned long long v = 0;
        for (int i = 0; i < Q; i++)
            for (int a = 0; a < 3; a++) {
                const int bit = 6 * i + 2 * a;
                if ((bit >= 64) == (half == 1))
                    v |= (unsigned long long)(Lat<Q>::e(i, a) + 1) << (bit - 64 * half);
            }
        return v;
    }
    static constexpr unsigned long long lo = word(0), hi = word(1);
};
template <int Q>
__device__ __forceinline__ int lat_e(int i, int a) {
    const int bit = 6 * i + 2 * a;  // 2-bit fields never straddle the words (6*10 = 60, 60+4 < 64)
    const unsigned long long w = bit < 64 ? LatPack<Q>::lo : LatPack<Q>::hi;
    return (int)((w >> (bit & 63)) & 3ull) - 1;
}
template <int Q>
__device__ __forceinline__ double lat_w(int i) {
    return i == 0 ? Lat<Q>::w(0) : (i <= 6 ? Lat<Q>::w(1) : Lat<Q>::w(Q - 1));
}

// ---------------------------------------------------------------------------
// Storage codecs, in offset form.  The sweep computes with
// g_i = f_i - w_i rho0, the deviation from the rest state (~w_i (rho' +
// 3 e_i.u + ...)): its rounding is then relative to the flow signal rather
// than to w_i rho0, which at low Mach keeps three to four more digits of the
// flow in FP32.  FP64 and FP32 store g; FP16 and BF16 store s = g / w_i
// (= f_i/w_i - rho0, O(|u|) in every direction, so no direction falls into
// the subnormal range).  ld/st read and write g; ldf/stf convert to and from
// f itself (set/get of populations, initialisation); ld_s/st_s carry
// evict-first cache hints (the plain sweep, whose data cannot survive in L2
// until the next step anyway, so the particle kernels beside it keep theirs).
// ---------------------------------------------------------------------------
template <typename S>
struct Codec;

template <>
struct Codec<double> {
    using C = double;
    static constexpr bool kScaled = false;  // collide-space values are the offsets g themselves
    __device__ __forceinline__ static double ldv(const double *p, double, double) { return __ldg(p); }
    __device__ __forceinline__ static double ldv_s(const double *p, double, double) { return __ldcs(p); }
    __device__ __forceinline__ static void stv(double *p, double v, double, double) { *p = v; }
    __device__ __forceinline__ static void stv_s(double *p, double v, double, double) { __stcs(p, v); }
    __device__ __forceinline__ static double g_to_v(double g, double) { return g; }
    __device__ __forceinline__ static double ld(const double *p, double, double) { return __ldg(p); }
    __device__ __forceinline__ static double ld_plain(const double *p, double, double) { return *p; }
    __device__ __forceinline__ static double ld_s(const double *p, double, double) { return __ldcs(p); }
    __device__ __forceinline__ static void st(double *p, double g, double, double) { *p = g; }
    __device__ __forceinline__ static void st_s(double *p, double g, double, double) { __stcs(p, g); }
    __device__ __forceinline__ static double ldf(const double *p, double w, double rho0) { return w * rho0 + *p; }
    __device__ __forceinline__ static void stf(double *p, double f, double w, double rho0) { *p = f - w * rho0; }
};
template <>
struct Codec<float> {
    using C = float;
    static constexpr bool kScaled = false;
    __device__ __forceinline__ static float ldv(const float *p, float, float) { return __ldg(p); }
    __device__ __forceinline__ static float ldv_s(const float *p, float, float) { return __ldcs(p); }
    __device__ __forceinline__ static void stv(float *p, float v, float, float) { *p = v; }
    __device__ __forceinline__ static void stv_s(float *p, float v, float, float) { __stcs(p, v); }
    __device__ __forceinline__ static float g_to_v(float g, float) { return g; }
    __device__ __forceinline__ static float ld(const float *p, float, float) { return __ldg(p); }
    __device__ __forceinline__ static float ld_plain(const float *p, float, float) { return *p; }
    __device__ __forceinline__ static float ld_s(const float *p, float, float) { return __ldcs(p); }
    __device__ __forceinline__ static void st(float *p, float g, float, float) { *p = g; }
    __device__ __forceinline__ static void st_s(float *p, float g, float, float) { __stcs(p, g); }
    __device__ __forceinline__ static float ldf(const float *p, float w, float rho0) { return w * rho0 + *p; }
    __device__ __forceinline__ static void stf(float *p, float f, float w, float rho0) { *p = f - w * rho0; }
};
template <>
struct Codec<__half> {
    using C = float;
    // collide-space values are the stored h = g / w, decoded without the
    // weight (the collision takes the weights into its constants)
    static constexpr bool kScaled = true;
    __device__ __forceinline__ static float ldv(const __half *p, float, float) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static float ldv_s(const __half *p, float, float) { return __half2float(__ldcs(p)); }
    __device__ __forceinline__ static void stv(__half *p, float v, float, float) { *p = __float2half_rn(v); }
    __device__ __forceinline__ static void stv_s(__half *p, float v, float, float) { __stcs(p, __float2half_rn(v)); }
    __device__ __forceinline__ static float g_to_v(float g, float w) { return g * (1.0f / w); }
    __device__ __forceinline__ static float ld(const __half *p, float w, float) { return w * __half2float(__ldg(p)); }
    __device__ __forceinline__ static float ld_plain(const __half *p, float w, float) { return w * __half2float(*p); }
    __device__ __forceinline__ static float ld_s(const __half *p, float w, float) { return w * __half2float(__ldcs(p)); }
    __device__ __forceinline__ static void st(__half *p, float g, float w, float) { *p = __float2half_rn(g * (1.0f / w)); }
    __device__ __forceinline__ static void st_s(__half *p, float g, float w, float) {
        __stcs(p, __float2half_rn(g * (1.0f / w)));
    }
    __device__ __forceinline__ static float ldf(const __half *p, float w, float rho0) {
        return w * (rho0 + __half2float(*p));
    }
    __device__ __forceinline__ static void stf(__half *p, float f, float w, float rho0) {
        *p = __float2half_rn(f * (1.0f / w) - rho0);
    }
};
template <>
struct Codec<__nv_bfloat16> {
    using C = float;
    static constexpr bool kScaled = true;
    __device__ __forceinline__ static float ldv(const __nv_bfloat16 *p, float, float) {
        return __bfloat162float(__ldg(p));
    }
    __device__ __forceinline__ static float ldv_s(const __nv_bfloat16 *p, float, float) {
        return __bfloat162float(__ldcs(p));
    }
    __device__ __forceinline__ static void stv(__nv_bfloat16 *p, float v, float, float) { *p = __float2bfloat16_rn(v); }
    __device__ __forceinline__ static void stv_s(__nv_bfloat16 *p, float v, float, float) {
        __stcs(p, __float2bfloat16_rn(v));
    }
    __device__ __forceinline__ static float g_to_v(float g, float w) { return g * (1.0f / w); }
    __device__ __forceinline__ static float ld(const __nv_bfloat16 *p, float w, float) {
        return w * __bfloat162float(__ldg(p));
    }
    __device__ __forceinline__ static float ld_plain(const __nv_bfloat16 *p, float w, float) {
        return w * __bfloat162float(*p);
    }
    __device__ __forceinline__ static float ld_s(const __nv_bfloat16 *p, float w, float) {
        return w * __bfloat162float(__ldcs(p));
    }
    __device__ __forceinline__ static void st(__nv_bfloat16 *p, float g, float w, float) {
        *p = __float2bfloat16_rn(g * (1.0f / w));
    }
    __device__ __forceinline__ static void st_s(__nv_bfloat16 *p, float g, float w, float) {
        __stcs(p, __float2bfloat16_rn(g * (1.0f / w)));
    }
    __device__ __forceinline__ static float ldf(const __nv_bfloat16 *p, float w, float rho0) {
        return w * (rho0 + __bfloat162float(*p));
    }
    __device__ __forceinline__ static void stf(__nv_bfloat16 *p, float f, float w, float rho0) {
        *p = __float2bfloat16_rn(f * (1.0f / w) - rho0);
    }
};

// ---------------------------------------------------------------------------
// Particle table entry (device, FP64).
// ---------------------------------------------------------------------------
// Internally the body frame is the principal frame of the inertia tensor
// (diagonal I), so Euler's equations need no matrix products; the caller's
// body frame is restored on output through qU.
struct DevParticle {
    double x[3], q[4], v[3], w[3];   // q: principal frame -> world
    double cpb[MAXCP][3];  // control points, principal frame
    double cpw[MAXCP][3];  // world, refreshed after every DEM phase
    double K[MAXCP];
    double mass, density, Rs, sumK;
    double Ip[3];          // principal moments
    double iI[3];          // 1 / Ip (0 for a zero moment)
    double cI[3];          // (I_{l+1} - I_{l+2}) / I_l, Euler's equations
    double qU[4];          // principal frame -> caller's body frame
    double cpu[MAXCP][3];  // control points in the caller's body frame
    double Iu[9];          // inertia in the caller's body frame
    double lo[3], hi[3];   // search box: AABB(cpw) -+ sqrt(sum K / c0)
    double brad;           // bounding radius about x (DEM broad phase)
    double inv_mass;       // 1 / mass
    double buoy;           // 1 - rho0 / rho_s (gravity factor, §3.1)
    int ncp, fixed, pad0, pad1;
    // FP32 DEM (lattices stored below FP64): constants in FP32, and the
    // rigid-body state as compensated pairs, value = [0] + [1] (the FP64
    // fields above are then written from it after every step)
    float cpb_f[MAXCP][3];
    float K_f[MAXCP];
    float iI_f[3], cI_f[3];
    float bg_f[3];         // buoy * g
    float inv_mass_f, Rs_f, brad_f, sumK_f;
    float sx[3][2], sv[3][2], sq[4][2];
    float swb[3][2];       // angular velocity, principal body frame
    // cpw and x split into FP32 pairs (value = [0] + [1]) by the binning, so
    // that brick-relative FP32 positions are formed without FP64 arithmetic
    float cpw_hl[MAXCP][3][2];
    float x_hl[3][2];
    float vw_f[6];         // v and w in FP32, for the sweeps' wall velocities (binning)
    // the particle's step if it touches nothing (FP64 integrator below FP64
    // storage: k_dem64_free, taken by k_dem64_commit when the plan leaves the
    // particle inactive)
    double nx[3], nv[3], nq[4], nw[3];
};

// Everything a kernel needs, passed by value.
struct Params {
    int nx, ny, nz, Q;
    int per[3];
    long long N;
    int nbx, nby, nbz, nbricks;
    int np, n_sub, vibb, missing_force;
    int q_exact;              // link fraction by Newton on Eq. (26) instead of Eq. (27)
    int plain_grid;           // CTAs of k_sweep_plain (0: one per brick)
    int chain_grid;           // CTAs of the persistent k_flags / k_sweep_near (0: default)
    int plain_spec;           // few near bricks expected: the plain sweep pulls before its skip entry arrives
    int idx32;                // Q N < 2^31: population indices fit 32 bits
    int dem_mode;             // enum DemKernel: which DEM kernels run
    int fc_valid;             // Fc/Tc hold the contact load of the current state (0 after set_particles)
    double tau, rho0, c0;
    double F[3], g[3], u0[3];
    // collision constants precomputed on the host (FP64 arithmetic runs at a
    // small fraction of the FP32 rate, so kernels take these ready-made)
    double omega_d, gfac_d;   // 1/tau, 1 - 1/(2 tau)
    double inv_n[3];          // 1/nx, 1/ny, 1/nz
    float omega_f, gfac_f, rho0_f, c0_f;
    float Ff[3];
    double kn, eta_n, kt, eta_t, mu_s, c_tol;
    // FP32 copies for the FP32 DEM
    float kn_f, eta_n_f, kt_f, eta_t_f, mu_s_f, inv_kt_f, c_tol_f, h_f;
    float dim_f[3], inv_n_f[3];
    void *fA;  // read (post-collision, time t)
    void *fB;  // write (post-collision, time t+1)
    uint16_t *flag_new;
    const uint16_t *flag_old;
    // Bricks whose flags need work: k_bin lists the bricks that gain a
    // particle this step (list ring slot step % 3, stamp = step); k_flags
    // visits the union of the lists of this step and the two before (solid
    // nodes of the previous step's flags, and stale ones in the buffer being
    // overwritten, lie only there).
    int step;
    int *wl_list;      // [3][nbricks]
    int *wl_count;     // [3], ring of list lengths (slot step % 3 is written by k_flags)
    int *stamp;        // [nbricks], last step the brick was listed
    // Predicted near set of a step: the bricks within two nodes of the
    // particles' search boxes of the step before (k_bin of that step scatters
    // them).  The plain sweep skips these bricks; the near sweep covers them
    // and the exactly listed ones, so a wrong prediction costs time only.
    int *pred_stamp_cur;   // [nbricks], == step: predicted near this step
    int *pred_stamp_next;  // [nbricks], written for step + 1 (NULL: no prediction)
    int *pred_list_cur;    // [nbricks]
    int *pred_list_next;   // [nbricks]
    int *pred_count;       // [3], ring by step
    // the near set's bricks without particle links, listed by the near sweep
    // for k_sweep_near_plain (this step's parity; NULL: not split)
    int *np_list;          // [nbricks]
    int *np_count;         // [1]
    // Bricks the plain sweep of a step leaves alone, ring of three by step
    // (== step: binned or predicted near).  The plain sweep of step t runs
    // while the chain of t and the binning of t+1 run; the binning of t+1
    // writes the slots of t+1 and t+2 only.
    int *skip;             // [3][nbricks], NULL: none
    int *bcount;       // [nbricks]
    uint8_t *brick_solid;  // [nbricks], the brick held a solid node at its last classification
    int *blist;        // [nbricks][MAXPB]
    double *partial;   // [nbricks][MAXPB][6] (FP64 lattices)
    unsigned long long *Ffix;  // [np][6] fixed-point totals (lattices below FP64), cleared every step
    int force_fixed, pad_ff;
    DevParticle *parts;
    double *Fh, *Th;   // [np][3]
    double *Fc, *Tc;   // [np][3]
    double *pairF;     // [np*np][9]: F_i, T_i, T_j of pair (i<j)
    int *pair_on;      // [np*np]
    double *pair_xi, *pair_xm;   // [np*np][3]
    int *wall_on;      // [np*6]
    double *wall_xi, *wall_xcw;  // [np*6][3]
    float *pair_xi_f, *pair_xm_f;   // [np*np][3], FP32 DEM: spring, warm start (relative to x_i)
    float *wall_xi_f, *wall_xcw_f;  // [np*6][3], FP32 DEM: spring, warm start (relative to x_k)
    void *bin_next;    // batched lattices: the other parity's per-step region (cleared by the binning)
    long long bin_next_bytes;
    int *dem_list;     // [8 + 8 np], k_dem64_plan's split of the particles (dem_free() and below)
    int *status;       // [ST_SLOTS], sticky error bits
    int *counters;     // per-step counters, zeroed with the brick lists
    // fixed-geometry sweep (every particle fixed, lattices below FP64): built
    // once by k_static_build, then every step runs k_static_plain over the
    // nodes with sskip == 0 and k_static_links over the listed link nodes
    uint8_t *sskip;             // [N] 1: solid node or fluid node with a particle link
    struct StaticNode *snodes;  // [snode_cap] the fluid nodes with particle links
    struct StaticLink *slinks;  // [slink_cap] their links, per node in direction order
    int *scount;                // [2] nodes, links written by the build
    unsigned long long *smf;    // [np][6] missing-force-point totals (fixed point, constant)
    int snode_cap, slink_cap;
    int snodes_n;               // link nodes (set by the host after the build)
};

// k_dem64_plan's split of the particles (P.dem_list): [0] inactive count,
// [1] active count, [2 + c] groups of class c (DemGroupClass), [5..7]
// unused; then the inactive particles, the active ones group by group, and
// per group of each class its (start in the active list, size) pair.
constexpr int kDemListHead = 8;
__host__ __device__ __forceinline__ int *dem_free(const Params &P) { return P.dem_list + kDemListHead; }
__host__ __device__ __forceinline__ int *dem_active(const Params &P) { return P.dem_list + kDemListHead + P.np; }
__host__ __device__ __forceinline__ int *dem_groups(const Params &P, int cls) {
    return P.dem_list + kDemListHead + (2 + 2 * cls) * P.np;
}

__host__ __device__ __forceinline__ int dim_of(const Params &P, int a) { return a == 0 ? P.nx : (a == 1 ? P.ny : P.nz); }

// Scalar fields of Params from a configuration (host): lattice size, brick
// grid, physics constants and their FP32 copies.  Pointers are left alone.
inline void fill_scalar_params(const lbm_config &c, Params &P) {
    P.nx = c.nx; P.ny = c.ny; P.nz = c.nz; P.Q = c.lattice;
    for (int a = 0; a < 3; a++) P.per[a] = c.periodic[a] != 0;
    P.N = (long long)c.nx * c.ny * c.nz;
    P.nbx = (c.nx + BX - 1) / BX;
    P.nby = (c.ny + BY - 1) / BY;
    P.nbz = (c.nz + BZ - 1) / BZ;
    P.nbricks = P.nbx * P.nby * P.nbz;
    P.n_sub = c.n_sub; P.vibb = c.vibb; P.missing_force = c.missing_force;
    P.q_exact = c.q_exact;
    P.tau = c.tau; P.rho0 = c.rho0; P.c0 = c.c0;
    for (int a = 0; a < 3; a++) { P.F[a] = c.force[a]; P.g[a] = c.gravity[a]; P.u0[a] = c.u0[a]; }
    P.kn = c.kn; P.eta_n = c.eta_n; P.kt = c.kt; P.eta_t = c.eta_t; P.mu_s = c.mu_s; P.c_tol = c.c_tol;
    P.omega_d = 1.0 / c.tau;
    P.gfac_d = 1.0 - 0.5 / c.tau;
    P.inv_n[0] = 1.0 / c.nx;
    P.inv_n[1] = 1.0 / c.ny;
    P.inv_n[2] = 1.0 / c.nz;
    P.omega_f = (float)P.omega_d;
    P.gfac_f = (float)P.gfac_d;
    P.rho0_f = (float)c.rho0;
    P.c0_f = (float)c.c0;
    for (int a = 0; a < 3; a++) P.Ff[a] = (float)c.force[a];
    P.kn_f = (float)c.kn; P.eta_n_f = (float)c.eta_n; P.kt_f = (float)c.kt; P.eta_t_f = (float)c.eta_t;
    P.mu_s_f = (float)c.mu_s; P.c_tol_f = (float)c.c_tol;
    P.inv_kt_f = c.kt > 0.0 ? (float)(1.0 / c.kt) : 0.0f;
    P.h_f = c.n_sub > 0 ? (float)(1.0 / c.n_sub) : 0.0f;
    P.dim_f[0] = (float)c.nx; P.dim_f[1] = (float)c.ny; P.dim_f[2] = (float)c.nz;
    for (int a = 0; a < 3; a++) P.inv_n_f[a] = (float)P.inv_n[a];
}

// Scalar parameters in the working precision C (float copies are made on the
// host, so no FP64 arithmetic happens per node).
template <typename C> struct Prm;
template <> struct Prm<float> {
    __device__ __forceinline__ static float rho0(const Params &P) { return P.rho0_f; }
    __device__ __forceinline__ static float omega(const Params &P) { return P.omega_f; }
    __device__ __forceinline__ static float gfac(const Params &P) { return P.gfac_f; }
    __device__ __forceinline__ static float F(const Params &P, int a) { return P.Ff[a]; }
};
template <> struct Prm<double> {
    __device__ __forceinline__ static double rho0(const Params &P) { return P.rho0; }
    __device__ __forceinline__ static double omega(const Params &P) { return P.omega_d; }
    __device__ __forceinline__ static double gfac(const Params &P) { return P.gfac_d; }
    __device__ __forceinline__ static double F(const Params &P, int a) { return P.F[a]; }
};

__device__ __forceinline__ double minimg_d(const Params &P, int a, double d) {
    if (P.per[a]) {
        const double L = (double)dim_of(P, a);
        d -= L * floor(d * P.inv_n[a] + 0.5);
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

__device__ __forceinline__ BrickRange brick_range(const Params &P, const DevParticle &p, int a, double grow = 1.0) {
    const int B = a == 0 ? BX : (a == 1 ? BY : BZ);
    const int nb = a == 0 ? P.nbx : (a == 1 ? P.nby : P.nbz);
    const int L = dim_of(P, a);
    int nlo = (int)floor(p.lo[a] - grow - 1e-6);
    int nhi = (int)ceil(p.hi[a] + grow + 1e-6);
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
    float brad2[MAXPB];    // (bounding radius + 1)^2: no node farther from the centroid lies inside
};

// Whether brick-local node (lx,ly,lz) may lie inside listed particle s: within
// its bounding sphere (M >= c0 forces min_k |x - x_k|^2 <= sum K / c0, so a
// solid node lies within max_k |x_k - x_c| + sqrt(sum K / c0) of the
// centroid; the radius carries R_s and one node more, which covers the FP32
// rounding).  A node outside needs no evaluation of M for s.
__device__ __forceinline__ bool in_bound(const Params &P, const SmemParticles &sp, int s, int lx, int ly, int lz) {
    float dx = (float)lx - sp.prel[s][0], dy = (float)ly - sp.prel[s][1], dz = (float)lz - sp.prel[s][2];
    // nearest periodic image, as metaball32 takes it per control point
    const float Lx = (float)P.nx, Ly = (float)P.ny, Lz = (float)P.nz;
    if (P.per[0]) { if (dx > 0.5f * Lx) dx -= Lx; else if (dx < -0.5f * Lx) dx += Lx; }
    if (P.per[1]) { if (dy > 0.5f * Ly) dy -= Ly; else if (dy < -0.5f * Ly) dy += Ly; }
    if (P.per[2]) { if (dz > 0.5f * Lz) dz -= Lz; else if (dz < -0.5f * Lz) dz += Lz; }
    return dx * dx + dy * dy + dz * dz <= sp.brad2[s];
}

// FP32 M of listed particle s at brick-local integer offset (lx,ly,lz) plus a
// fractional offset; `unsure` is set when the FP32 value cannot decide
// M >= c0 (inside the relative band 2^-12 around c0, or a control point
// closer than 1/2, where the rounding of its position dominates).
//
// Error budget: the control point's brick-relative position is rounded once
// to FP32 (from the FP32 pair of its FP64 value, see df_minus_int: within a
// 2^-24 fraction of an ulp of that; |error| <= 2^-24 times its magnitude
// plus 2^-48 of it, < 2^-16 for magnitudes
// below 256), each difference along an axis is exact or rounded once, the
// square sum, the reciprocal and the product add 5 roundings; for distances
// r >= 1/2 each term K/r^2 is off by at most 2^-13 relative, well inside the
// band.
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
        M += sp.K[s][k] * __frcp_rn(r2);  // correctly rounded 1/r2, then one more rounding
    }
    const float c0 = P.c0_f;
    unsure = close || fabsf(M - c0) <= c0 * (1.0f / 4096.0f);
    return M;
}

// c - o rounded once to FP32, for c = hl[0] + hl[1] (an FP64 value split into
// two floats) and an integer-valued o: Knuth's two-sum gives hl[0] - o
// exactly as s + e, and s + (e + hl[1]) rounds once (up to a 2^-24 fraction
// of an ulp from the correctly rounded c - o).  Adds only, so nothing is
// contracted into an FMA.
__device__ __forceinline__ float df_minus_int(const float hl[2], float o) {
    const float s = hl[0] - o;
    const float bb = s - hl[0];
    const float e = (hl[0] - (s - bb)) + (-o - bb);
    return s + (e + hl[1]);
}

// Periodic minimum image of a brick-relative FP32 coordinate about the brick
// centre (h = half the brick's extent along the axis); the shift by the box
// length is exact.
__device__ __forceinline__ float minimg_rel_f(const Params &P, int a, float d, float h) {
    if (P.per[a]) {
        const float L = (float)dim_of(P, a);
        d -= L * rintf((d - h) * P.inv_n_f[a]);
    }
    return d;
}

// The records of the particles whose ids are in sp.id[0..cnt) into shared
// memory, positions brick-relative in FP32 (called by the whole CTA; ends
// with __syncthreads()).
__device__ inline void load_particle_records(const Params &P, SmemParticles &sp, int cnt, int bx0, int by0,
                                             int bz0) {
    const float org[3] = {(float)bx0, (float)by0, (float)bz0};
    const float half[3] = {0.5f * BX, 0.5f * BY, 0.5f * BZ};
    // every control-point slot is read (slots past ncp hold zeros, unused),
    // so no load waits for ncp; FP32 copies only (no FP64 conversions)
    for (int t = threadIdx.x; t < cnt * MAXCP; t += blockDim.x) {
        int s = t / MAXCP, k = t % MAXCP;
        const DevParticle &p = P.parts[sp.id[s]];
        if (k == 0) {
            sp.ncp[s] = p.ncp;
            for (int a = 0; a < 3; a++) {
                sp.prel[s][a] = minimg_rel_f(P, a, df_minus_int(p.x_hl[a], org[a]), half[a]);
                sp.v[s][a] = p.vw_f[a];
                sp.w[s][a] = p.vw_f[3 + a];
            }
            sp.brad2[s] = (p.brad_f + 1.0f) * (p.brad_f + 1.0f);
        }
        for (int a = 0; a < 3; a++)
            sp.crel[s][k][a] = minimg_rel_f(P, a, df_minus_int(p.cpw_hl[k][a], org[a]), half[a]);
        sp.K[s][k] = p.K_f[k];
    }
    __syncthreads();
}

// Load the listed particles of brick b into shared memory (called by the
// whole CTA; ends with __syncthreads()).
__device__ inline void load_smem_particles(const Params &P, SmemParticles &sp, int b, int bx0, int by0, int bz0) {
    const int cnt = min(P.bcount[b], MAXPB);
    if ((int)threadIdx.x < cnt) sp.id[threadIdx.x] = P.blist[b * MAXPB + threadIdx.x];
    if (threadIdx.x == 0) sp.n = cnt;
    __syncthreads();
    load_particle_records(P, sp, cnt, bx0, by0, bz0);
}

__device__ __forceinline__ void brick_coords(const Params &P, int b, int &bx, int &by, int &bz) {
    bx = b % P.nbx;
    by = (b / P.nbx) % P.nby;
    bz = b / (P.nbx * P.nby);
}

// Launchers of the particle-side kernels (k_particles.cu).
void launch_bin(const Params &P, cudaStream_t st);
void launch_force_reduce(const Params &P, cudaStream_t st);
// st2 and the two events serve the FP64-integrator DEM (inactive particles on
// st2, forked from st after the plan and joined back)
void launch_dem(const Params &P, cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_split, cudaEvent_t ev_free);
void launch_dem32(const Params &P, cudaStream_t st);   // k_dem32.cu
void launch_dem64c(const Params &P, cudaStream_t st);  // k_dem32.cu

// ---------------------------------------------------------------------------
// Batched lattices (lbm_batch_*): independent cases stepped together, one
// launch per phase for all cases.  Each case keeps the single-lattice layout
// in its own part of the workspace; its Params live in a device table with
// one row per step parity, and the step numbers come from device counters, so
// a captured CUDA graph replays correctly.
// ---------------------------------------------------------------------------
struct BatchArgs {
    const Params *tab;      // [2][ncases], row = step parity
    int ncases;
    const int *span_off;    // [ncases + 1] prefix sums of the cases' plain spans (ceil(N / BRICK) each)
    const int *item_off;    // [ncases + 1] prefix sums of max(1, particles) (binning CTAs)
    const uint16_t *span_case;  // [total spans] case of each span of the concatenated ranges
    unsigned *ctr;          // [0] step of the particle chain, [1] step of the plain sweep,
                            // [2], [3] CTAs done in the last kernel of each (reset by the last)
    int g_chain;            // CTAs per case of the flag and near sweeps
    int plain_chunk;        // spans per CTA of the plain sweep
    const int *swarp_off;   // [ncases + 1] prefix sums of the cases' link-node warps (>= 1 each;
                            // fixed-geometry sweep)
};

// The case's Params for the current step into shared memory (all threads).
__device__ __forceinline__ void load_case_params(const BatchArgs &B, int c, const volatile unsigned *step_ctr,
                                                 Params &sP) {
    __shared__ unsigned s_step;
    if (threadIdx.x == 0) s_step = *step_ctr;
    __syncthreads();
    const unsigned step = s_step;
    const int *src = reinterpret_cast<const int *>(B.tab + (size_t)(step & 1) * B.ncases + c);
    int *dst = reinterpret_cast<int *>(&sP);
    for (int k = threadIdx.x; k < (int)(sizeof(Params) / 4); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    if (threadIdx.x == 0) sP.step = (int)step;
    __syncthreads();
}

// The last CTA of a kernel to finish advances a step counter (every CTA read
// it at its start, and all have finished once the arrival count is full).
__device__ __forceinline__ void advance_step_when_last(unsigned *arrived, unsigned *step_ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned n = atomicAdd(arrived, 1u);
        if (n == gridDim.x - 1) {
            *arrived = 0;
            __threadfence();
            atomicAdd(step_ctr, 1u);
        }
    }
}

// Case of a global index given the prefix sums off[0..n] (off[n] > i).
__device__ __forceinline__ int case_of(const int *off, int n, int i) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

void launch_bin_batch(const BatchArgs &B, int grid, cudaStream_t st);

// Launchers of the storage-templated kernels (launch_impl.cuh, one
// instantiation per storage type in sweep_<type>.cu).
template <typename S> void launch_init_t(const Params &P, void *f, cudaStream_t st);
template <typename S> void launch_flags_t(const Params &P, cudaStream_t st);
template <typename S> void launch_sweep_plain_t(const Params &P, cudaStream_t st);
template <typename S> void launch_sweep_near_t(const Params &P, cudaStream_t st);
template <typename S> void launch_sweep_near_plain_t(const Params &P, cudaStream_t st);
template <typename S>
void launch_fields_t(const Params &P, const void *f, const uint16_t *flags, double *rho, double *u, uint16_t *fl,
                     cudaStream_t st);
template <typename S> void launch_get_pop_t(const Params &P, const void *f, double *out, cudaStream_t st);
template <typename S> void launch_set_pop_t(const Params &P, void *f, const double *in, cudaStream_t st);
template <typename S> void launch_check_t(const Params &P, const void *f, const uint16_t *flags, cudaStream_t st);
template <typename S> void launch_flags_batch_t(const BatchArgs &B, int Q, cudaStream_t st);
template <typename S> void launch_near_batch_t(const BatchArgs &B, int Q, bool force, cudaStream_t st);
template <typename S> void launch_plain_batch_t(const BatchArgs &B, int Q, bool force, int grid, cudaStream_t st);
template <typename S> void launch_static_build_t(const Params &P, cudaStream_t st);
template <typename S> void launch_static_plain_t(const Params &P, cudaStream_t st);
template <typename S> void launch_static_links_t(const Params &P, cudaStream_t st);
template <typename S> void launch_static_plain_batch_t(const BatchArgs &B, int Q, bool force, int grid, cudaStream_t st);
template <typename S> void launch_static_links_batch_t(const BatchArgs &B, int Q, bool force, int warps,
                                                       cudaStream_t st);

}  // namespace lbmmb
