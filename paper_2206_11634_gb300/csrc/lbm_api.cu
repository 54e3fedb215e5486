// Host side of the C ABI (include/lbm_metaball.h): configuration checks,
// workspace layout, particle set-up (mass properties), and the per-step
// launch sequence.  No device memory is allocated here: every device array
// lives in the caller's workspace.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_internal.cuh"

using namespace lbmmb;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t storage_bytes(int s) { return s == LBM_STORE_F64 ? 8 : (s == LBM_STORE_F32 ? 4 : 2); }

// A double as a compensated FP32 pair: hi = fl32(v), lo = fl32(v - hi).
void split_pair(double v, float out[2]) {
    out[0] = (float)v;
    out[1] = (float)(v - (double)out[0]);
}

// Byte offsets of every array in the workspace.
struct Layout {
    size_t f[2], flags[2];
    size_t wl_list, wl_count, stamp;
    size_t pred_stamp, pred_list, pred_count, skip, brick_solid, np_list, np_count;
    size_t bin;        // bcount[nbricks] followed by the per-step counters
    size_t bin_bytes;
    size_t bin_alt;    // second per-step region: step t uses bin (t even) or bin_alt (t odd)
    size_t ffix_off;   // offset of the fixed-point force totals within bin
    size_t blist, partial, parts, Fh, Th, Fc, Tc;
    size_t pairF, pair_on, pair_xi, pair_xm, wall_on, wall_xi, wall_xcw;
    size_t pair_xi_f, pair_xm_f, wall_xi_f, wall_xcw_f;
    size_t sskip, snodes, slinks, scount, smf;  // fixed-geometry sweep (below FP64)
    size_t dem_list;   // k_dem64_plan's split of the particles [kDemListHead + 8P]
    int snode_cap, slink_cap;
    size_t status;
    size_t total;
    long long N;
    int nbx, nby, nbz, nbricks;
};

// Steps with the flag pass after the particles were set, before a geometry of
// fixed particles counts as static: the pass visits the bricks listed in the
// last three steps, so three passes leave both flag buffers and the per-brick
// solid marks holding exactly the fixed particles' flags.
constexpr int kStaticFlagSteps = 3;
// Steps per captured graph of a batch (replayed as often as a call needs).
constexpr int kBatchGraphSteps = 16;

const char *check_config(const lbm_config *c) {
    if (!c) return "config is NULL";
    if (c->nx < 2 || c->ny < 2 || c->nz < 2) return "nx, ny, nz must be >= 2";
    if ((long long)c->nx * c->ny * c->nz >= (1LL << 31)) return "lattice must hold fewer than 2^31 nodes";
    if (c->lattice != 19 && c->lattice != 15) return "lattice must be 19 (D3Q19) or 15 (D3Q15)";
    if (c->storage < LBM_STORE_F64 || c->storage > LBM_STORE_BF16) return "storage must be one of enum lbm_storage";
    if (!(c->tau > 0.5) || !std::isfinite(c->tau)) return "tau must be > 1/2";
    if (!(c->rho0 > 0.0)) return "rho0 must be > 0";
    if (!(c->c0 > 0.0)) return "c0 must be > 0";
    if (c->max_particles < 1 || c->max_particles > 65534) return "max_particles must be in 1..65534";
    if (c->n_sub < 0) return "n_sub must be >= 0";
    for (int a = 0; a < 3; a++)
        if (c->periodic[a] != 0 && c->periodic[a] != 1) return "periodic[] must be 0 or 1";
    if (c->mass_spacing < 0.0) return "mass_spacing must be >= 0";
    if (c->dem_mode < LBM_DEM_FP64 || c->dem_mode > LBM_DEM_FP64_ALL) return "dem_mode must be one of enum lbm_dem_mode";
    if (c->q_exact != 0 && c->q_exact != 1) return "q_exact must be 0 or 1";
    return nullptr;
}

void make_layout(const lbm_config *c, Layout *L) {
    const long long N = (long long)c->nx * c->ny * c->nz;
    L->N = N;
    L->nbx = (c->nx + BX - 1) / BX;
    L->nby = (c->ny + BY - 1) / BY;
    L->nbz = (c->nz + BZ - 1) / BZ;
    L->nbricks = L->nbx * L->nby * L->nbz;
    const size_t P = (size_t)c->max_particles, nb = (size_t)L->nbricks;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t fbytes = (size_t)c->lattice * (size_t)N * storage_bytes(c->storage);
    L->f[0] = take(fbytes);
    L->f[1] = take(fbytes);
    L->flags[0] = take((size_t)N * 2);
    L->flags[1] = take((size_t)N * 2);
    L->wl_list = take(3 * nb * 4);
    L->wl_count = take(3 * 4);
    L->stamp = take(nb * 4);
    L->pred_stamp = take(2 * nb * 4);
    L->pred_list = take(2 * nb * 4);
    L->pred_count = take(3 * 4);
    L->skip = take(3 * nb * 4);
    L->brick_solid = take(nb);
    L->np_list = take(2 * nb * 4);  // by step parity
    L->np_count = take(2 * 4);
    // per-step regions, one per step parity, clear when a step starts: brick
    // counts, counters, and (FP32 and below) the fixed-point force/torque
    // totals; the binning of step t clears the region of step t + 1
    L->ffix_off = (nb * 4 + kStepCounters * 4 + 7) / 8 * 8;
    L->bin_bytes = L->ffix_off + P * 6 * 8;
    L->bin = take(L->bin_bytes);
    L->bin_alt = take(L->bin_bytes);  // the other parity's region (odd steps)
    L->blist = take(nb * MAXPB * 4);
    L->partial = take(nb * MAXPB * 6 * 8);
    L->parts = take(P * sizeof(DevParticle));
    L->Fh = take(P * 24);
    L->Th = take(P * 24);
    L->Fc = take(P * 24);
    L->Tc = take(P * 24);
    L->pairF = take(P * P * 9 * 8);
    L->pair_on = take(P * P * 4);
    L->pair_xi = take(P * P * 24);
    L->pair_xm = take(P * P * 24);
    L->wall_on = take(P * NWALL * 4);
    L->wall_xi = take(P * NWALL * 24);
    L->wall_xcw = take(P * NWALL * 24);
    L->pair_xi_f = take(P * P * 12);
    L->pair_xm_f = take(P * P * 12);
    L->wall_xi_f = take(P * NWALL * 12);
    L->wall_xcw_f = take(P * NWALL * 12);
    // fixed-geometry sweep: link nodes lie next to particle surfaces, so room
    // for an eighth of the nodes as link nodes and a quarter as links (at
    // least 4096 and 16384, for small boxes holding large particles) is
    // ample: about 10 bytes per node beside the populations' 76-304; a build
    // that does not fit falls back to the brick sweeps
    const bool fixed_sweep = c->storage != LBM_STORE_F64;
    L->snode_cap = fixed_sweep ? (int)std::max<long long>(4096, N / 8) : 0;
    L->slink_cap = fixed_sweep ? (int)std::max<long long>(16384, N / 4) : 0;
    L->sskip = take(fixed_sweep ? (size_t)N : 0);
    L->snodes = take((size_t)L->snode_cap * sizeof(StaticNode));
    L->slinks = take((size_t)L->slink_cap * sizeof(StaticLink));
    L->scount = take(fixed_sweep ? 8 : 0);
    L->smf = take(fixed_sweep ? P * 48 : 0);
    L->dem_list = take((kDemListHead + 8 * P) * 4);
    L->status = take(ST_SLOTS * 4);
    L->total = o;
}

thread_local char g_init_error[256] = "no error";

}  // namespace

constexpr int kProfKernels = 7;
constexpr int kProfCap = 65536;

// Principal axes of a particle's inertia tensor, kept per particle slot so
// that lbm_set_particles with an unchanged tensor (every call of a run that
// feeds back the state) skips the eigen-decomposition.
struct InertiaCache {
    double key[9];            // the tensor decomposed
    double Ip[3], U[9], qU[4];
    bool valid;
};

struct lbm_handle {
    lbm_config cfg;
    std::vector<InertiaCache> icache;  // [max_particles]
    // Each lbm_step() call forks two library streams from `stream` and joins
    // them back: `hi` (highest priority) runs the latency-bound chain (binning,
    // flags, near sweep, force reduction, DEM), `aux` (lowest priority) the
    // plain sweep, so the chain's small grids are dispatched ahead of the
    // plain sweep's bricks while both run.  The plain sweep of step t starts
    // after the binning of t (it leaves the bricks binned or predicted near)
    // and the near sweep of t-1 (whose input buffer it overwrites); the near
    // sweep of t+1 waits for it (it reads its halo).
    cudaStream_t aux, hi;
    cudaEvent_t ev_fork, ev_bin, ev_plain, ev_near, ev_join;
    // FP64-integrator DEM: the particles that cannot touch anything during a
    // step move on dem2 (high priority), forked from hi after the split
    cudaStream_t dem2;
    cudaEvent_t ev_dsplit, ev_dfree;
    // page-locked host buffer for the particle exchange (set_particles,
    // get_forces): copies from and to it are asynchronous, so a call waits on
    // the stream once; ev_pin marks the end of the last upload from it
    unsigned char *pin;
    size_t pin_bytes;
    cudaEvent_t ev_pin;
    bool pin_busy;
    // kernel timing (lbm_profile): event pairs per kernel, in launch order
    unsigned prof;  // kernels whose launches are bracketed by events (bit k: kernel k)
    std::vector<cudaEvent_t> ev[kProfKernels][2];
    int64_t nrec[kProfKernels];
    int64_t nseen[kProfKernels];  // launches since profiling was enabled (recorded or not)
    int prof_every;               // record every prof_every-th launch of a profiled kernel
    Layout L;
    char *ws;
    cudaStream_t stream;
    int cur;    // populations consistent with flags[fcur] live in f[cur]
    int fcur;
    int np;
    int dem_mode;  // enum DemKernel: the DEM kernels of the current particle set
    int fc_valid;  // the DEM of the last step left the contact load of the current state
    int all_fixed;     // every particle is fixed: the geometry cannot change between set_particles calls
    int static_steps;  // steps run since set_particles with all_fixed (saturating)
    int static_state;  // fixed-geometry sweep: 0 not built, 1 built, -1 did not fit (brick sweeps)
    int snodes_n;      // its link nodes
    int nsm;       // SMs of the device
    int plain_per_sm, chain_per_sm;  // launch schedule (lbm_set_schedule)
    int bin_clean[2];     // the per-step region of that parity is known to be all zero
    int plain_spec;       // the particles' search boxes cover under a tenth of the bricks (set_particles)
    int plain_after_near; // the plain sweep of a step follows its near sweep (else runs beside the chain)
    int plain_spec_mode;  // lbm_set_plain_speculation: -1 auto (plain_spec), 0 off, 1 on
    int64_t steps;
    char err[256];
};

namespace {

int fail(lbm_handle *h, int code, const char *fmt, ...) {
    char *buf = h ? h->err : g_init_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_check(lbm_handle *h, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    return fail(h, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

template <typename T>
T *at(lbm_handle *h, size_t off) {
    return reinterpret_cast<T *>(h->ws + off);
}

// The per-step region of step t (brick counts, counters, fixed-point force
// totals): one per step parity.
static size_t bin_region(const lbm_handle *h, int64_t t) { return (t & 1) ? h->L.bin_alt : h->L.bin; }
// The region holding the results of the last step issued.
static size_t last_bin_region(const lbm_handle *h) { return bin_region(h, h->steps > 0 ? h->steps - 1 : 0); }

Params make_params(lbm_handle *h) {
    const lbm_config &c = h->cfg;
    Params P;
    std::memset(&P, 0, sizeof(P));
    fill_scalar_params(c, P);
    P.np = h->np;
    P.fA = h->ws + h->L.f[h->cur];
    P.fB = h->ws + h->L.f[1 - h->cur];
    P.flag_new = at<uint16_t>(h, h->L.flags[1 - h->fcur]);
    P.flag_old = at<uint16_t>(h, h->L.flags[h->fcur]);
    P.step = (int)h->steps;
    P.wl_list = at<int>(h, h->L.wl_list);
    P.wl_count = at<int>(h, h->L.wl_count);
    P.stamp = at<int>(h, h->L.stamp);
    const int cur = (int)(h->steps & 1);
    P.pred_stamp_cur = at<int>(h, h->L.pred_stamp + (size_t)cur * h->L.nbricks * 4);
    P.pred_stamp_next = at<int>(h, h->L.pred_stamp + (size_t)(1 - cur) * h->L.nbricks * 4);
    P.pred_list_cur = at<int>(h, h->L.pred_list + (size_t)cur * h->L.nbricks * 4);
    P.pred_list_next = at<int>(h, h->L.pred_list + (size_t)(1 - cur) * h->L.nbricks * 4);
    P.pred_count = at<int>(h, h->L.pred_count);
    P.skip = at<int>(h, h->L.skip);
    P.np_list = at<int>(h, h->L.np_list + (size_t)cur * h->L.nbricks * 4);
    P.np_count = at<int>(h, h->L.np_count + (size_t)cur * 4);
    P.brick_solid = at<uint8_t>(h, h->L.brick_solid);
    if (h->L.snode_cap > 0) {
        P.sskip = at<uint8_t>(h, h->L.sskip);
        P.snodes = at<StaticNode>(h, h->L.snodes);
        P.slinks = at<StaticLink>(h, h->L.slinks);
        P.scount = at<int>(h, h->L.scount);
        P.smf = at<unsigned long long>(h, h->L.smf);
    }
    P.snode_cap = h->L.snode_cap;
    P.slink_cap = h->L.slink_cap;
    P.snodes_n = h->snodes_n;
    P.bcount = at<int>(h, bin_region(h, h->steps));
    P.bin_next = h->ws + bin_region(h, h->steps + 1);
    P.bin_next_bytes = (long long)((h->L.bin_bytes + 15) / 16 * 16);
    P.blist = at<int>(h, h->L.blist);
    P.partial = at<double>(h, h->L.partial);
    P.parts = at<DevParticle>(h, h->L.parts);
    P.Fh = at<double>(h, h->L.Fh);
    P.Th = at<double>(h, h->L.Th);
    P.Fc = at<double>(h, h->L.Fc);
    P.Tc = at<double>(h, h->L.Tc);
    P.pairF = at<double>(h, h->L.pairF);
    P.pair_on = at<int>(h, h->L.pair_on);
    P.pair_xi = at<double>(h, h->L.pair_xi);
    P.pair_xm = at<double>(h, h->L.pair_xm);
    P.wall_on = at<int>(h, h->L.wall_on);
    P.wall_xi = at<double>(h, h->L.wall_xi);
    P.wall_xcw = at<double>(h, h->L.wall_xcw);
    P.pair_xi_f = at<float>(h, h->L.pair_xi_f);
    P.pair_xm_f = at<float>(h, h->L.pair_xm_f);
    P.wall_xi_f = at<float>(h, h->L.wall_xi_f);
    P.wall_xcw_f = at<float>(h, h->L.wall_xcw_f);
    P.dem_mode = h->dem_mode;
    P.dem_list = at<int>(h, h->L.dem_list);
    P.fc_valid = h->fc_valid;
    P.plain_grid = h->plain_per_sm > 0 ? h->plain_per_sm * h->nsm : 0;
    P.chain_grid = h->chain_per_sm > 0 ? h->chain_per_sm * h->nsm : 0;
    P.plain_spec = h->plain_spec_mode >= 0 ? h->plain_spec_mode : h->plain_spec;
    P.idx32 = (long long)c.lattice * (long long)c.nx * c.ny * c.nz <= 0x7fffffffLL;
    P.status = at<int>(h, h->L.status);
    P.counters = at<int>(h, bin_region(h, h->steps) + (size_t)h->L.nbricks * 4);
    P.force_fixed = h->cfg.storage != LBM_STORE_F64;
    P.Ffix = at<unsigned long long>(h, bin_region(h, h->steps) + h->L.ffix_off);
    return P;
}

// Parameters of the read-only paths (fields, populations, check): the
// current populations are f[cur], the current flags flags[fcur].
Params current_params(lbm_handle *h) {
    Params P = make_params(h);
    P.fA = h->ws + h->L.f[h->cur];
    P.flag_new = at<uint16_t>(h, h->L.flags[h->fcur]);
    return P;
}

template <template <typename> class F, typename... A>
void by_storage(int storage, A &&...args) {
    switch (storage) {
        case LBM_STORE_F64: F<double>::run(args...); break;
        case LBM_STORE_F32: F<float>::run(args...); break;
        case LBM_STORE_F16: F<__half>::run(args...); break;
        default: F<__nv_bfloat16>::run(args...); break;
    }
}
template <typename S> struct DoInit { static void run(const Params &P, void *f, cudaStream_t st) { launch_init_t<S>(P, f, st); } };
template <typename S> struct DoFlags { static void run(const Params &P, cudaStream_t st) { launch_flags_t<S>(P, st); } };
template <typename S> struct DoPlain { static void run(const Params &P, cudaStream_t st) { launch_sweep_plain_t<S>(P, st); } };
template <typename S> struct DoNear { static void run(const Params &P, cudaStream_t st) { launch_sweep_near_t<S>(P, st); } };
template <typename S> struct DoNearPlain { static void run(const Params &P, cudaStream_t st) { launch_sweep_near_plain_t<S>(P, st); } };
template <typename S> struct DoFields {
    static void run(const Params &P, double *rho, double *u, uint16_t *fl, cudaStream_t st) {
        launch_fields_t<S>(P, P.fA, P.flag_new, rho, u, fl, st);
    }
};
template <typename S> struct DoGetPop { static void run(const Params &P, double *out, cudaStream_t st) { launch_get_pop_t<S>(P, P.fA, out, st); } };
template <typename S> struct DoSetPop { static void run(const Params &P, const double *in, cudaStream_t st) { launch_set_pop_t<S>(P, P.fA, in, st); } };
template <typename S> struct DoCheck { static void run(const Params &P, cudaStream_t st) { launch_check_t<S>(P, P.fA, P.flag_new, st); } };
template <typename S> struct DoStaticBuild { static void run(const Params &P, cudaStream_t st) { launch_static_build_t<S>(P, st); } };
template <typename S> struct DoStaticPlain { static void run(const Params &P, cudaStream_t st) { launch_static_plain_t<S>(P, st); } };
template <typename S> struct DoStaticLinks { static void run(const Params &P, cudaStream_t st) { launch_static_links_t<S>(P, st); } };

// ---------------------------------------------------------------------------
// Host particle set-up.
// ---------------------------------------------------------------------------
void quat_matrix(const double q[4], double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations:
// A = V diag(d) V^T, V's columns the eigenvectors, det V = +1.
void jacobi3(const double A_in[9], double d[3], double V[9]) {
    double A[9];
    for (int i = 0; i < 9; i++) { A[i] = A_in[i]; V[i] = (i % 4 == 0) ? 1.0 : 0.0; }
    for (int sweep = 0; sweep < 50; sweep++) {
        const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-34 * dia || off == 0.0) break;
        for (int p = 0; p < 2; p++)
            for (int q = p + 1; q < 3; q++) {
                const double apq = A[3 * p + q];
                if (apq == 0.0) continue;
                const double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; k++) {  // A <- J^T A J
                    const double akp = A[3 * k + p], akq = A[3 * k + q];
                    A[3 * k + p] = c * akp - s * akq;
                    A[3 * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; k++) {
                    const double apk = A[3 * p + k], aqk = A[3 * q + k];
                    A[3 * p + k] = c * apk - s * aqk;
                    A[3 * q + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; k++) {  // V <- V J
                    const double vkp = V[3 * k + p], vkq = V[3 * k + q];
                    V[3 * k + p] = c * vkp - s * vkq;
                    V[3 * k + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; i++) d[i] = A[4 * i];
    const double det = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                       V[2] * (V[3] * V[7] - V[4] * V[6]);
    if (det < 0.0)
        for (int k = 0; k < 3; k++) V[3 * k + 2] = -V[3 * k + 2];
}

// Unit quaternion (w,x,y,z) of a rotation matrix.
void matrix_quat(const double R[9], double q[4]) {
    const double tr = R[0] + R[4] + R[8];
    if (tr > 0.0) {
        const double s = std::sqrt(tr + 1.0) * 2.0;
        q[0] = 0.25 * s; q[1] = (R[7] - R[5]) / s; q[2] = (R[2] - R[6]) / s; q[3] = (R[3] - R[1]) / s;
    } else if (R[0] > R[4] && R[0] > R[8]) {
        const double s = std::sqrt(1.0 + R[0] - R[4] - R[8]) * 2.0;
        q[0] = (R[7] - R[5]) / s; q[1] = 0.25 * s; q[2] = (R[1] + R[3]) / s; q[3] = (R[2] + R[6]) / s;
    } else if (R[4] > R[8]) {
        const double s = std::sqrt(1.0 + R[4] - R[0] - R[8]) * 2.0;
        q[0] = (R[2] - R[6]) / s; q[1] = (R[1] + R[3]) / s; q[2] = 0.25 * s; q[3] = (R[5] + R[7]) / s;
    } else {
        const double s = std::sqrt(1.0 + R[8] - R[0] - R[4]) * 2.0;
        q[0] = (R[3] - R[1]) / s; q[1] = (R[2] + R[6]) / s; q[2] = (R[5] + R[7]) / s; q[3] = 0.25 * s;
    }
    const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; a++) q[a] /= n;
}

void quat_mul(const double a[4], const double b[4], double r[4]) {
    r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Volume, centroid and inertia of {M >= c0} by counting cell-centre samples
// of a grid of spacing hs (each cell adds its own hs^2/12 per axis to the
// second moments), then the body frame is moved to the centroid.
bool mass_properties(lbm_particle &p, double c0, double hs) {
    double B = 0.0, Ks = 0.0;
    for (int k = 0; k < p.n_cp; k++) {
        for (int a = 0; a < 3; a++) B = std::fmax(B, std::fabs(p.cp[k][a]));
        Ks += p.K[k];
    }
    B += std::sqrt(Ks / c0);
    const int n = (int)std::ceil(B / hs);
    double cnt = 0, s[3] = {0, 0, 0}, S[6] = {0, 0, 0, 0, 0, 0};
    for (int k = -n; k < n; k++)
        for (int j = -n; j < n; j++)
            for (int i = -n; i < n; i++) {
                const double x = (i + 0.5) * hs, y = (j + 0.5) * hs, z = (k + 0.5) * hs;
                double M = 0.0;
                for (int c = 0; c < p.n_cp; c++) {
                    const double dx = x - p.cp[c][0], dy = y - p.cp[c][1], dz = z - p.cp[c][2];
                    M += p.K[c] / (dx * dx + dy * dy + dz * dz);
                }
                if (M >= c0) {
                    cnt += 1.0;
                    s[0] += x; s[1] += y; s[2] += z;
                    S[0] += x * x; S[1] += y * y; S[2] += z * z;
                    S[3] += x * y; S[4] += x * z; S[5] += y * z;
                }
            }
    if (cnt == 0.0) return false;
    const double V = cnt * hs * hs * hs;
    const double c[3] = {s[0] / cnt, s[1] / cnt, s[2] / cnt};
    const double cell = hs * hs / 12.0;
    const double Cxx = S[0] / cnt - c[0] * c[0] + cell, Cyy = S[1] / cnt - c[1] * c[1] + cell,
                 Czz = S[2] / cnt - c[2] * c[2] + cell;
    const double Cxy = S[3] / cnt - c[0] * c[1], Cxz = S[4] / cnt - c[0] * c[2], Cyz = S[5] / cnt - c[1] * c[2];
    const double m = p.density * V;
    p.mass = m;
    p.inertia[0] = m * (Cyy + Czz); p.inertia[1] = -m * Cxy;        p.inertia[2] = -m * Cxz;
    p.inertia[3] = -m * Cxy;        p.inertia[4] = m * (Cxx + Czz); p.inertia[5] = -m * Cyz;
    p.inertia[6] = -m * Cxz;        p.inertia[7] = -m * Cyz;        p.inertia[8] = m * (Cxx + Cyy);
    double R[9];
    quat_matrix(p.q, R);
    for (int k = 0; k < p.n_cp; k++)
        for (int a = 0; a < 3; a++) p.cp[k][a] -= c[a];
    for (int a = 0; a < 3; a++) p.x[a] += R[3 * a] * c[0] + R[3 * a + 1] * c[1] + R[3 * a + 2] * c[2];
    return true;
}

}  // namespace

extern "C" {

int lbm_workspace_size(const lbm_config *cfg, size_t *bytes) {
    if (const char *m = check_config(cfg)) return fail(nullptr, LBM_ERR_BAD_ARG, "%s", m);
    if (!bytes) return fail(nullptr, LBM_ERR_BAD_ARG, "bytes is NULL");
    Layout L;
    make_layout(cfg, &L);
    *bytes = L.total;
    return LBM_OK;
}

}  // extern "C"

namespace {
// A handle on its workspace; own_streams = false for the cases of a batch
// (the batch owns the streams, events and step sequence).
int init_handle(const lbm_config *cfg, void *dev_ws, size_t ws_bytes, void *cuda_stream, bool own_streams,
                lbm_handle **out) {
    if (!out) return fail(nullptr, LBM_ERR_BAD_ARG, "out is NULL");
    *out = nullptr;
    if (const char *m = check_config(cfg)) return fail(nullptr, LBM_ERR_BAD_ARG, "%s", m);
    Layout L;
    make_layout(cfg, &L);
    if (!dev_ws) return fail(nullptr, LBM_ERR_BAD_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(dev_ws) % kAlign) return fail(nullptr, LBM_ERR_BAD_ARG, "workspace not 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(nullptr, LBM_ERR_WS_TOO_SMALL, "workspace of %zu bytes, %zu needed", ws_bytes, L.total);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, dev_ws) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(nullptr, LBM_ERR_BAD_ARG, "workspace is not device memory");
    }
    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "out of host memory");
    h->cfg = *cfg;
    if (h->cfg.mass_spacing == 0.0) h->cfg.mass_spacing = 0.5;
    h->L = L;
    h->ws = static_cast<char *>(dev_ws);
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->cur = 0;
    h->fcur = 0;
    h->np = 0;
    h->steps = 0;
    h->all_fixed = 1;
    h->static_steps = 0;
    h->static_state = 0;
    h->snodes_n = 0;
    h->prof = 0u;
    for (int k = 0; k < kProfKernels; k++) h->nrec[k] = h->nseen[k] = 0;
    h->prof_every = 1;
    std::snprintf(h->err, sizeof(h->err), "no error");
    // everything but the populations starts at zero: all nodes fluid, no
    // bricks occupied, no contacts, no errors
    const size_t zero_from = L.flags[0];
    h->aux = h->hi = h->dem2 = nullptr;
    h->ev_fork = h->ev_bin = h->ev_plain = h->ev_near = h->ev_join = nullptr;
    h->ev_dsplit = h->ev_dfree = nullptr;
    h->dem_mode = DEM_FP64_ALL;
    h->pin = nullptr;
    h->ev_pin = nullptr;
    h->pin_busy = false;
    // status slots, fixed-point totals [P][6], FP64 totals [P][6], particle records
    h->pin_bytes = ST_SLOTS * 4 + (size_t)cfg->max_particles * (48 + 48 + sizeof(DevParticle));
    {
        int dev = 0;
        h->nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (h->nsm <= 0) h->nsm = 1;
        h->plain_per_sm = kDefaultPlainPerSm;
        h->chain_per_sm = kDefaultChainPerSm;
        h->plain_spec = 1;
        h->plain_after_near = 1;
        h->plain_spec_mode = -1;
        h->bin_clean[0] = h->bin_clean[1] = 1;  // the workspace is cleared below
    }
    int rc = LBM_OK;
    if (own_streams) {
        int prio_low = 0, prio_high = 0;
        rc = cuda_check(h, cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high), "cudaDeviceGetStreamPriorityRange");
        if (rc == LBM_OK)
            rc = cuda_check(h, cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, prio_low), "cudaStreamCreateWithPriority");
        if (rc == LBM_OK)
            rc = cuda_check(h, cudaStreamCreateWithPriority(&h->hi, cudaStreamNonBlocking, prio_high), "cudaStreamCreateWithPriority");
        if (rc == LBM_OK) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "cudaEventCreate");
        if (rc == LBM_OK) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
        if (rc == LBM_OK) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_bin, cudaEventDisableTiming), "cudaEventCreate");
        if (rc == LBM_OK) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_plain, cudaEventDisableTiming), "cudaEventCreate");
        if (rc == LBM_OK) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_near, cudaEventDisableTiming), "cudaEventCreate");
        if (rc == LBM_OK)
            rc = cuda_check(h, cudaStreamCreateWithPriority(&h->dem2, cudaStreamNonBlocking, prio_high), "cudaStreamCreateWithPriority");
        if (rc == LBM_OK) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_dsplit, cudaEventDisableTiming), "cudaEventCreate");
        if (rc == LBM_OK) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_dfree, cudaEventDisableTiming), "cudaEventCreate");
    }
    if (rc == LBM_OK) rc = cuda_check(h, cudaHostAlloc((void **)&h->pin, h->pin_bytes, cudaHostAllocDefault), "cudaHostAlloc");
    if (rc == LBM_OK) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_pin, cudaEventDisableTiming), "cudaEventCreate");
    if (rc == LBM_OK) rc = cuda_check(h, cudaMemsetAsync(h->ws + zero_from, 0, L.total - zero_from, h->stream), "cudaMemsetAsync");
    if (rc == LBM_OK)  // no brick is predicted near (or skipped) before the first step
        rc = cuda_check(h, cudaMemsetAsync(h->ws + L.pred_stamp, 0xFF, 2 * (size_t)L.nbricks * 4, h->stream), "cudaMemsetAsync");
    if (rc == LBM_OK)
        rc = cuda_check(h, cudaMemsetAsync(h->ws + L.skip, 0xFF, 3 * (size_t)L.nbricks * 4, h->stream), "cudaMemsetAsync");
    if (rc == LBM_OK) {
        Params P = make_params(h);
        by_storage<DoInit>(h->cfg.storage, P, (void *)(h->ws + L.f[0]), h->stream);
        by_storage<DoInit>(h->cfg.storage, P, (void *)(h->ws + L.f[1]), h->stream);
        rc = cuda_check(h, cudaGetLastError(), "init kernel launch");
    }
    if (rc == LBM_OK) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) {
        std::snprintf(g_init_error, sizeof(g_init_error), "%s", h->err);
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        if (h->ev_bin) cudaEventDestroy(h->ev_bin);
        if (h->ev_plain) cudaEventDestroy(h->ev_plain);
        if (h->ev_near) cudaEventDestroy(h->ev_near);
        if (h->ev_join) cudaEventDestroy(h->ev_join);
        if (h->ev_pin) cudaEventDestroy(h->ev_pin);
        if (h->ev_dsplit) cudaEventDestroy(h->ev_dsplit);
        if (h->ev_dfree) cudaEventDestroy(h->ev_dfree);
        if (h->pin) cudaFreeHost(h->pin);
        if (h->aux) cudaStreamDestroy(h->aux);
        if (h->hi) cudaStreamDestroy(h->hi);
        if (h->dem2) cudaStreamDestroy(h->dem2);
        delete h;
        return rc;
    }
    *out = h;
    return LBM_OK;
}
}  // namespace

extern "C" {

int lbm_init(const lbm_config *cfg, void *dev_ws, size_t ws_bytes, void *cuda_stream, lbm_handle **out) {
    return init_handle(cfg, dev_ws, ws_bytes, cuda_stream, true, out);
}

// Zero a few word-aligned device ranges in one launch (the resets of
// lbm_set_particles), instead of one memset node each.
struct ClearRanges {
    static constexpr int kMax = 8;
    unsigned *p[kMax];
    long long words[kMax];
    int n;
};
__global__ void k_clear_ranges(ClearRanges R) {
    for (int r = 0; r < R.n; r++)
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < R.words[r];
             k += (long long)gridDim.x * blockDim.x)
            R.p[r][k] = 0u;
}

// Whether the plain sweep may issue its pulls before it knows if the near
// sweep takes the brick: worth it when the near set is a small share of the
// bricks (its pulls are then wasted on few bricks), not when many particles
// fill the box.  Estimated from each particle's bounding sphere (control
// points, the radius where M falls to c0, Rs) plus two nodes of margin,
// counted in whole bricks.
static int plain_speculates(const lbm_config &c, const lbm_particle *host, int n) {
    const int nbx = (c.nx + BX - 1) / BX, nby = (c.ny + BY - 1) / BY, nbz = (c.nz + BZ - 1) / BZ;
    const double nbricks = (double)nbx * nby * nbz;
    double near = 0.0;
    for (int j = 0; j < n; j++) {
        const lbm_particle &p = host[j];
        double Ks = 0.0, rmax = 0.0;
        for (int k = 0; k < p.n_cp; k++) {
            Ks += p.K[k];
            rmax = std::fmax(rmax, std::sqrt(p.cp[k][0] * p.cp[k][0] + p.cp[k][1] * p.cp[k][1] + p.cp[k][2] * p.cp[k][2]));
        }
        const double d = 2.0 * (rmax + std::sqrt(Ks / c.c0) + p.Rs + 2.0);
        near += std::fmin(std::ceil(d / BX) + 1, nbx) * std::fmin(std::ceil(d / BY) + 1, nby) *
                std::fmin(std::ceil(d / BZ) + 1, nbz);
    }
    return near < 0.1 * nbricks ? 1 : 0;
}

int lbm_set_particles(lbm_handle *h, const lbm_particle *host, int n) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (n < 0 || (n > 0 && !host)) return fail(h, LBM_ERR_BAD_ARG, "bad particle array");
    if (n > h->cfg.max_particles)
        return fail(h, LBM_ERR_CAPACITY, "%d particles, capacity %d", n, h->cfg.max_particles);
    // the table is built in place in the page-locked buffer, once its
    // previous upload is done, and goes up from there
    if (n > 0 && h->pin_busy) {
        const int rc0 = cuda_check(h, cudaEventSynchronize(h->ev_pin), "cudaEventSynchronize");
        if (rc0 != LBM_OK) return rc0;
        h->pin_busy = false;
    }
    DevParticle *dev = reinterpret_cast<DevParticle *>(h->pin + ST_SLOTS * 4 + (size_t)h->cfg.max_particles * 96);
    int nc_total = 0;
    for (int j = 0; j < n; j++) {
        lbm_particle p = host[j];
        if (p.n_cp < 1 || p.n_cp > LBM_MAX_CP) return fail(h, LBM_ERR_BAD_ARG, "particle %d: n_cp out of range", j);
        const double qn = std::sqrt(p.q[0] * p.q[0] + p.q[1] * p.q[1] + p.q[2] * p.q[2] + p.q[3] * p.q[3]);
        if (!(qn > 0.0)) return fail(h, LBM_ERR_BAD_ARG, "particle %d: zero quaternion", j);
        for (int a = 0; a < 4; a++) p.q[a] /= qn;
        for (int k = 0; k < p.n_cp; k++)
            if (!(p.K[k] >= 0.0)) return fail(h, LBM_ERR_BAD_ARG, "particle %d: negative weight", j);
        if (!(p.density > 0.0)) return fail(h, LBM_ERR_BAD_ARG, "particle %d: density must be > 0", j);
        if (p.mass <= 0.0 && !mass_properties(p, h->cfg.c0, h->cfg.mass_spacing))
            return fail(h, LBM_ERR_BAD_ARG, "particle %d: empty shape", j);
        DevParticle &d = dev[j];
        std::memset(&d, 0, sizeof(d));
        for (int a = 0; a < 3; a++) { d.x[a] = p.x[a]; d.v[a] = p.v[a]; d.w[a] = p.w[a]; }
        for (int a = 0; a < 4; a++) d.q[a] = p.q[a];
        d.ncp = p.n_cp;
        d.fixed = p.fixed != 0;
        double Ks = 0.0, rmax = 0.0;
        for (int k = 0; k < p.n_cp; k++) {
            d.K[k] = p.K[k];
            Ks += p.K[k];
            rmax = std::fmax(rmax, std::sqrt(p.cp[k][0] * p.cp[k][0] + p.cp[k][1] * p.cp[k][1] + p.cp[k][2] * p.cp[k][2]));
        }
        d.sumK = Ks;
        d.brad = rmax + std::sqrt(Ks / h->cfg.c0) + p.Rs;
        d.mass = p.mass;
        d.density = p.density;
        d.Rs = p.Rs;
        // principal frame: I_user = U diag(Ip) U^T, q_principal = q_user (x) q(U)
        double Ip[3], U[9], qU[4];
        if (h->icache.size() != (size_t)h->cfg.max_particles) h->icache.assign((size_t)h->cfg.max_particles, InertiaCache{});
        InertiaCache &ic = h->icache[(size_t)j];
        if (ic.valid && std::memcmp(ic.key, p.inertia, sizeof(ic.key)) == 0) {
            std::memcpy(Ip, ic.Ip, sizeof(Ip));
            std::memcpy(U, ic.U, sizeof(U));
            std::memcpy(qU, ic.qU, sizeof(qU));
        } else {
            jacobi3(p.inertia, Ip, U);
            matrix_quat(U, qU);
            std::memcpy(ic.key, p.inertia, sizeof(ic.key));
            std::memcpy(ic.Ip, Ip, sizeof(Ip));
            std::memcpy(ic.U, U, sizeof(U));
            std::memcpy(ic.qU, qU, sizeof(qU));
            ic.valid = true;
        }
        for (int a = 0; a < 9; a++) d.Iu[a] = p.inertia[a];
        for (int a = 0; a < 4; a++) d.qU[a] = qU[a];
        quat_mul(p.q, qU, d.q);
        for (int l = 0; l < 3; l++) {
            d.Ip[l] = Ip[l];
            d.iI[l] = Ip[l] != 0.0 ? 1.0 / Ip[l] : 0.0;
            d.cI[l] = Ip[l] != 0.0 ? (Ip[(l + 1) % 3] - Ip[(l + 2) % 3]) / Ip[l] : 0.0;
        }
        if (!d.fixed && !(Ip[0] > 0.0 && Ip[1] > 0.0 && Ip[2] > 0.0))
            return fail(h, LBM_ERR_BAD_ARG, "particle %d: inertia not positive definite", j);
        for (int k = 0; k < p.n_cp; k++)
            for (int a = 0; a < 3; a++) {
                d.cpu[k][a] = p.cp[k][a];
                d.cpb[k][a] = U[a] * p.cp[k][0] + U[3 + a] * p.cp[k][1] + U[6 + a] * p.cp[k][2];  // U^T cp
            }
        // world control points and search box (refreshed by every step)
        double R[9];
        quat_matrix(d.q, R);
        for (int a = 0; a < 3; a++) { d.lo[a] = 1e300; d.hi[a] = -1e300; }
        for (int k = 0; k < d.ncp; k++)
            for (int a = 0; a < 3; a++) {
                d.cpw[k][a] = d.x[a] + R[3 * a] * d.cpb[k][0] + R[3 * a + 1] * d.cpb[k][1] + R[3 * a + 2] * d.cpb[k][2];
                d.lo[a] = std::fmin(d.lo[a], d.cpw[k][a]);
                d.hi[a] = std::fmax(d.hi[a], d.cpw[k][a]);
            }
        for (int a = 0; a < 3; a++) { d.lo[a] -= std::sqrt(Ks / h->cfg.c0); d.hi[a] += std::sqrt(Ks / h->cfg.c0); }
        // divisions done here once (FP64 division is slow on the device)
        d.inv_mass = p.mass > 0.0 ? 1.0 / p.mass : 0.0;
        d.buoy = 1.0 - h->cfg.rho0 / p.density;
        // FP32 DEM: constants and the compensated state
        for (int k = 0; k < d.ncp; k++) {
            for (int a = 0; a < 3; a++) d.cpb_f[k][a] = (float)d.cpb[k][a];
            d.K_f[k] = (float)d.K[k];
        }
        for (int l = 0; l < 3; l++) {
            d.iI_f[l] = (float)d.iI[l];
            d.cI_f[l] = (float)d.cI[l];
            d.bg_f[l] = (float)(d.buoy * h->cfg.gravity[l]);
        }
        d.inv_mass_f = (float)d.inv_mass;
        d.Rs_f = (float)d.Rs;
        d.brad_f = (float)d.brad;
        d.sumK_f = (float)d.sumK;
        double wb[3];
        for (int a = 0; a < 3; a++) wb[a] = R[a] * d.w[0] + R[3 + a] * d.w[1] + R[6 + a] * d.w[2];  // R^T w
        for (int a = 0; a < 3; a++) {
            split_pair(d.x[a], d.sx[a]);
            split_pair(d.v[a], d.sv[a]);
            split_pair(wb[a], d.swb[a]);
        }
        for (int a = 0; a < 4; a++) split_pair(d.q[a], d.sq[a]);
        nc_total += d.ncp;
    }
    // the FP32-geometry DEM kernels keep their per-particle tables in shared
    // memory; beyond those limits, and on FP64 lattices, the FP64 k_dem runs
    const bool fits = n <= kDem32MaxParticles && nc_total <= kDem32MaxCp;
    if (h->cfg.storage == LBM_STORE_F64 || h->cfg.dem_mode == LBM_DEM_FP64_ALL || !fits) h->dem_mode = DEM_FP64_ALL;
    else if (h->cfg.dem_mode == LBM_DEM_FP32_COMPENSATED) h->dem_mode = DEM_FP32;
    else h->dem_mode = DEM_FP64_INTEGRATOR;
    int rc = LBM_OK;
    if (n > 0) {
        // asynchronous upload from the page-locked buffer: the call returns
        // without waiting for the stream
        rc = cuda_check(h, cudaMemcpyAsync(h->ws + h->L.parts, dev, sizeof(DevParticle) * (size_t)n,
                                           cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync(particles)");
        if (rc == LBM_OK) rc = cuda_check(h, cudaEventRecord(h->ev_pin, h->stream), "cudaEventRecord");
        h->pin_busy = rc == LBM_OK;
    }
    // contact pairs and walls, hydrodynamic totals, both per-step regions
    const size_t P = (size_t)h->cfg.max_particles;
    if (rc == LBM_OK) {
        ClearRanges R;
        const size_t off[6] = {h->L.pair_on, h->L.wall_on, h->L.Fh, h->L.Th, h->L.bin, h->L.bin_alt};
        const size_t bytes[6] = {P * P * 4, P * NWALL * 4, P * 24, P * 24, h->L.bin_bytes, h->L.bin_bytes};
        R.n = 6;
        long long most = 0;
        for (int r = 0; r < 6; r++) {
            R.p[r] = reinterpret_cast<unsigned *>(h->ws + off[r]);
            R.words[r] = (long long)(bytes[r] / 4);
            most = std::max(most, R.words[r]);
        }
        const int grid = (int)std::min<long long>((most + 255) / 256, 1024);
        k_clear_ranges<<<grid > 0 ? grid : 1, 256, 0, h->stream>>>(R);
        rc = cuda_check(h, cudaGetLastError(), "clear launch");
    }
    if (rc == LBM_OK) h->bin_clean[0] = h->bin_clean[1] = 1;
    if (rc == LBM_OK) h->np = n;
    h->fc_valid = 0;
    h->all_fixed = 1;
    for (int j = 0; j < n; j++)
        if (!host[j].fixed) h->all_fixed = 0;
    h->plain_spec = plain_speculates(h->cfg, host, n);
    // with few near bricks the flag pass and near sweep are short and run
    // faster alone, and the plain sweep then overlaps the DEM and the next
    // binning and flag pass; with many, the near sweep is long and the plain
    // sweep beside it
    h->plain_after_near = h->plain_spec;
    h->static_steps = 0;
    h->static_state = 0;
    h->snodes_n = 0;
    return rc;
}

// Event pair around one kernel launch when profiling.
struct ProfScope {
    lbm_handle *h;
    int k;
    bool on;
    cudaStream_t st;
    ProfScope(lbm_handle *h_, int k_, bool launched, cudaStream_t st_)
        : h(h_), k(k_), on(((h_->prof >> k_) & 1u) && launched && h_->nseen[k_]++ % h_->prof_every == 0 &&
                           h_->nrec[k_] < kProfCap),
          st(st_) {
        if (!on) return;
        const size_t i = (size_t)h->nrec[k];
        if (h->ev[k][0].size() <= i) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) { on = false; return; }
            h->ev[k][0].push_back(a);
            h->ev[k][1].push_back(b);
        }
        cudaEventRecord(h->ev[k][0][i], st);
    }
    ~ProfScope() {
        if (!on) return;
        cudaEventRecord(h->ev[k][1][(size_t)h->nrec[k]], st);
        h->nrec[k]++;
    }
};

int lbm_step(lbm_handle *h, int nsteps) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (nsteps < 0) return fail(h, LBM_ERR_BAD_ARG, "nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    // fork: both library streams start after everything issued so far
    cudaError_t e = cudaEventRecord(h->ev_fork, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->hi, h->ev_fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, h->ev_fork, 0);
    if (e != cudaSuccess) return cuda_check(h, e, "stream fork");
    cudaStream_t hs = h->hi;
    for (int t = 0; t < nsteps; t++) {
        Params P = make_params(h);
        // with every particle fixed the flags cannot change: once both flag
        // buffers and the per-brick solid marks hold them (the pass visits the
        // bricks listed in the last three steps), it is left out, and below
        // FP64 the fixed-geometry sweep takes over
        const bool geom_static = h->all_fixed && h->static_steps >= kStaticFlagSteps;
        const bool fixed_sweep = geom_static && h->L.snode_cap > 0 && h->static_state >= 0;
        // fresh brick lists and step counters: the region of this step was
        // cleared by the previous step's binning, else here
        const int rp = (int)(h->steps & 1);
        const size_t region = bin_region(h, h->steps);
        if (!h->bin_clean[rp]) {
            e = cudaMemsetAsync(h->ws + region, 0, h->L.bin_bytes, hs);
            if (e != cudaSuccess) return cuda_check(h, e, "cudaMemsetAsync(bricks)");
        }
        h->bin_clean[rp] = 0;
        if (fixed_sweep && h->static_state == 0) {
            // record the fixed geometry once, from this step's brick lists
            { ProfScope s(h, 0, true, hs); launch_bin(P, hs); }
            h->bin_clean[rp ^ 1] = 1;
            e = cudaMemsetAsync(h->ws + h->L.sskip, 0, (size_t)h->L.N, hs);
            if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->L.scount, 0, 8, hs);
            if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->L.smf, 0, (size_t)h->cfg.max_particles * 48, hs);
            if (e != cudaSuccess) return cuda_check(h, e, "cudaMemsetAsync(static)");
            by_storage<DoStaticBuild>(h->cfg.storage, P, hs);
            int cnt[2] = {0, 0}, st[ST_SLOTS];
            e = cudaMemcpyAsync(cnt, h->ws + h->L.scount, 8, cudaMemcpyDeviceToHost, hs);
            if (e == cudaSuccess) e = cudaMemcpyAsync(st, h->ws + h->L.status, ST_SLOTS * 4, cudaMemcpyDeviceToHost, hs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(hs);
            if (e != cudaSuccess) return cuda_check(h, e, "fixed-geometry build");
            if (st[ST_ERR] & ERRB_STATIC_CAPACITY) {
                // did not fit: clear the mark and keep the brick sweeps
                st[ST_ERR] &= ~ERRB_STATIC_CAPACITY;
                e = cudaMemcpyAsync(h->ws + h->L.status, st, ST_SLOTS * 4, cudaMemcpyHostToDevice, hs);
                if (e == cudaSuccess) e = cudaStreamSynchronize(hs);
                if (e != cudaSuccess) return cuda_check(h, e, "fixed-geometry build");
                h->static_state = -1;
                std::snprintf(h->err, sizeof(h->err),
                              "fixed-geometry sweep: %d link nodes and %d links exceed %d and %d; brick sweeps kept",
                              cnt[0], cnt[1], h->L.snode_cap, h->L.slink_cap);
            } else {
                h->static_state = 1;
                h->snodes_n = cnt[0];
                P = make_params(h);
            }
            // the lists this build read are cleared again for the step
            e = cudaMemsetAsync(h->ws + region, 0, h->L.bin_bytes, hs);
            if (e != cudaSuccess) return cuda_check(h, e, "cudaMemsetAsync(bricks)");
        }
        if (fixed_sweep && h->static_state == 1) {
            // the link nodes after the previous step's plain nodes (they read
            // them, and overwrite the array that sweep read), the plain nodes
            // after the previous step's link nodes, concurrently otherwise
            if (t > 0) e = cudaStreamWaitEvent(hs, h->ev_plain, 0);
            if (e == cudaSuccess && t > 0) e = cudaStreamWaitEvent(h->aux, h->ev_near, 0);
            if (e != cudaSuccess) return cuda_check(h, e, "stream wait");
            { ProfScope s(h, 3, true, hs); by_storage<DoStaticLinks>(h->cfg.storage, P, hs); }
            { ProfScope s(h, 2, true, h->aux); by_storage<DoStaticPlain>(h->cfg.storage, P, h->aux); }
            e = cudaEventRecord(h->ev_plain, h->aux);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_near, hs);
            if (e != cudaSuccess) return cuda_check(h, e, "event record");
        } else {
            { ProfScope s(h, 0, true, hs); launch_bin(P, hs); }
            h->bin_clean[rp ^ 1] = 1;
            e = cudaEventRecord(h->ev_bin, hs);
            if (e != cudaSuccess) return cuda_check(h, e, "event record");
            { ProfScope s(h, 1, !geom_static, hs); if (!geom_static) by_storage<DoFlags>(h->cfg.storage, P, hs); }
            // the near sweep reads the halo the previous plain sweep wrote (this
            // wait is issued before ev_plain is recorded again below; the plain
            // sweep of the call before was joined into `stream` before the fork,
            // so every event waited on is recorded within this call, as stream
            // capture requires)
            if (t > 0) e = cudaStreamWaitEvent(hs, h->ev_plain, 0);
            if (e != cudaSuccess) return cuda_check(h, e, "stream wait");
            if (h->plain_after_near) {
                // few near bricks: the near sweep alone, then the plain bricks
                // on the low-priority stream beside the DEM and the next
                // step's binning and flag pass (whose refill touches only
                // nodes next to this step's solid ones, all in near bricks)
                { ProfScope s(h, 3, true, hs); by_storage<DoNear>(h->cfg.storage, P, hs); }
                e = cudaEventRecord(h->ev_near, hs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, h->ev_near, 0);
                if (e != cudaSuccess) return cuda_check(h, e, "stream fork");
                { ProfScope s(h, 2, true, h->aux); by_storage<DoPlain>(h->cfg.storage, P, h->aux); }
                { ProfScope s(h, 6, true, h->aux); by_storage<DoNearPlain>(h->cfg.storage, P, h->aux); }
                e = cudaEventRecord(h->ev_plain, h->aux);
                if (e != cudaSuccess) return cuda_check(h, e, "event record");
            } else {
                // plain bricks on the low-priority stream, concurrent with the chain
                e = cudaStreamWaitEvent(h->aux, h->ev_bin, 0);
                if (e != cudaSuccess) return cuda_check(h, e, "stream wait");
                { ProfScope s(h, 2, true, h->aux); by_storage<DoPlain>(h->cfg.storage, P, h->aux); }
                { ProfScope s(h, 3, true, hs); by_storage<DoNear>(h->cfg.storage, P, hs); }
                e = cudaEventRecord(h->ev_near, hs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, h->ev_near, 0);
                if (e != cudaSuccess) return cuda_check(h, e, "stream fork");
                // then the near set's bricks without particle links, as the
                // near sweep listed them
                { ProfScope s(h, 6, true, h->aux); by_storage<DoNearPlain>(h->cfg.storage, P, h->aux); }
                e = cudaEventRecord(h->ev_plain, h->aux);
                if (e != cudaSuccess) return cuda_check(h, e, "event record");
            }
        }
        if (!P.force_fixed) { ProfScope s(h, 4, P.np > 0, hs); launch_force_reduce(P, hs); }
        { ProfScope s(h, 5, P.np > 0 && P.n_sub > 0, hs); launch_dem(P, hs, h->dem2, h->ev_dsplit, h->ev_dfree); }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(h, e, "kernel launch");
        h->cur ^= 1;
        h->fcur ^= 1;
        h->steps++;
        if (P.np > 0 && P.n_sub > 0) h->fc_valid = 1;
        if (h->all_fixed && h->static_steps < kStaticFlagSteps) h->static_steps++;
    }
    // join: the caller's stream continues after the last DEM and the last
    // plain sweep
    e = cudaEventRecord(h->ev_join, hs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_plain, 0);
    if (e != cudaSuccess) return cuda_check(h, e, "stream join");
    return LBM_OK;
}

int lbm_kernels_per_step(const lbm_handle *h) {
    if (!h) return 0;
    // binning (every step), flags (left out once the geometry is static),
    // the plain sweep, the near sweep and the near set's bricks without
    // particle links; force reduction (FP64 lattices with particles); DEM
    // (particles, n_sub > 0); once the fixed-geometry sweep runs: its link and
    // plain kernels
    const bool geom_static = h->all_fixed && h->static_steps >= kStaticFlagSteps;
    // the FP64-integrator DEM is six kernels (every particle's free step, the
    // split, tiny, small and large contact groups, the free steps taken)
    const int dem = h->np > 0 && h->cfg.n_sub > 0 ? (h->dem_mode == DEM_FP64_INTEGRATOR ? 6 : 1) : 0;
    if (geom_static && h->static_state == 1) return 2 + dem;
    const int flags = geom_static ? 0 : 1;
    if (h->np == 0) return 4 + flags;
    return 4 + flags + (h->cfg.storage == LBM_STORE_F64 ? 1 : 0) + dem;
}

static int read_status(lbm_handle *h, int *st) {
    int rc = cuda_check(h, cudaMemcpyAsync(st, h->ws + h->L.status, ST_SLOTS * 4, cudaMemcpyDeviceToHost, h->stream),
                        "cudaMemcpyAsync(status)");
    if (rc == LBM_OK) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

static int status_code(lbm_handle *h, const int *st) {
    if (st[ST_ERR] & ERRB_BRICK_OVERFLOW)
        return fail(h, LBM_ERR_CAPACITY, "more than %d particles met one brick; results are invalid", MAXPB);
    if (st[ST_ERR] & ERRB_DEM_CAPACITY)
        return fail(h, LBM_ERR_CAPACITY, "a particle had more than %d candidate contact partners; results are invalid",
                    kDemMaxAdj);
    if (st[ST_ERR] & ERRB_DEM_REACH)
        return fail(h, LBM_ERR_CAPACITY, "a particle moved further in one step than |v| + |a| + %.2f lu, the bound the "
                    "DEM's contact planning assumed; results are invalid", (double)0.25f);
    return LBM_OK;
}

int lbm_get_forces(lbm_handle *h, double *F, double *T, lbm_particle *state_out) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    // everything is read into the page-locked buffer with asynchronous
    // copies and one wait; the status is checked before anything is returned
    const size_t n = (size_t)h->np;
    const size_t P = (size_t)h->cfg.max_particles;
    int *st = reinterpret_cast<int *>(h->pin);
    long long *fix = reinterpret_cast<long long *>(h->pin + ST_SLOTS * 4);
    double *fd = reinterpret_cast<double *>(h->pin + ST_SLOTS * 4 + P * 48);
    DevParticle *dev = reinterpret_cast<DevParticle *>(h->pin + ST_SLOTS * 4 + P * 96);
    const bool f64 = h->cfg.storage == LBM_STORE_F64;
    int rc = cuda_check(h, cudaMemcpyAsync(st, h->ws + h->L.status, ST_SLOTS * 4, cudaMemcpyDeviceToHost, h->stream),
                        "cudaMemcpyAsync(status)");
    if (rc == LBM_OK && n > 0 && (F || T)) {
        if (!f64) {
            // FP32 and below: exact fixed-point totals (units of 2^-40)
            rc = cuda_check(h, cudaMemcpyAsync(fix, h->ws + last_bin_region(h) + h->L.ffix_off, n * 48,
                                               cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(F)");
        } else {
            rc = cuda_check(h, cudaMemcpyAsync(fd, h->ws + h->L.Fh, n * 24, cudaMemcpyDeviceToHost, h->stream),
                            "cudaMemcpyAsync(F)");
            if (rc == LBM_OK)
                rc = cuda_check(h, cudaMemcpyAsync(fd + 3 * n, h->ws + h->L.Th, n * 24, cudaMemcpyDeviceToHost,
                                                   h->stream), "cudaMemcpyAsync(T)");
        }
    }
    if (rc == LBM_OK && n > 0 && state_out)
        rc = cuda_check(h, cudaMemcpyAsync(dev, h->ws + h->L.parts, n * sizeof(DevParticle), cudaMemcpyDeviceToHost,
                                           h->stream), "cudaMemcpyAsync(particles)");
    if (rc == LBM_OK) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    // the last upload from the buffer may have gone out on a stream used
    // before lbm_set_stream(): wait for it by its own event
    if (rc == LBM_OK && h->pin_busy) rc = cuda_check(h, cudaEventSynchronize(h->ev_pin), "cudaEventSynchronize");
    if (rc != LBM_OK) return rc;
    h->pin_busy = false;  // every earlier upload from the buffer is done
    if ((rc = status_code(h, st)) != LBM_OK) return rc;
    if (n == 0) return LBM_OK;
    for (size_t j = 0; j < n; j++)
        for (int a = 0; a < 3; a++) {
            if (F) F[3 * j + a] = f64 ? fd[3 * j + a] : std::ldexp((double)fix[6 * j + a], -kForceFixBits);
            if (T) T[3 * j + a] = f64 ? fd[3 * n + 3 * j + a] : std::ldexp((double)fix[6 * j + 3 + a], -kForceFixBits);
        }
    if (state_out) {
        for (size_t j = 0; j < n; j++) {
            const DevParticle &d = dev[j];
            lbm_particle &p = state_out[j];
            std::memset(&p, 0, sizeof(p));
            p.n_cp = d.ncp;
            p.fixed = d.fixed;
            for (int k = 0; k < d.ncp; k++) {
                for (int a = 0; a < 3; a++) p.cp[k][a] = d.cpu[k][a];
                p.K[k] = d.K[k];
            }
            p.Rs = d.Rs; p.density = d.density; p.mass = d.mass;
            for (int a = 0; a < 9; a++) p.inertia[a] = d.Iu[a];
            for (int a = 0; a < 3; a++) { p.x[a] = d.x[a]; p.v[a] = d.v[a]; p.w[a] = d.w[a]; }
            const double qUc[4] = {d.qU[0], -d.qU[1], -d.qU[2], -d.qU[3]};
            quat_mul(d.q, qUc, p.q);  // back to the caller's body frame
        }
    }
    return LBM_OK;
}

int lbm_get_contact_forces(lbm_handle *h, double *F, double *T) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    int st[ST_SLOTS];
    int rc = read_status(h, st);
    if (rc != LBM_OK) return rc;
    if ((rc = status_code(h, st)) != LBM_OK) return rc;
    const size_t n = (size_t)h->np;
    if (n == 0) return LBM_OK;
    if (F) rc = cuda_check(h, cudaMemcpyAsync(F, h->ws + h->L.Fc, n * 24, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(Fc)");
    if (rc == LBM_OK && T)
        rc = cuda_check(h, cudaMemcpyAsync(T, h->ws + h->L.Tc, n * 24, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(Tc)");
    if (rc == LBM_OK) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

int lbm_get_fields(lbm_handle *h, void *dev_rho, void *dev_u, void *dev_flags) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    Params P = current_params(h);
    by_storage<DoFields>(h->cfg.storage, P, (double *)dev_rho, (double *)dev_u, (uint16_t *)dev_flags, h->stream);
    int rc = cuda_check(h, cudaGetLastError(), "fields kernel launch");
    if (rc == LBM_OK) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

int lbm_set_populations(lbm_handle *h, const void *dev_f) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (!dev_f) return fail(h, LBM_ERR_BAD_ARG, "dev_f is NULL");
    Params P = current_params(h);
    by_storage<DoSetPop>(h->cfg.storage, P, (const double *)dev_f, h->stream);
    int rc = cuda_check(h, cudaGetLastError(), "set_populations kernel launch");
    if (rc == LBM_OK) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

int lbm_get_populations(lbm_handle *h, void *dev_f) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (!dev_f) return fail(h, LBM_ERR_BAD_ARG, "dev_f is NULL");
    Params P = current_params(h);
    by_storage<DoGetPop>(h->cfg.storage, P, (double *)dev_f, h->stream);
    int rc = cuda_check(h, cudaGetLastError(), "get_populations kernel launch");
    if (rc == LBM_OK) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

int lbm_check(lbm_handle *h) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    Params P = current_params(h);
    by_storage<DoCheck>(h->cfg.storage, P, h->stream);
    int rc = cuda_check(h, cudaGetLastError(), "check kernel launch");
    if (rc != LBM_OK) return rc;
    int st[ST_SLOTS];
    if ((rc = read_status(h, st)) != LBM_OK) return rc;
    if ((rc = status_code(h, st)) != LBM_OK) return rc;
    if (st[ST_ERR] & ERRB_DIVERGED)
        return fail(h, LBM_ERR_DIVERGED, "non-finite populations or |u| > 0.5 at a fluid node");
    return LBM_OK;
}

int lbm_get_counters(lbm_handle *h, int64_t *steps, int32_t *nrefill, int32_t *nlinks, int32_t *near_bricks) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    int c[kStepCounters];
    int rc = cuda_check(h, cudaMemcpyAsync(c, h->ws + last_bin_region(h) + (size_t)h->L.nbricks * 4, sizeof(c),
                                           cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(counters)");
    if (rc == LBM_OK) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) return rc;
    if (steps) *steps = h->steps;
    if (nrefill) *nrefill = c[CNT_NREFILL];
    if (nlinks) *nlinks = c[CNT_NLINKS];
    if (near_bricks) *near_bricks = c[CNT_NEAR];
    return LBM_OK;
}

static void release_profile(lbm_handle *h) {
    for (int k = 0; k < kProfKernels; k++) {
        for (int a = 0; a < 2; a++) {
            for (cudaEvent_t e : h->ev[k][a]) cudaEventDestroy(e);
            h->ev[k][a].clear();
        }
        h->nrec[k] = h->nseen[k] = 0;
    }
}

int lbm_profile(lbm_handle *h, int enable) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    cudaStreamSynchronize(h->stream);
    cudaStreamSynchronize(h->aux);
    cudaStreamSynchronize(h->hi);
    release_profile(h);
    h->prof = enable != 0 ? (1u << kProfKernels) - 1u : 0u;
    h->prof_every = 1;
    return LBM_OK;
}

int lbm_profile_mask(lbm_handle *h, unsigned mask, int every) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (mask >> kProfKernels) return fail(h, LBM_ERR_BAD_ARG, "mask has bits beyond the %d kernels", kProfKernels);
    if (every < 1) return fail(h, LBM_ERR_BAD_ARG, "every must be >= 1");
    cudaStreamSynchronize(h->stream);
    cudaStreamSynchronize(h->aux);
    cudaStreamSynchronize(h->hi);
    release_profile(h);
    h->prof = mask;
    h->prof_every = every;
    return LBM_OK;
}

int lbm_profile_read(lbm_handle *h, int kernel, double *total_ms, int64_t *launches) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (kernel < 0 || kernel >= kProfKernels) return fail(h, LBM_ERR_BAD_ARG, "kernel index out of range");
    int rc = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) return rc;
    double sum = 0.0;
    for (int64_t i = 0; i < h->nrec[kernel]; i++) {
        float ms = 0.f;
        rc = cuda_check(h, cudaEventElapsedTime(&ms, h->ev[kernel][0][(size_t)i], h->ev[kernel][1][(size_t)i]),
                        "cudaEventElapsedTime");
        if (rc != LBM_OK) return rc;
        sum += ms;
    }
    if (total_ms) *total_ms = sum;
    if (launches) *launches = h->nrec[kernel];
    return LBM_OK;
}

int lbm_set_schedule(lbm_handle *h, int plain_ctas_per_sm, int chain_ctas_per_sm) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (plain_ctas_per_sm < 0 || plain_ctas_per_sm > 4 || chain_ctas_per_sm < 0 || chain_ctas_per_sm > 4)
        return fail(h, LBM_ERR_BAD_ARG, "CTAs per SM must be in 0..4");
    h->plain_per_sm = plain_ctas_per_sm;
    h->chain_per_sm = chain_ctas_per_sm;
    return LBM_OK;
}

int lbm_set_plain_speculation(lbm_handle *h, int mode) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (mode < -1 || mode > 1) return fail(h, LBM_ERR_BAD_ARG, "mode must be -1, 0 or 1");
    h->plain_spec_mode = mode;
    return LBM_OK;
}

int lbm_set_stream(lbm_handle *h, void *cuda_stream) {
    if (!h) return fail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return LBM_OK;
}

int lbm_destroy(lbm_handle *h) {
    if (!h) return LBM_OK;
    cudaStreamSynchronize(h->stream);
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->hi) cudaStreamSynchronize(h->hi);
    if (h->dem2) cudaStreamSynchronize(h->dem2);
    release_profile(h);
    for (cudaEvent_t e : {h->ev_fork, h->ev_bin, h->ev_plain, h->ev_near, h->ev_join, h->ev_pin, h->ev_dsplit,
                          h->ev_dfree})
        if (e) cudaEventDestroy(e);
    if (h->pin) cudaFreeHost(h->pin);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->hi) cudaStreamDestroy(h->hi);
    if (h->dem2) cudaStreamDestroy(h->dem2);
    delete h;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_handle *h) { return h ? h->err : g_init_error; }

}  // extern "C"

// ===========================================================================
// Batched lattices
// ===========================================================================
struct lbm_batch {
    int n;
    std::vector<lbm_handle *> cases;
    std::vector<size_t> bin1;   // workspace offset of each case's second per-step region
    char *ws;
    // `stream` is the caller's; graphs are captured on and launched into the
    // private `cap` (capture is not allowed on the legacy default stream),
    // ordered after and before `stream` by ev_pre / ev_post
    cudaStream_t stream, cap, hi, aux;
    cudaEvent_t ev_fork, ev_bin, ev_plain, ev_near, ev_join, ev_pre, ev_post;
    size_t tab_off, span_off, item_off, ctr_off, span_case_off, swarp_off;  // device tables at the workspace start
    int Q, storage;
    bool force;
    int g_chain, plain_chunk;
    int total_spans, bin_items, total_swarps;
    int static_state;            // fixed-geometry sweep of all cases: 0 not built, 1 built, -1 did not fit
    bool graph_fixed;            // the captured graph runs the fixed-geometry sweep
    std::vector<Params> tab_host;  // the device table's rows
    bool dirty;
    int64_t steps;
    int static_steps;  // steps since the last lbm_batch_set_particles (saturating)
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int graph_steps;
    char err[256];
};

namespace {

thread_local char g_batch_error[256] = "no error";

int bfail(lbm_batch *b, int code, const char *fmt, ...) {
    char *buf = b ? b->err : g_batch_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}
int bcheck(lbm_batch *b, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    return bfail(b, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Workspace: tables, then per case its single-lattice layout followed by a
// second per-step region (the per-step region alternates by step parity).
struct BatchLayout {
    size_t tab, span_off, item_off, ctr, span_case, swarp_off, total;
    std::vector<size_t> base, bin1;
};

const char *batch_check(const lbm_config *cfgs, int n) {
    if (!cfgs || n < 1) return "need at least one case";
    if (n > 65535) return "at most 65535 cases";
    for (int c = 0; c < n; c++) {
        if (const char *m = check_config(&cfgs[c])) return m;
        if (cfgs[c].lattice != cfgs[0].lattice) return "all cases must use the same lattice";
        if (cfgs[c].storage != cfgs[0].storage) return "all cases must use the same storage";
        if (cfgs[c].storage == LBM_STORE_F64) return "batched cases store FP32, FP16 or BF16";
        if (cfgs[c].n_sub != 0) return "batched cases hold fixed particles (n_sub = 0)";
    }
    return nullptr;
}

void batch_layout(const lbm_config *cfgs, int n, BatchLayout *B) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    B->tab = take(2 * (size_t)n * sizeof(Params));
    B->span_off = take(((size_t)n + 1) * 4);
    B->item_off = take(((size_t)n + 1) * 4);
    B->ctr = take(4 * 4);
    B->swarp_off = take(((size_t)n + 1) * 4);
    size_t spans = 0;
    for (int c = 0; c < n; c++) {
        Layout L;
        make_layout(&cfgs[c], &L);
        spans += (size_t)((L.N + BRICK - 1) / BRICK);
    }
    B->span_case = take(spans * 2);
    B->base.resize(n);
    B->bin1.resize(n);
    for (int c = 0; c < n; c++) {
        Layout L;
        make_layout(&cfgs[c], &L);
        B->base[c] = take(L.total);
        B->bin1[c] = take(L.bin_bytes);
    }
    B->total = o;
}

// Device tables: per case its Params for either step parity, and the prefix
// sums the batched kernels map their CTAs with.
int batch_tables(lbm_batch *b) {
    std::vector<Params> tab(2 * (size_t)b->n);
    std::vector<int> soff(b->n + 1), ioff(b->n + 1), woff(b->n + 1);
    soff[0] = ioff[0] = woff[0] = 0;
    for (int c = 0; c < b->n; c++) {
        lbm_handle *h = b->cases[c];
        const int64_t keep_steps = h->steps;
        const int keep_cur = h->cur, keep_fcur = h->fcur;
        for (int p = 0; p < 2; p++) {
            h->cur = p;
            h->fcur = p;
            h->steps = p;
            Params P = make_params(h);
            char *bin_p = p == 0 ? h->ws + h->L.bin : b->ws + b->bin1[c];
            char *bin_q = p == 0 ? b->ws + b->bin1[c] : h->ws + h->L.bin;
            P.bcount = reinterpret_cast<int *>(bin_p);
            P.counters = reinterpret_cast<int *>(bin_p + (size_t)h->L.nbricks * 4);
            P.Ffix = reinterpret_cast<unsigned long long *>(bin_p + h->L.ffix_off);
            P.bin_next = bin_q;
            // rounded up to whole 16-byte stores: each region is a 256-byte
            // aligned allocation of its own
            P.bin_next_bytes = (long long)((h->L.bin_bytes + 15) / 16 * 16);
            tab[(size_t)p * b->n + c] = P;
        }
        h->steps = keep_steps;
        h->cur = keep_cur;
        h->fcur = keep_fcur;
        soff[c + 1] = soff[c] + (int)((h->L.N + BRICK - 1) / BRICK);
        // link-node warps of the fixed-geometry sweep, at least one per case
        woff[c + 1] = woff[c] + std::max(1, (h->snodes_n + kStaticNodesPerWarp - 1) / kStaticNodesPerWarp);
        ioff[c + 1] = ioff[c] + (h->np > 0 ? h->np : 1);
    }
    b->total_spans = soff[b->n];
    b->total_swarps = woff[b->n];
    b->tab_host = tab;
    b->bin_items = ioff[b->n];
    int rc = bcheck(b, cudaMemcpyAsync(b->ws + b->tab_off, tab.data(), tab.size() * sizeof(Params),
                                       cudaMemcpyHostToDevice, b->stream), "cudaMemcpyAsync(tables)");
    if (rc == LBM_OK)
        rc = bcheck(b, cudaMemcpyAsync(b->ws + b->span_off, soff.data(), soff.size() * 4, cudaMemcpyHostToDevice,
                                       b->stream), "cudaMemcpyAsync(tables)");
    if (rc == LBM_OK)
        rc = bcheck(b, cudaMemcpyAsync(b->ws + b->item_off, ioff.data(), ioff.size() * 4, cudaMemcpyHostToDevice,
                                       b->stream), "cudaMemcpyAsync(tables)");
    std::vector<uint16_t> scase((size_t)soff[b->n]);
    for (int c = 0; c < b->n; c++)
        for (int k = soff[c]; k < soff[c + 1]; k++) scase[(size_t)k] = (uint16_t)c;
    if (rc == LBM_OK)
        rc = bcheck(b, cudaMemcpyAsync(b->ws + b->span_case_off, scase.data(), scase.size() * 2,
                                       cudaMemcpyHostToDevice, b->stream), "cudaMemcpyAsync(tables)");
    if (rc == LBM_OK)
        rc = bcheck(b, cudaMemcpyAsync(b->ws + b->swarp_off, woff.data(), woff.size() * 4, cudaMemcpyHostToDevice,
                                       b->stream), "cudaMemcpyAsync(tables)");
    if (rc == LBM_OK) rc = bcheck(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (rc == LBM_OK) b->dirty = false;
    return rc;
}

BatchArgs batch_args(lbm_batch *b) {
    BatchArgs B;
    B.tab = reinterpret_cast<const Params *>(b->ws + b->tab_off);
    B.ncases = b->n;
    B.span_off = reinterpret_cast<const int *>(b->ws + b->span_off);
    B.item_off = reinterpret_cast<const int *>(b->ws + b->item_off);
    B.span_case = reinterpret_cast<const uint16_t *>(b->ws + b->span_case_off);
    B.ctr = reinterpret_cast<unsigned *>(b->ws + b->ctr_off);
    B.g_chain = b->g_chain;
    B.plain_chunk = b->plain_chunk;
    B.swarp_off = reinterpret_cast<const int *>(b->ws + b->swarp_off);
    return B;
}

template <typename S>
struct DoBatchStep {
    static void flags(const BatchArgs &B, int Q, cudaStream_t st) { launch_flags_batch_t<S>(B, Q, st); }
    static void near(const BatchArgs &B, int Q, bool f, cudaStream_t st) { launch_near_batch_t<S>(B, Q, f, st); }
    static void plain(const BatchArgs &B, int Q, bool f, int grid, cudaStream_t st) {
        launch_plain_batch_t<S>(B, Q, f, grid, st);
    }
    static void static_plain(const BatchArgs &B, int Q, bool f, int grid, cudaStream_t st) {
        launch_static_plain_batch_t<S>(B, Q, f, grid, st);
    }
    static void static_links(const BatchArgs &B, int Q, bool f, int warps, cudaStream_t st) {
        launch_static_links_batch_t<S>(B, Q, f, warps, st);
    }
    static void static_build(const Params &P, cudaStream_t st) { launch_static_build_t<S>(P, st); }
};

template <typename Fn>
void by_batch_storage(int storage, Fn &&fn) {
    switch (storage) {
        case LBM_STORE_F32: fn(DoBatchStep<float>()); break;
        case LBM_STORE_F16: fn(DoBatchStep<__half>()); break;
        default: fn(DoBatchStep<__nv_bfloat16>()); break;
    }
}

// nsteps steps on the batch's streams, forked from and joined into b->cap
// (the sequence a graph is captured from).
int batch_issue(lbm_batch *b, int nsteps, bool flags, bool fixed) {
    const BatchArgs B = batch_args(b);
    const int plain_grid = (b->total_spans + b->plain_chunk - 1) / b->plain_chunk;
    cudaError_t e = cudaEventRecord(b->ev_fork, b->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->hi, b->ev_fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->aux, b->ev_fork, 0);
    for (int t = 0; fixed && t < nsteps && e == cudaSuccess; t++) {
        // fixed-geometry sweep: the link nodes after the previous step's plain
        // nodes, the plain nodes after the previous step's link nodes
        if (t > 0) e = cudaStreamWaitEvent(b->hi, b->ev_plain, 0);
        if (e == cudaSuccess && t > 0) e = cudaStreamWaitEvent(b->aux, b->ev_near, 0);
        if (e != cudaSuccess) break;
        by_batch_storage(b->storage, [&](auto D) { D.static_links(B, b->Q, b->force, b->total_swarps, b->hi); });
        by_batch_storage(b->storage, [&](auto D) { D.static_plain(B, b->Q, b->force, plain_grid, b->aux); });
        e = cudaEventRecord(b->ev_plain, b->aux);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_near, b->hi);
    }
    for (int t = 0; !fixed && t < nsteps && e == cudaSuccess; t++) {
        launch_bin_batch(B, b->bin_items, b->hi);
        e = cudaEventRecord(b->ev_bin, b->hi);
        if (e != cudaSuccess) break;
        if (flags) by_batch_storage(b->storage, [&](auto D) { D.flags(B, b->Q, b->hi); });
        if (t > 0) e = cudaStreamWaitEvent(b->hi, b->ev_plain, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->aux, b->ev_bin, 0);
        if (e != cudaSuccess) break;
        by_batch_storage(b->storage, [&](auto D) { D.plain(B, b->Q, b->force, plain_grid, b->aux); });
        e = cudaEventRecord(b->ev_plain, b->aux);
        if (e != cudaSuccess) break;
        by_batch_storage(b->storage, [&](auto D) { D.near(B, b->Q, b->force, b->hi); });
        e = cudaEventRecord(b->ev_near, b->hi);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->aux, b->ev_near, 0);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_join, b->hi);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev_join, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev_plain, 0);
    if (e == cudaSuccess) e = cudaGetLastError();
    return bcheck(b, e, "batched step launch");
}

void drop_graph(lbm_batch *b);

// Record the fixed geometry of every case from the brick lists of the last
// step taken (steps_done of them), on `cap`, and synchronise; all cases take
// the fixed-geometry sweep, or none if one did not fit.
int batch_build_static(lbm_batch *b, int64_t steps_done) {
    const int p = (int)((steps_done - 1) & 1);
    int rc = LBM_OK;
    for (int c = 0; c < b->n && rc == LBM_OK; c++) {
        lbm_handle *h = b->cases[c];
        Params P = b->tab_host[(size_t)p * b->n + c];
        P.step = (int)(steps_done - 1);
        cudaError_t e = cudaMemsetAsync(h->ws + h->L.sskip, 0, (size_t)h->L.N, b->cap);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->L.scount, 0, 8, b->cap);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->L.smf, 0, (size_t)h->cfg.max_particles * 48, b->cap);
        if (e == cudaSuccess) by_batch_storage(b->storage, [&](auto D) { D.static_build(P, b->cap); });
        if (e == cudaSuccess) e = cudaGetLastError();
        rc = bcheck(b, e, "fixed-geometry build");
    }
    std::vector<int> cnt(2 * (size_t)b->n), st((size_t)ST_SLOTS * b->n);
    for (int c = 0; c < b->n && rc == LBM_OK; c++) {
        lbm_handle *h = b->cases[c];
        cudaError_t e = cudaMemcpyAsync(&cnt[2 * (size_t)c], h->ws + h->L.scount, 8, cudaMemcpyDeviceToHost, b->cap);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&st[(size_t)ST_SLOTS * c], h->ws + h->L.status, ST_SLOTS * 4, cudaMemcpyDeviceToHost,
                                b->cap);
        rc = bcheck(b, e, "fixed-geometry build");
    }
    if (rc == LBM_OK) rc = bcheck(b, cudaStreamSynchronize(b->cap), "cudaStreamSynchronize");
    if (rc != LBM_OK) return rc;
    bool fits = true;
    for (int c = 0; c < b->n; c++)
        if (st[(size_t)ST_SLOTS * c + ST_ERR] & ERRB_STATIC_CAPACITY) fits = false;
    for (int c = 0; c < b->n && rc == LBM_OK; c++) {
        lbm_handle *h = b->cases[c];
        if (st[(size_t)ST_SLOTS * c + ST_ERR] & ERRB_STATIC_CAPACITY) {
            int *err = &st[(size_t)ST_SLOTS * c + ST_ERR];
            *err &= ~ERRB_STATIC_CAPACITY;
            rc = bcheck(b, cudaMemcpy(h->ws + h->L.status, err, 4, cudaMemcpyHostToDevice), "cudaMemcpy(status)");
        }
        h->static_state = fits ? 1 : -1;
        h->snodes_n = fits ? cnt[2 * (size_t)c] : 0;
    }
    if (rc != LBM_OK) return rc;
    b->static_state = fits ? 1 : -1;
    drop_graph(b);
    return batch_tables(b);
}

void drop_graph(lbm_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_steps = 0;
}

}  // namespace

extern "C" {

int lbm_batch_workspace_size(const lbm_config *cfgs, int ncases, size_t *bytes) {
    if (const char *m = batch_check(cfgs, ncases)) return bfail(nullptr, LBM_ERR_BAD_ARG, "%s", m);
    if (!bytes) return bfail(nullptr, LBM_ERR_BAD_ARG, "bytes is NULL");
    BatchLayout BL;
    batch_layout(cfgs, ncases, &BL);
    *bytes = BL.total;
    return LBM_OK;
}

int lbm_batch_init(const lbm_config *cfgs, int ncases, void *dev_ws, size_t ws_bytes, void *cuda_stream,
                   lbm_batch **out) {
    if (!out) return bfail(nullptr, LBM_ERR_BAD_ARG, "out is NULL");
    *out = nullptr;
    if (const char *m = batch_check(cfgs, ncases)) return bfail(nullptr, LBM_ERR_BAD_ARG, "%s", m);
    if (!dev_ws || reinterpret_cast<uintptr_t>(dev_ws) % kAlign)
        return bfail(nullptr, LBM_ERR_BAD_ARG, "workspace NULL or not 256-byte aligned");
    BatchLayout BL;
    batch_layout(cfgs, ncases, &BL);
    if (ws_bytes < BL.total)
        return bfail(nullptr, LBM_ERR_WS_TOO_SMALL, "workspace of %zu bytes, %zu needed", ws_bytes, BL.total);
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ERR_BAD_ARG, "out of host memory");
    b->n = ncases;
    b->ws = static_cast<char *>(dev_ws);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->tab_off = BL.tab;
    b->span_off = BL.span_off;
    b->item_off = BL.item_off;
    b->ctr_off = BL.ctr;
    b->span_case_off = BL.span_case;
    b->swarp_off = BL.swarp_off;
    b->bin1 = BL.bin1;
    b->Q = cfgs[0].lattice;
    b->storage = cfgs[0].storage;
    b->force = false;
    for (int c = 0; c < ncases; c++)
        for (int a = 0; a < 3; a++) b->force = b->force || cfgs[c].force[a] != 0.0;
    b->g_chain = kDefaultBatchChainCtas;
    b->plain_chunk = kDefaultBatchPlainChunk;
    b->steps = 0;
    b->static_steps = 0;
    b->static_state = 0;
    b->graph_fixed = false;
    b->total_swarps = 0;
    std::snprintf(b->err, sizeof(b->err), "no error");
    int rc = LBM_OK;
    int prio_low = 0, prio_high = 0;
    rc = bcheck(b, cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high), "cudaDeviceGetStreamPriorityRange");
    if (rc == LBM_OK)
        rc = bcheck(b, cudaStreamCreateWithPriority(&b->aux, cudaStreamNonBlocking, prio_low), "cudaStreamCreate");
    if (rc == LBM_OK)
        rc = bcheck(b, cudaStreamCreateWithPriority(&b->hi, cudaStreamNonBlocking, prio_high), "cudaStreamCreate");
    if (rc == LBM_OK) rc = bcheck(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    for (cudaEvent_t *e : {&b->ev_fork, &b->ev_bin, &b->ev_plain, &b->ev_near, &b->ev_join, &b->ev_pre, &b->ev_post})
        if (rc == LBM_OK) rc = bcheck(b, cudaEventCreateWithFlags(e, cudaEventDisableTiming), "cudaEventCreate");
    // tables, counters and the second per-step regions start at zero
    if (rc == LBM_OK) rc = bcheck(b, cudaMemsetAsync(b->ws, 0, BL.total, b->stream), "cudaMemsetAsync");
    for (int c = 0; c < ncases && rc == LBM_OK; c++) {
        lbm_handle *h = nullptr;
        Layout L;
        make_layout(&cfgs[c], &L);
        rc = init_handle(&cfgs[c], b->ws + BL.base[c], L.total, b->stream, false, &h);
        if (rc != LBM_OK) {
            bfail(b, rc, "case %d: %s", c, g_init_error);
            break;
        }
        b->cases.push_back(h);
    }
    if (rc == LBM_OK) rc = batch_tables(b);
    if (rc != LBM_OK) {
        std::snprintf(g_batch_error, sizeof(g_batch_error), "%s", b->err);
        lbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_particles(lbm_batch *b, int c, const lbm_particle *host, int n) {
    if (!b) return bfail(nullptr, LBM_ERR_BAD_ARG, "batch is NULL");
    if (c < 0 || c >= b->n) return bfail(b, LBM_ERR_BAD_ARG, "case %d out of range", c);
    for (int j = 0; j < n; j++)
        if (host && !host[j].fixed) return bfail(b, LBM_ERR_BAD_ARG, "batched cases hold fixed particles");
    const int rc = lbm_set_particles(b->cases[c], host, n);
    if (rc != LBM_OK) return bfail(b, rc, "case %d: %s", c, b->cases[c]->err);
    b->dirty = true;
    b->static_steps = 0;
    b->static_state = 0;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int nsteps) {
    if (!b) return bfail(nullptr, LBM_ERR_BAD_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(b, LBM_ERR_BAD_ARG, "nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    int rc = LBM_OK;
    if (b->dirty) {
        const int items = b->bin_items;
        rc = batch_tables(b);
        if (rc != LBM_OK) return rc;
        if (b->bin_items != items) drop_graph(b);
    }
    // the steps run on `cap`, after everything issued on the caller's stream
    // so far, and the caller's stream continues after them
    rc = bcheck(b, cudaEventRecord(b->ev_pre, b->stream), "cudaEventRecord");
    if (rc == LBM_OK) rc = bcheck(b, cudaStreamWaitEvent(b->cap, b->ev_pre, 0), "cudaStreamWaitEvent");
    if (rc != LBM_OK) return rc;
    // every particle of a batch is fixed: the first kStaticFlagSteps steps
    // after particles are set run the flag pass (then both flag buffers and
    // the per-brick solid marks hold the flags); the fixed geometry is then
    // recorded once, and the later steps run the fixed-geometry sweep (or the
    // brick sweeps without the flag pass, if it did not fit), as replays of
    // one captured graph of kBatchGraphSteps steps and a direct remainder
    const int direct = std::min(nsteps, std::max(0, kStaticFlagSteps - b->static_steps));
    if (direct > 0) rc = batch_issue(b, direct, true, false);
    if (rc != LBM_OK) return rc;
    if (direct < nsteps && b->static_state == 0) {
        rc = batch_build_static(b, b->steps + direct);
        if (rc != LBM_OK) return rc;
    }
    const bool fixed = b->static_state == 1;
    const int reps = (nsteps - direct) / kBatchGraphSteps;
    const int rest = (nsteps - direct) % kBatchGraphSteps;
    if (reps > 0 && b->exec && b->graph_fixed != fixed) drop_graph(b);
    if (reps > 0 && !b->exec) {
        // replays read the step numbers from the device counters, so the same
        // graph serves every later call
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bcheck(b, e, "cudaStreamBeginCapture");
        const int rc_issue = batch_issue(b, kBatchGraphSteps, false, fixed);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->cap, &g);
        if (rc_issue != LBM_OK) {
            if (g) cudaGraphDestroy(g);
            return rc_issue;
        }
        if (e != cudaSuccess) return bcheck(b, e, "cudaStreamEndCapture");
        b->graph = g;
        // the kernel nodes keep the priorities of the streams they were
        // captured from (the particle chain above the plain sweep)
        e = cudaGraphInstantiateWithFlags(&b->exec, g, cudaGraphInstantiateFlagUseNodePriority);
        if (e != cudaSuccess) {
            drop_graph(b);
            return bcheck(b, e, "cudaGraphInstantiate");
        }
        b->graph_steps = kBatchGraphSteps;
        b->graph_fixed = fixed;
    }
    for (int k = 0; k < reps && rc == LBM_OK; k++) rc = bcheck(b, cudaGraphLaunch(b->exec, b->cap), "cudaGraphLaunch");
    if (rc == LBM_OK && rest > 0) rc = batch_issue(b, rest, false, fixed);
    if (rc == LBM_OK) rc = bcheck(b, cudaEventRecord(b->ev_post, b->cap), "cudaEventRecord");
    if (rc == LBM_OK) rc = bcheck(b, cudaStreamWaitEvent(b->stream, b->ev_post, 0), "cudaStreamWaitEvent");
    if (rc != LBM_OK) return rc;
    b->static_steps = std::min(kStaticFlagSteps, b->static_steps + nsteps);
    b->steps += nsteps;
    for (lbm_handle *h : b->cases) {
        h->steps = b->steps;
        h->cur = (int)(b->steps & 1);
        h->fcur = h->cur;
    }
    return LBM_OK;
}

int lbm_batch_get_forces(lbm_batch *b, int c, double *F, double *T) {
    if (!b) return bfail(nullptr, LBM_ERR_BAD_ARG, "batch is NULL");
    if (c < 0 || c >= b->n) return bfail(b, LBM_ERR_BAD_ARG, "case %d out of range", c);
    lbm_handle *h = b->cases[c];
    const size_t n = (size_t)h->np;
    if (n == 0) return LBM_OK;
    // the last step's per-step region (parity of step steps-1)
    const char *bin = b->steps > 0 && ((b->steps - 1) & 1) ? b->ws + b->bin1[c] : h->ws + h->L.bin;
    std::vector<long long> fix(n * 6);
    int st[ST_SLOTS];
    int rc = bcheck(b, cudaMemcpyAsync(fix.data(), bin + h->L.ffix_off, n * 48, cudaMemcpyDeviceToHost, b->stream),
                    "cudaMemcpyAsync(F)");
    if (rc == LBM_OK)
        rc = bcheck(b, cudaMemcpyAsync(st, h->ws + h->L.status, sizeof(st), cudaMemcpyDeviceToHost, b->stream),
                    "cudaMemcpyAsync(status)");
    if (rc == LBM_OK) rc = bcheck(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) return rc;
    if (st[ST_ERR] & ERRB_BRICK_OVERFLOW)
        return bfail(b, LBM_ERR_CAPACITY, "case %d: more than %d particles met one brick", c, MAXPB);
    for (size_t j = 0; j < n; j++)
        for (int a = 0; a < 3; a++) {
            if (F) F[3 * j + a] = std::ldexp((double)fix[6 * j + a], -kForceFixBits);
            if (T) T[3 * j + a] = std::ldexp((double)fix[6 * j + 3 + a], -kForceFixBits);
        }
    return LBM_OK;
}

int lbm_batch_get_all_forces(lbm_batch *b, double *F, double *T) {
    if (!b) return bfail(nullptr, LBM_ERR_BAD_ARG, "batch is NULL");
    // every case's status and totals into its handle's page-locked buffer
    // with asynchronous copies, then one wait
    int rc = LBM_OK;
    for (int c = 0; c < b->n && rc == LBM_OK; c++) {
        lbm_handle *h = b->cases[c];
        const size_t n = (size_t)h->np;
        rc = bcheck(b, cudaMemcpyAsync(h->pin, h->ws + h->L.status, ST_SLOTS * 4, cudaMemcpyDeviceToHost, b->stream),
                    "cudaMemcpyAsync(status)");
        if (rc != LBM_OK || n == 0) continue;
        const char *bin = b->steps > 0 && ((b->steps - 1) & 1) ? b->ws + b->bin1[c] : h->ws + h->L.bin;
        rc = bcheck(b, cudaMemcpyAsync(h->pin + ST_SLOTS * 4, bin + h->L.ffix_off, n * 48, cudaMemcpyDeviceToHost,
                                       b->stream), "cudaMemcpyAsync(F)");
    }
    if (rc == LBM_OK) rc = bcheck(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) return rc;
    size_t row = 0;
    for (int c = 0; c < b->n; c++) {
        lbm_handle *h = b->cases[c];
        const int *st = reinterpret_cast<const int *>(h->pin);
        if (st[ST_ERR] & ERRB_BRICK_OVERFLOW)
            return bfail(b, LBM_ERR_CAPACITY, "case %d: more than %d particles met one brick", c, MAXPB);
        const long long *fix = reinterpret_cast<const long long *>(h->pin + ST_SLOTS * 4);
        for (int j = 0; j < h->np; j++, row++)
            for (int a = 0; a < 3; a++) {
                if (F) F[3 * row + a] = std::ldexp((double)fix[6 * j + a], -kForceFixBits);
                if (T) T[3 * row + a] = std::ldexp((double)fix[6 * j + 3 + a], -kForceFixBits);
            }
    }
    return LBM_OK;
}

int lbm_batch_get_populations(lbm_batch *b, int c, void *dev_f) {
    if (!b) return bfail(nullptr, LBM_ERR_BAD_ARG, "batch is NULL");
    if (c < 0 || c >= b->n) return bfail(b, LBM_ERR_BAD_ARG, "case %d out of range", c);
    const int rc = lbm_get_populations(b->cases[c], dev_f);
    if (rc != LBM_OK) return bfail(b, rc, "case %d: %s", c, b->cases[c]->err);
    return LBM_OK;
}

int lbm_batch_set_schedule(lbm_batch *b, int chain_ctas_per_case, int plain_blocks_per_cta) {
    if (!b) return bfail(nullptr, LBM_ERR_BAD_ARG, "batch is NULL");
    if (chain_ctas_per_case < 1 || chain_ctas_per_case > 64 || plain_blocks_per_cta < 1 || plain_blocks_per_cta > 64)
        return bfail(b, LBM_ERR_BAD_ARG, "schedule out of range");
    if (chain_ctas_per_case != b->g_chain || plain_blocks_per_cta != b->plain_chunk) drop_graph(b);
    b->g_chain = chain_ctas_per_case;
    b->plain_chunk = plain_blocks_per_cta;
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch *b, int trial_steps, int *chain_ctas_per_case, int *plain_blocks_per_cta,
                   double *best_ms_per_step) {
    if (!b) return bfail(nullptr, LBM_ERR_BAD_ARG, "batch is NULL");
    if (trial_steps < 1) return bfail(b, LBM_ERR_BAD_ARG, "trial_steps < 1");
    static const int kChain[] = {4, 8, 16, 32, 64};
    static const int kChunk[] = {1, 2, 4, 8};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = bcheck(b, cudaEventCreate(&e0), "cudaEventCreate");
    if (rc == LBM_OK) rc = bcheck(b, cudaEventCreate(&e1), "cudaEventCreate");
    float best = 0.f;
    int bg = b->g_chain, bc = b->plain_chunk;
    for (int gi = 0; gi < 5 && rc == LBM_OK; gi++)
        for (int ci = 0; ci < 4 && rc == LBM_OK; ci++) {
            rc = lbm_batch_set_schedule(b, kChain[gi], kChunk[ci]);
            if (rc == LBM_OK) rc = lbm_batch_step(b, trial_steps);  // capture and warm up
            if (rc == LBM_OK) rc = bcheck(b, cudaEventRecord(e0, b->stream), "cudaEventRecord");
            if (rc == LBM_OK) rc = lbm_batch_step(b, trial_steps);
            if (rc == LBM_OK) rc = bcheck(b, cudaEventRecord(e1, b->stream), "cudaEventRecord");
            if (rc == LBM_OK) rc = bcheck(b, cudaEventSynchronize(e1), "cudaEventSynchronize");
            float ms = 0.f;
            if (rc == LBM_OK) rc = bcheck(b, cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            if (rc == LBM_OK && (best == 0.f || ms < best)) {
                best = ms;
                bg = kChain[gi];
                bc = kChunk[ci];
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != LBM_OK) return rc;
    rc = lbm_batch_set_schedule(b, bg, bc);
    if (chain_ctas_per_case) *chain_ctas_per_case = bg;
    if (plain_blocks_per_cta) *plain_blocks_per_cta = bc;
    if (best_ms_per_step) *best_ms_per_step = best / trial_steps;
    return rc;
}

int64_t lbm_batch_steps(const lbm_batch *b) { return b ? b->steps : 0; }

int lbm_batch_destroy(lbm_batch *b) {
    if (!b) return LBM_OK;
    cudaStreamSynchronize(b->stream);
    if (b->hi) cudaStreamSynchronize(b->hi);
    if (b->aux) cudaStreamSynchronize(b->aux);
    if (b->cap) cudaStreamSynchronize(b->cap);
    drop_graph(b);
    for (lbm_handle *h : b->cases) lbm_destroy(h);
    for (cudaEvent_t e : {b->ev_fork, b->ev_bin, b->ev_plain, b->ev_near, b->ev_join, b->ev_pre, b->ev_post})
        if (e) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->aux) cudaStreamDestroy(b->aux);
    if (b->hi) cudaStreamDestroy(b->hi);
    delete b;
    return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err : g_batch_error; }

}  // extern "C"
