// k_dem32: the DEM of §2.3.4 for lattices stored in FP32 or below.
//
// On this GPU an FP64 warp instruction occupies its SM sub-partition for 64
// cycles whether or not its lanes depend on one another (measured with
// clock64: dependent and independent FP64 FMAs alike; FP64 division ~560
// cycles, square root ~680, an FP64<->FP32 conversion ~100), against ~5
// cycles for a dependent FP32 FMA.  The n_s sub-steps of an LBM step are one
// serial chain, so this kernel computes them in FP32:
// - the rigid-body state (x, v, q and the principal-frame angular velocity)
//   is kept as compensated pairs hi + lo (Knuth's two-sum, renormalised), so
//   the state carries ~48 significant bits, while each increment is computed
//   in FP32 from the leading words (relative error ~6e-8 of an increment of
//   size ~h |v|);
// - the contact geometry of Eqs. (5)-(13) is solved by Newton iterations in
//   FP32 in a frame centred on the particle, where coordinates are O(radius),
//   so the overlap delta carries an absolute error of ~1e-6 lu;
// - contact forces are summed per particle in the order of the FP64 path:
//   pairs (m, k) by ascending m, pairs (k, m) by ascending m, walls 0..5.
// The sub-step sequence is that of k_dem: contact forces at the start, then
// per sub-step the first half-kick and drift, the rotation q <- q (x) exp(h
// w/2), the contacts at the new positions, the closing half-kick (implicit in
// w).  Candidate pairs come from a Verlet list (bounding spheres closer than a
// skin), rebuilt when a particle has moved half the skin since.
#include "lbm_internal.cuh"
#include "dem_fp64.cuh"

namespace lbmmb {
namespace {

constexpr int kThreads = 512;
constexpr int kMaxP = kDem32MaxParticles;
constexpr int kMaxAdj = kDemMaxAdj;
constexpr int kWords = kMaxP / 32;
constexpr int kMaxItems = 1024;  // candidate pairs resident in shared memory
constexpr float kSkin = 1.0f;

// ---------------------------------------------------------------------------
// compensated scalar
// ---------------------------------------------------------------------------
struct DF { float hi, lo; };
__device__ __forceinline__ DF df_load(const float s[2]) { return {s[0], s[1]}; }
__device__ __forceinline__ void df_store(float s[2], DF a) { s[0] = a.hi; s[1] = a.lo; }
// a + b: two-sum of hi and b, error and lo folded into the new low word
__device__ __forceinline__ DF df_add(DF a, float b) {
    const float s = __fadd_rn(a.hi, b);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    const float lo = __fadd_rn(a.lo, e);
    const float hi = __fadd_rn(s, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}
// the leading word after adding b (what the increments downstream use)
__device__ __forceinline__ float df_lead(DF a, float b) { return __fadd_rn(a.hi, b); }

// ---------------------------------------------------------------------------
// FP32 vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot3f(const float a[3], const float b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3f(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
// R(q) v (to_world) or R(q)^T v: v + 2(+-w c + u x c), c = u x v
__device__ __forceinline__ void qrot_f(const float q[4], const float v[3], float r[3], bool to_world) {
    const float u[3] = {q[1], q[2], q[3]};
    float c[3], uc[3];
    cross3f(u, v, c);
    cross3f(u, c, uc);
    const float s = to_world ? q[0] : -q[0];
    for (int a = 0; a < 3; a++) r[a] = v[a] + 2.0f * fmaf(s, c[a], uc[a]);
}
// Euler's equations, principal frame
__device__ __forceinline__ void euler_f(const float iI[3], const float cI[3], const float w[3], const float T[3],
                                        float out[3]) {
    out[0] = fmaf(cI[0] * w[1], w[2], iI[0] * T[0]);
    out[1] = fmaf(cI[1] * w[2], w[0], iI[1] * T[1]);
    out[2] = fmaf(cI[2] * w[0], w[1], iI[2] * T[2]);
}
__device__ __forceinline__ float minimg_f(const Params &P, int a, float d) {
    if (P.per[a]) d -= P.dim_f[a] * rintf(d * P.inv_n_f[a]);
    return d;
}

// exp(h w / 2) as (cos - 1, sin(|a|)/|a| * h/2): a = h w / 2
__device__ __forceinline__ void exp_half(float hh, float qh2, const float w[3], float &cm1, float &sc) {
    const float a2 = qh2 * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (a2 <= 1.0f / 256.0f) {
        sc = hh * (1.0f + a2 * (-1.0f / 6.0f + a2 * (1.0f / 120.0f)));
        cm1 = a2 * (-0.5f + a2 * (1.0f / 24.0f + a2 * (-1.0f / 720.0f)));
    } else {
        const float an = sqrtf(a2);
        float sn, cs;
        sincosf(an, &sn, &cs);
        const float s2 = sinf(0.5f * an);
        sc = hh * sn / an;
        cm1 = -2.0f * s2 * s2;
    }
}

// ---------------------------------------------------------------------------
// shared tables: everything a sub-step touches lives here for the whole
// launch (the contact state is loaded from global memory once and written
// back once), so the sub-step chain never waits on an L2 round trip
// ---------------------------------------------------------------------------
template <int CAP, int ITEMS, int CPS, bool kCpb, bool kWarpGroup>
struct SharedT {
    static constexpr bool kCacheCpb = kCpb;         // body-frame control points kept in shared memory
    static constexpr bool kWarp = kWarpGroup;       // one warp per table (else the whole CTA)
    static constexpr int kCap = CAP;                // particles in the tables
    static constexpr int kItems = ITEMS;            // candidate pairs resident in shared memory
    static constexpr int kWordsT = (CAP + 31) / 32;
    static constexpr int kCps = CPS;                // control points of all particles
    float xh[CAP][3], xl[CAP][3];   // position, compensated
    float v[CAP][3];                // velocity (world)
    float w[CAP][3];                // angular velocity (world)
    float xref[CAP][3];             // position at the last list build
    float Fc[CAP][3], Tc[CAP][3];   // contact force / torque of the last evaluation
    float brad[CAP], Rs[CAP], reach[CAP];
    float4 rc[CPS];                 // control points R(q) cpb relative to x, and K
    float4 rc_pad[kWarpGroup ? 32 : 1];  // warp tables: where lanes without a control point store theirs
    float4 cpb[kCpb ? CPS : 1];     // control points in the body frame, and K (put_rc's input)
    int cpo[CAP + 1];               // offsets into rc
    unsigned bits[CAP][(CAP + 31) / 32];  // candidate pairs (i < j)
    unsigned short up[CAP][kMaxAdj];      // partners j > i, ascending
    int dn[CAP][kMaxAdj];                 // (m << 8 | slot of k in up[m]), m < k, ascending
    int nup[CAP], ndn[CAP];
    int gid[CAP];                   // particle index of table entry k (k_dem32: k itself)
    int n;                          // entries in the tables
    int ioff[CAP + 1];              // prefix sums of nup: item of (i, slot) = ioff[i] + slot
    // candidate pairs: contact history and results
    int it_on[ITEMS];
    float it_xm[ITEMS][3], it_xi[ITEMS][3];
    float it_res[ITEMS][9];         // F_i, T_i, T_j
    // walls: contact history
    int w_on[CAP][NWALL];
    float w_xcw[CAP][NWALL][3], w_xi[CAP][NWALL][3];
};
// every particle in one CTA (k_dem32, and k_dem64c for a large contact group)
using Shared = SharedT<kMaxP, kMaxItems, kDem32MaxCp, false, false>;
// a contact group of up to 32 particles (k_dem64c, one CTA per group)
using SharedSmall = SharedT<kSmallContactGroup, 256, kSmallContactGroup * MAXCP, true, false>;
// a contact group of up to kTinyContactGroup particles (one warp each,
// kTinyGroupsPerCta tables per CTA; at most 6 candidate pairs)
using SharedTiny = SharedT<kTinyContactGroup, 8, kTinyContactGroup * MAXCP, false, true>;

// The threads that share one table: the CTA, or for warp tables the warp.
template <class SH> __device__ __forceinline__ int gtid() { return SH::kWarp ? (int)(threadIdx.x & 31) : (int)threadIdx.x; }
template <class SH> __device__ __forceinline__ int gdim() { return SH::kWarp ? 32 : (int)blockDim.x; }
template <class SH> __device__ __forceinline__ void gsync() {
    if constexpr (SH::kWarp) __syncwarp();
    else __syncthreads();
}
template <class SH> __device__ __forceinline__ int gsync_or(int v) {
    if constexpr (SH::kWarp) return __any_sync(0xffffffffu, v);
    else return __syncthreads_or(v);
}

template <class SH>
__device__ __forceinline__ void rel_vec(const SH &S, const Params &P, int i, int j, float d[3]) {
    for (int a = 0; a < 3; a++)
        d[a] = minimg_f(P, a, (S.xh[j][a] - S.xh[i][a]) + (S.xl[j][a] - S.xl[i][a]));
}

// M, grad M and Hessian (xx yy zz xy xz yz) of one metaball at y, control
// points at rc + off (weights in rc[].w), Eq. (4).  Two interleaved partial
// sums, so that consecutive control points do not wait on each other, and
// the approximate FP32 reciprocal (the contact geometry is FP32 throughout).
struct MbSum {
    float M, g0, g1, g2, h0, h1, h2, h3, h4, h5;
};
// the terms of one control point (position cp.xyz, weight cp.w) at y
__device__ __forceinline__ void mb_acc0(const float4 cp, const float y[3], MbSum &A) {
    const float r0 = y[0] - cp.x, r1 = y[1] - cp.y, r2_ = y[2] - cp.z;
    const float r2 = r0 * r0 + r1 * r1 + r2_ * r2_;
    const float ir = __fdividef(1.0f, r2);
    const float Kr = cp.w * ir;            // K / r^2
    const float a1 = -2.0f * Kr * ir;      // -2 K / r^4
    const float a2 = 8.0f * Kr * ir * ir;  // 8 K / r^6
    A.M += Kr;
    A.g0 = fmaf(a1, r0, A.g0);
    A.g1 = fmaf(a1, r1, A.g1);
    A.g2 = fmaf(a1, r2_, A.g2);
    A.h0 += fmaf(a2 * r0, r0, a1);
    A.h1 += fmaf(a2 * r1, r1, a1);
    A.h2 += fmaf(a2 * r2_, r2_, a1);
    A.h3 = fmaf(a2 * r0, r1, A.h3);
    A.h4 = fmaf(a2 * r0, r2_, A.h4);
    A.h5 = fmaf(a2 * r1, r2_, A.h5);
}
// ... of a control point at cp.xyz + off
__device__ __forceinline__ void mb_acc(const float4 cp, const float off[3], const float y[3], MbSum &A) {
    mb_acc0(make_float4(cp.x + off[0], cp.y + off[1], cp.z + off[2], cp.w), y, A);
}
__device__ __forceinline__ void mb_dd_f(const float4 *rc, int ncp, const float off[3], const float y[3], float &M,
                                        float g[3], float H[6]) {
    MbSum A = {}, B = {};
    int c = 0;
    for (; c + 1 < ncp; c += 2) {
        mb_acc(rc[c], off, y, A);
        mb_acc(rc[c + 1], off, y, B);
    }
    if (c < ncp) mb_acc(rc[c], off, y, A);
    M = A.M + B.M;
    g[0] = A.g0 + B.g0; g[1] = A.g1 + B.g1; g[2] = A.g2 + B.g2;
    H[0] = A.h0 + B.h0; H[1] = A.h1 + B.h1; H[2] = A.h2 + B.h2;
    H[3] = A.h3 + B.h3; H[4] = A.h4 + B.h4; H[5] = A.h5 + B.h5;
}

// Contact law of §2.1.1 (Eqs. (2)-(3)) in FP32; xi: tangential spring.
__device__ void contact_law_f(const Params &P, float delta, const float n[3], const float vij[3], float xi[3], float h,
                              float F[3]) {
    const float vn = dot3f(vij, n);
    float Fn = P.kn_f * delta - P.eta_n_f * vn;
    if (Fn < 0.f) Fn = 0.f;
    float vt[3];
    for (int a = 0; a < 3; a++) vt[a] = vij[a] - vn * n[a];
    const float xn = dot3f(xi, n);
    for (int a = 0; a < 3; a++) xi[a] = xi[a] - xn * n[a] + vt[a] * h;
    float Ft[3];
    for (int a = 0; a < 3; a++) Ft[a] = -P.kt_f * xi[a] - P.eta_t_f * vt[a];
    const float ft = sqrtf(dot3f(Ft, Ft));
    if (ft > P.mu_s_f * Fn) {
        const float sc = ft > 0.f ? P.mu_s_f * Fn * __frcp_rn(ft) : 0.f;
        for (int a = 0; a < 3; a++) {
            Ft[a] *= sc;
            xi[a] = -(Ft[a] + P.eta_t_f * vt[a]) * P.inv_kt_f;
        }
    }
    for (int a = 0; a < 3; a++) F[a] = Fn * n[a] + Ft[a];
}

// Newton stops when the step is below 1e-5 lu (FP32 resolution of these
// O(radius) coordinates is ~1e-6) or stops shrinking after a few steps.
constexpr int kNewtonMax = 30;
constexpr float kNewtonTol2 = 1e-10f;

// Pair geometry, Eqs. (5)-(9), in the frame centred on particle i (d = x_j -
// x_i).  Same steps as the FP64 path: Newton on grad(M_i + M_j) = 0, valid
// when c_tol < M < 1 for both, closest points by the first-order step, contact
// point in the middle of the overlap.
template <class SH>
__device__ bool pair_geom_f(const Params &P, const SH &S, int i, int j, const float d[3], bool warm, float xm[3],
                            float &delta, float nv[3], float xcp[3], bool &valid) {
    const float4 *rci = S.rc + S.cpo[i];
    const float4 *rcj = S.rc + S.cpo[j];
    const int nci = S.cpo[i + 1] - S.cpo[i], ncj = S.cpo[j + 1] - S.cpo[j];
    const float zero[3] = {0.f, 0.f, 0.f};
    float x[3];
    if (warm) {
        for (int a = 0; a < 3; a++) x[a] = xm[a];
    } else {
        float best = 3.4e38f;
        x[0] = x[1] = x[2] = 0.f;
        for (int a = 0; a < nci; a++)
            for (int b = 0; b < ncj; b++) {
                const float dd[3] = {(d[0] + rcj[b].x) - rci[a].x, (d[1] + rcj[b].y) - rci[a].y,
                                     (d[2] + rcj[b].z) - rci[a].z};
                const float d2 = dot3f(dd, dd);
                if (d2 < best) {
                    best = d2;
                    x[0] = rci[a].x + 0.5f * dd[0];
                    x[1] = rci[a].y + 0.5f * dd[1];
                    x[2] = rci[a].z + 0.5f * dd[2];
                }
            }
    }
    // M, grad M at the last iterate evaluated (xe): once the step is below
    // the tolerance the point moves by less than 1e-5 lu, and the closest
    // points of Eqs. (8)-(9) are taken there without another evaluation
    float M0, g0[3], H0[6], M1, g1[3], H1[6], xe[3];
    float prev = 3.4e38f;
    bool converged = false;
    valid = false;
    for (int it = 0;; it++) {
        mb_dd_f(rci, nci, zero, x, M0, g0, H0);
        mb_dd_f(rcj, ncj, d, x, M1, g1, H1);
        for (int a = 0; a < 3; a++) xe[a] = x[a];
        if (it == kNewtonMax) break;
        float H[6], g[3];
        for (int a = 0; a < 6; a++) H[a] = H0[a] + H1[a];
        for (int a = 0; a < 3; a++) g[a] = -(g0[a] + g1[a]);
        // symmetric 3x3 solve by cofactors
        const float c0 = H[1] * H[2] - H[5] * H[5];
        const float c1 = H[5] * H[4] - H[3] * H[2];
        const float c2 = H[3] * H[5] - H[1] * H[4];
        const float det = H[0] * c0 + H[3] * c1 + H[4] * c2;
        if (det == 0.f || !isfinite(det)) break;
        const float id = __frcp_rn(det);
        const float b11 = H[0] * H[2] - H[4] * H[4], b12 = H[4] * H[3] - H[0] * H[5];
        const float b22 = H[0] * H[1] - H[3] * H[3];
        float dx[3];
        dx[0] = (c0 * g[0] + c1 * g[1] + c2 * g[2]) * id;
        dx[1] = (c1 * g[0] + b11 * g[1] + b12 * g[2]) * id;
        dx[2] = (c2 * g[0] + b12 * g[1] + b22 * g[2]) * id;
        for (int a = 0; a < 3; a++) x[a] += dx[a];
        const float s2 = dot3f(dx, dx);
        if (s2 < kNewtonTol2) { converged = true; break; }
        if (it >= 3 && s2 >= prev) break;
        prev = s2;
    }
    for (int a = 0; a < 3; a++) xm[a] = x[a];
    if (!(M0 > P.c_tol_f && M0 < 1.0f && M1 > P.c_tol_f && M1 < 1.0f)) return false;
    valid = converged;
    const float q0 = (1.0f - M0) * __frcp_rn(dot3f(g0, g0)), q1 = (1.0f - M1) * __frcp_rn(dot3f(g1, g1));
    float dc[3];
    for (int a = 0; a < 3; a++) dc[a] = q0 * g0[a] - q1 * g1[a];
    const float dist = sqrtf(dot3f(dc, dc));
    delta = S.Rs[i] + S.Rs[j] - dist;
    if (!(delta > 0.f) || dist == 0.f) return false;
    const float idist = __frcp_rn(dist);
    for (int a = 0; a < 3; a++) {
        nv[a] = dc[a] * idist;
        xcp[a] = (xe[a] + q0 * g0[a]) - (S.Rs[i] - 0.5f * delta) * nv[a];
    }
    return true;
}

// Wall geometry, Eqs. (10)-(13), frame centred on the particle; prel: the
// wall plane's coordinate relative to x along its axis.
// The wall's axis is a template parameter, so that every index into x, g
// and H is a constant and they stay in registers.
template <int AX, class SH>
__device__ __forceinline__ bool wall_geom_f(const Params &P, const SH &S, int k, int side, float prel, bool warm, float xcw[3],
                            float &delta, float nv[3], float xcp[3], bool &valid) {
    constexpr int ax = AX, t1 = (AX + 1) % 3, t2 = (AX + 2) % 3;
    const float m_ax = side ? 1.0f : -1.0f;
    const float4 *rc = S.rc + S.cpo[k];
    const int nc = S.cpo[k + 1] - S.cpo[k];
    const float zero[3] = {0.f, 0.f, 0.f};
    float x[3];
    if (warm) {
        for (int a = 0; a < 3; a++) x[a] = xcw[a];
    } else {
        int kb = 0;
        float best = 3.4e38f;
        for (int c = 0; c < nc; c++) {
            const float pc = ax == 0 ? rc[c].x : (ax == 1 ? rc[c].y : rc[c].z);
            const float dd = fabsf(prel - pc);
            if (dd < best) { best = dd; kb = c; }
        }
        x[0] = rc[kb].x; x[1] = rc[kb].y; x[2] = rc[kb].z;
    }
    x[ax] = prel;
    // H index of (a, b)
    constexpr int i11 = t1, i22 = t2, i12 = t1 + t2 == 1 ? 3 : (t1 + t2 == 2 ? 4 : 5);
    float M, g[3], H[6], xe[3];  // the last evaluation, at xe (as for pairs)
    float prev = 3.4e38f;
    bool converged = false;
    valid = false;
    for (int it = 0;; it++) {
        mb_dd_f(rc, nc, zero, x, M, g, H);
        for (int a = 0; a < 3; a++) xe[a] = x[a];
        if (it == kNewtonMax) break;
        const float J00 = H[i11], J01 = H[i12], J11 = H[i22];
        const float det = J00 * J11 - J01 * J01;
        if (det == 0.f || !isfinite(det)) break;
        const float id = __frcp_rn(det);
        const float r0 = -g[t1], r1 = -g[t2];
        const float d0 = (J11 * r0 - J01 * r1) * id, d1 = (-J01 * r0 + J00 * r1) * id;
        x[t1] += d0;
        x[t2] += d1;
        const float s2 = d0 * d0 + d1 * d1;
        if (s2 < kNewtonTol2) { converged = true; break; }
        if (it >= 3 && s2 >= prev) break;
        prev = s2;
    }
    for (int a = 0; a < 3; a++) xcw[a] = x[a];
    if (!(g[ax] * m_ax < 0.f)) return false;
    valid = converged;
    const float qR = (1.0f - M) * __frcp_rn(dot3f(g, g));
    float dc[3];
    for (int a = 0; a < 3; a++) dc[a] = qR * g[a];
    const float dist = sqrtf(dot3f(dc, dc));
    delta = S.Rs[k] - dist;
    if (!(delta > 0.f) || dist == 0.f) return false;
    const float idist = __frcp_rn(dist);
    for (int a = 0; a < 3; a++) {
        nv[a] = dc[a] * idist;
        xcp[a] = xe[a] - 0.5f * delta * nv[a];
    }
    return true;
}

// Pair contact history of the candidate items to global memory (before the
// list is rebuilt, and at the end of the launch).
template <class SH>
__device__ void store_items(const Params &P, SH &S) {
    const int np = S.n;
    for (int i = gtid<SH>(); i < np; i += gdim<SH>())
        for (int s = 0; s < S.nup[i]; s++) {
            const int it = S.ioff[i] + s;
            if (it >= SH::kItems) break;
            const int pidx = S.gid[i] * P.np + S.gid[S.up[i][s]];
            P.pair_on[pidx] = S.it_on[it];
            for (int a = 0; a < 3; a++) {
                P.pair_xm_f[3 * pidx + a] = S.it_xm[it][a];
                P.pair_xi_f[3 * pidx + a] = S.it_xi[it][a];
            }
        }
}

// Candidate pairs: bounding spheres closer than the skin.  Pairs that drop
// out lose their contact history, as in the FP64 path.  Sets *possible when
// some pair is within reach of a contact this step (or one is active).
// Loads the candidates' contact history into shared memory.
template <class SH>
__device__ void build_lists(const Params &P, SH &S, int *possible) {
    const int np = S.n, tid = gtid<SH>(), nth = gdim<SH>();
    const int nw = (np + 31) / 32;
    for (int idx = tid; idx < np * nw; idx += nth) {
        const int i = idx / nw, wd = idx % nw;
        unsigned m = 0;
        const float bri = S.brad[i], ri = S.reach[i];
        for (int b = 0; b < 32; b++) {
            const int j = wd * 32 + b;
            if (j <= i || j >= np) continue;
            float d[3];
            rel_vec(S, P, i, j, d);
            const float d2 = dot3f(d, d);
            const float brs = bri + S.brad[j];
            const float lim = brs + kSkin;
            const int pidx = S.gid[i] * P.np + S.gid[j];
            const int fl = P.pair_on[pidx];
            const bool on = (fl & CONTACT_ON) != 0;
            if (d2 < lim * lim) {
                m |= 1u << b;
                const float lr = brs + ri + S.reach[j] + 1e-2f;
                if (on || d2 <= lr * lr) *possible = 1;
            } else if (fl) {
                P.pair_on[pidx] = 0;
                if (on) *possible = 1;
            }
        }
        S.bits[i][wd] = m;
    }
    for (int k = tid; k < np; k += nth) S.ndn[k] = 0;
    gsync<SH>();
    for (int i = tid; i < np; i += nth) {
        int n = 0;
        for (int wd = 0; wd < nw; wd++) {
            unsigned m = S.bits[i][wd];
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int j = wd * 32 + b;
                if (n < kMaxAdj) {
                    S.up[i][n] = (unsigned short)j;
                    const int pos = atomicAdd(&S.ndn[j], 1);
                    if (pos < kMaxAdj) S.dn[j][pos] = (i << 8) | n;
                    else atomicOr(&P.status[ST_ERR], ERRB_DEM_CAPACITY);
                    n++;
                } else {
                    atomicOr(&P.status[ST_ERR], ERRB_DEM_CAPACITY);
                }
            }
        }
        S.nup[i] = n;
    }
    gsync<SH>();
    for (int k = tid; k < np; k += nth) {
        const int n = min(S.ndn[k], kMaxAdj);
        S.ndn[k] = n;
        for (int a = 1; a < n; a++) {  // ascending m
            const int e = S.dn[k][a];
            int b = a - 1;
            while (b >= 0 && S.dn[k][b] > e) { S.dn[k][b + 1] = S.dn[k][b]; b--; }
            S.dn[k][b + 1] = e;
        }
        for (int a = 0; a < 3; a++) S.xref[k][a] = S.xh[k][a] + S.xl[k][a];
    }
    if (tid == 0) {
        int o = 0;
        for (int i = 0; i < np; i++) { S.ioff[i] = o; o += S.nup[i]; }
        S.ioff[np] = o;
        if (o > SH::kItems) atomicOr(&P.status[ST_ERR], ERRB_DEM_CAPACITY);
    }
    gsync<SH>();
    for (int i = tid; i < np; i += nth)
        for (int s = 0; s < S.nup[i]; s++) {
            const int it = S.ioff[i] + s;
            if (it >= SH::kItems) break;
            const int pidx = S.gid[i] * P.np + S.gid[S.up[i][s]];
            S.it_on[it] = P.pair_on[pidx];
            for (int a = 0; a < 3; a++) {
                S.it_xm[it][a] = P.pair_xm_f[3 * pidx + a];
                S.it_xi[it][a] = P.pair_xi_f[3 * pidx + a];
            }
        }
    gsync<SH>();
}

// Pair contacts of the candidate list (one item per thread); results into
// it_res (zeros when not in contact).
template <class SH>
__device__ void pair_contacts(const Params &P, SH &S, float h) {
    const int np = S.n;
    const int total = min(S.ioff[np], SH::kItems);
    for (int it = gtid<SH>(); it < total; it += gdim<SH>()) {
        int lo = 0, hi = np - 1;  // item -> (i, slot): last i with ioff[i] <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.ioff[mid] <= it) lo = mid; else hi = mid - 1;
        }
        const int i = lo, s = it - S.ioff[i], j = S.up[i][s];
        float d[3];
        rel_vec(S, P, i, j, d);
        const float brs = S.brad[i] + S.brad[j];
        float Fi[3] = {0.f, 0.f, 0.f}, ti[3] = {0.f, 0.f, 0.f}, tj[3] = {0.f, 0.f, 0.f};
        if (dot3f(d, d) > brs * brs) {
            S.it_on[it] = 0;
        } else {
            const int was = S.it_on[it];
            float xm[3] = {S.it_xm[it][0], S.it_xm[it][1], S.it_xm[it][2]}, delta, nv[3], xcp[3];
            bool valid;
            const bool hit = pair_geom_f(P, S, i, j, d, (was & CONTACT_WARM) != 0, xm, delta, nv, xcp, valid);
            for (int a = 0; a < 3; a++) S.it_xm[it][a] = xm[a];
            const int warm = valid ? CONTACT_WARM : 0;
            if (!hit) {
                S.it_on[it] = warm;
            } else {
                float xi[3];
                for (int a = 0; a < 3; a++) xi[a] = (was & CONTACT_ON) ? S.it_xi[it][a] : 0.f;
                S.it_on[it] = warm | CONTACT_ON;
                float rj[3], wri[3], wrj[3], vij[3];
                for (int a = 0; a < 3; a++) rj[a] = xcp[a] - d[a];
                cross3f(S.w[i], xcp, wri);
                cross3f(S.w[j], rj, wrj);
                for (int a = 0; a < 3; a++) vij[a] = (S.v[i][a] + wri[a]) - (S.v[j][a] + wrj[a]);
                contact_law_f(P, delta, nv, vij, xi, h, Fi);
                for (int a = 0; a < 3; a++) S.it_xi[it][a] = xi[a];
                const float Fj[3] = {-Fi[0], -Fi[1], -Fi[2]};
                cross3f(xcp, Fi, ti);
                cross3f(rj, Fj, tj);
            }
        }
        for (int a = 0; a < 3; a++) { S.it_res[it][a] = Fi[a]; S.it_res[it][3 + a] = ti[a]; S.it_res[it][6 + a] = tj[a]; }
    }
}

// Per particle: its pair terms, in index order.
template <class SH>
__device__ __forceinline__ void gather_pairs(const SH &S, int k, float F[3], float T[3]) {
    for (int a = 0; a < 3; a++) { F[a] = 0.f; T[a] = 0.f; }
    for (int e = 0; e < S.ndn[k]; e++) {
        const int m = S.dn[k][e] >> 8, s = S.dn[k][e] & 255;
        const int it = S.ioff[m] + s;
        if (it >= SH::kItems) continue;
        for (int a = 0; a < 3; a++) { F[a] += -S.it_res[it][a]; T[a] += S.it_res[it][6 + a]; }
    }
    for (int s = 0; s < S.nup[k]; s++) {
        const int it = S.ioff[k] + s;
        if (it >= SH::kItems) break;
        for (int a = 0; a < 3; a++) { F[a] += S.it_res[it][a]; T[a] += S.it_res[it][3 + a]; }
    }
}

// Per particle: pair terms in index order, then the walls.
template <class SH>
__device__ void gather_contacts(const Params &P, SH &S, int k, float h, float F[3], float T[3]) {
    gather_pairs(S, k, F, T);
    for (int wall = 0; wall < NWALL; wall++) {
        const int ax = wall / 2, side = wall % 2;
        if (P.per[ax]) { S.w_on[k][wall] = 0; continue; }
        const float plane = side ? P.dim_f[ax] - 0.5f : -0.5f;
        const float prel = (plane - S.xh[k][ax]) - S.xl[k][ax];
        if (fabsf(prel) > S.brad[k]) { S.w_on[k][wall] = 0; continue; }
        const int was = S.w_on[k][wall];
        float xcw[3] = {S.w_xcw[k][wall][0], S.w_xcw[k][wall][1], S.w_xcw[k][wall][2]}, delta, nv[3], xcp[3];
        bool valid;
        const bool start = (was & CONTACT_WARM) != 0;
        const bool hit = ax == 0   ? wall_geom_f<0>(P, S, k, side, prel, start, xcw, delta, nv, xcp, valid)
                         : ax == 1 ? wall_geom_f<1>(P, S, k, side, prel, start, xcw, delta, nv, xcp, valid)
                                   : wall_geom_f<2>(P, S, k, side, prel, start, xcw, delta, nv, xcp, valid);
        for (int a = 0; a < 3; a++) S.w_xcw[k][wall][a] = xcw[a];
        const int warm = valid ? CONTACT_WARM : 0;
        if (!hit) { S.w_on[k][wall] = warm; continue; }
        float xi[3];
        for (int a = 0; a < 3; a++) xi[a] = (was & CONTACT_ON) ? S.w_xi[k][wall][a] : 0.f;
        S.w_on[k][wall] = warm | CONTACT_ON;
        float wr[3], vi[3], Fi[3], ti[3];
        cross3f(S.w[k], xcp, wr);
        for (int a = 0; a < 3; a++) vi[a] = S.v[k][a] + wr[a];
        contact_law_f(P, delta, nv, vi, xi, h, Fi);
        for (int a = 0; a < 3; a++) S.w_xi[k][wall][a] = xi[a];
        cross3f(xcp, Fi, ti);
        for (int a = 0; a < 3; a++) { F[a] += Fi[a]; T[a] += ti[a]; }
    }
}

// Body-frame control points of particle k into the shared table (once per
// launch, by the thread that rotates them), where the tables have room.
template <class SH>
__device__ __forceinline__ void load_cpb(const Params &P, SH &S, int k) {
    if constexpr (SH::kCacheCpb) {
        const DevParticle &p = P.parts[S.gid[k]];
        const int o = S.cpo[k], nc = S.cpo[k + 1] - o;
        for (int c = 0; c < nc; c++) S.cpb[o + c] = make_float4(p.cpb_f[c][0], p.cpb_f[c][1], p.cpb_f[c][2], p.K_f[c]);
    }
}

// Rotated control points of particle k into the shared table.
template <class SH>
__device__ __forceinline__ void put_rc(const Params &P, SH &S, int k, const float q[4]) {
    const int o = S.cpo[k], nc = S.cpo[k + 1] - o;
    const DevParticle &p = P.parts[S.gid[k]];
    for (int c = 0; c < nc; c++) {
        const float4 b = SH::kCacheCpb ? S.cpb[o + c]
                                       : make_float4(p.cpb_f[c][0], p.cpb_f[c][1], p.cpb_f[c][2], p.K_f[c]);
        const float v[3] = {b.x, b.y, b.z};
        float r[3];
        qrot_f(q, v, r, true);
        S.rc[o + c] = make_float4(r[0], r[1], r[2], b.w);
    }
}

}  // namespace

__global__ void __launch_bounds__(kThreads) k_dem32(Params P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared &S = *reinterpret_cast<Shared *>(smem_raw);
    const int tid = threadIdx.x, np = P.np;
    const float h = P.h_f, hh = 0.5f * h, qh2 = 0.25f * h * h;
    const bool own = tid < np;
    const DevParticle *pp = own ? &P.parts[tid] : nullptr;

    DF x[3], v[3], q[4], wb[3];
    float Fh[3] = {0.f, 0.f, 0.f}, Th[3] = {0.f, 0.f, 0.f}, iI[3], cI[3], bg[3], inv_m = 0.f;
    bool mov = false;
    if (own) {
        for (int a = 0; a < 3; a++) {
            x[a] = df_load(pp->sx[a]);
            v[a] = df_load(pp->sv[a]);
            wb[a] = df_load(pp->swb[a]);
            // the near sweep's fixed-point totals (2^-40 units)
            Fh[a] = (float)(long long)P.Ffix[6 * tid + a] * (1.0f / (float)(1ull << kForceFixBits));
            Th[a] = (float)(long long)P.Ffix[6 * tid + 3 + a] * (1.0f / (float)(1ull << kForceFixBits));
            iI[a] = pp->iI_f[a];
            cI[a] = pp->cI_f[a];
            bg[a] = pp->bg_f[a];
        }
        for (int a = 0; a < 4; a++) q[a] = df_load(pp->sq[a]);
        inv_m = pp->inv_mass_f;
        mov = !pp->fixed;
    }
    if (tid == 0) {
        int o = 0;
        for (int k = 0; k < np; k++) { S.cpo[k] = o; o += P.parts[k].ncp; }
        S.cpo[np] = o;
        S.n = np;
    }
    for (int k = tid; k < np; k += blockDim.x) S.gid[k] = k;
    __syncthreads();

    // shared state, reach over the step without contacts (|v| + |a|), walls
    int possible = 0;
    if (own) {
        float qf[4] = {q[0].hi, q[1].hi, q[2].hi, q[3].hi}, wbf[3] = {wb[0].hi, wb[1].hi, wb[2].hi}, ww[3];
        qrot_f(qf, wbf, ww, true);
        float a2 = 0.f, v2 = 0.f;
        for (int a = 0; a < 3; a++) {
            S.xh[tid][a] = x[a].hi;
            S.xl[tid][a] = x[a].lo;
            S.v[tid][a] = v[a].hi;
            S.w[tid][a] = ww[a];
            const float acc = bg[a] + Fh[a] * inv_m;
            a2 += acc * acc;
            v2 += v[a].hi * v[a].hi;
        }
        const float reach = mov ? (sqrtf(v2) + sqrtf(a2)) * 1.001f + 1e-4f : 0.f;
        S.reach[tid] = reach;
        S.brad[tid] = pp->brad_f;
        S.Rs[tid] = pp->Rs_f;
        if (reach > 0.4f * kSkin) possible = 1;
        load_cpb(P, S, tid);
        put_rc(P, S, tid, qf);
        for (int wall = 0; wall < NWALL; wall++) {
            const int ax = wall / 2, side = wall % 2;
            const int wj = tid * NWALL + wall;
            S.w_on[tid][wall] = P.wall_on[wj];
            for (int a = 0; a < 3; a++) {
                S.w_xcw[tid][wall][a] = P.wall_xcw_f[3 * wj + a];
                S.w_xi[tid][wall][a] = P.wall_xi_f[3 * wj + a];
            }
            if (P.wall_on[wj] & CONTACT_ON) possible = 1;
            if (P.per[ax]) continue;
            const float plane = side ? P.dim_f[ax] - 0.5f : -0.5f;
            const float prel = (plane - x[ax].hi) - x[ax].lo;
            if (fabsf(prel) - pp->brad_f <= reach + 1e-2f) possible = 1;
        }
    }
    __syncthreads();
    if (np > 1) build_lists(P, S, &possible);
    else if (tid == 0) {
        S.nup[0] = 0; S.ndn[0] = 0; S.ioff[0] = 0; S.ioff[1] = 0;
        for (int a = 0; a < 3; a++) S.xref[0][a] = S.xh[0][a] + S.xl[0][a];
    }
    possible = __syncthreads_or(possible);

    if (!possible) {
        // translation in closed form over the unit step (what the sub-steps
        // give in exact arithmetic), rotation sub-stepped
        if (own) {
            for (int a = 0; a < 3; a++) {
                const float acc = bg[a] + Fh[a] * inv_m;
                x[a] = df_add(df_add(x[a], v[a].hi), v[a].lo + 0.5f * acc);
                v[a] = df_add(v[a], acc);
            }
            bool turns = mov;
            if (turns) {
                float qf[4] = {q[0].hi, q[1].hi, q[2].hi, q[3].hi};
                float Tb[3];
                qrot_f(qf, Th, Tb, false);
                turns = !(wb[0].hi == 0.f && wb[1].hi == 0.f && wb[2].hi == 0.f && Tb[0] == 0.f && Tb[1] == 0.f &&
                          Tb[2] == 0.f);
                for (int sub = 0; turns && sub < P.n_sub; sub++) {
                    float wbf[3] = {wb[0].hi, wb[1].hi, wb[2].hi}, dw[3];
                    euler_f(iI, cI, wbf, Tb, dw);
                    DF wh[3];
                    float xf[3];
                    for (int a = 0; a < 3; a++) {
                        xf[a] = df_lead(wb[a], hh * dw[a]);
                        wh[a] = df_add(wb[a], hh * dw[a]);
                    }
                    float cm1, sc;
                    exp_half(hh, qh2, xf, cm1, sc);
                    const float d1 = sc * xf[0], d2 = sc * xf[1], d3 = sc * xf[2];
                    const float q0 = q[0].hi, q1 = q[1].hi, q2 = q[2].hi, q3 = q[3].hi;
                    const float i0 = q0 * cm1 - (q1 * d1 + q2 * d2 + q3 * d3);
                    const float i1 = q0 * d1 + q1 * cm1 + (q2 * d3 - q3 * d2);
                    const float i2 = q0 * d2 + q2 * cm1 + (q3 * d1 - q1 * d3);
                    const float i3 = q0 * d3 + q3 * cm1 + (q1 * d2 - q2 * d1);
                    qf[0] = df_lead(q[0], i0); qf[1] = df_lead(q[1], i1); qf[2] = df_lead(q[2], i2); qf[3] = df_lead(q[3], i3);
                    q[0] = df_add(q[0], i0); q[1] = df_add(q[1], i1); q[2] = df_add(q[2], i2); q[3] = df_add(q[3], i3);
                    qrot_f(qf, Th, Tb, false);
                    float w1[3] = {xf[0], xf[1], xf[2]};
                    for (int it = 0; it + 1 < ROT_ITERS; it++) {
                        euler_f(iI, cI, w1, Tb, dw);
                        for (int a = 0; a < 3; a++) w1[a] = xf[a] + hh * dw[a];
                    }
                    euler_f(iI, cI, w1, Tb, dw);
                    for (int a = 0; a < 3; a++) wb[a] = df_add(wh[a], hh * dw[a]);
                }
            }
            for (int a = 0; a < 3; a++) { S.Fc[tid][a] = 0.f; S.Tc[tid][a] = 0.f; }
        }
    } else {
        // contact load at the start: left by the previous step's DEM (same
        // state), unless the particles were set since
        if (!P.fc_valid) {
            pair_contacts(P, S, 0.f);
            __syncthreads();
            if (own) {
                float F[3], T[3];
                gather_contacts(P, S, tid, 0.f, F, T);
                for (int a = 0; a < 3; a++) { S.Fc[tid][a] = F[a]; S.Tc[tid][a] = T[a]; }
            }
        } else if (own) {
            for (int a = 0; a < 3; a++) {
                S.Fc[tid][a] = (float)P.Fc[3 * tid + a];
                S.Tc[tid][a] = (float)P.Tc[3 * tid + a];
            }
        }
        __syncthreads();
        for (int sub = 0; sub < P.n_sub; sub++) {
            DF wh[3];
            float whf[3] = {0.f, 0.f, 0.f};
            int moved = 0;
            if (own) {
                float qf[4] = {q[0].hi, q[1].hi, q[2].hi, q[3].hi};
                if (mov) {
                    // first half-kick and drift
                    for (int a = 0; a < 3; a++) {
                        const float acc = bg[a] + (Fh[a] + S.Fc[tid][a]) * inv_m;
                        const float vl = df_lead(v[a], hh * acc);
                        v[a] = df_add(v[a], hh * acc);
                        x[a] = df_add(x[a], h * vl);
                    }
                    // rotation: half-kick, q <- q (x) exp(h wh / 2)
                    float Tw[3], Tb[3], wbf[3] = {wb[0].hi, wb[1].hi, wb[2].hi}, dw[3];
                    for (int a = 0; a < 3; a++) Tw[a] = Th[a] + S.Tc[tid][a];
                    qrot_f(qf, Tw, Tb, false);
                    euler_f(iI, cI, wbf, Tb, dw);
                    for (int a = 0; a < 3; a++) {
                        whf[a] = df_lead(wb[a], hh * dw[a]);
                        wh[a] = df_add(wb[a], hh * dw[a]);
                    }
                    float cm1, sc;
                    exp_half(hh, qh2, whf, cm1, sc);
                    const float d1 = sc * whf[0], d2 = sc * whf[1], d3 = sc * whf[2];
                    const float q0 = qf[0], q1 = qf[1], q2 = qf[2], q3 = qf[3];
                    const float i0 = q0 * cm1 - (q1 * d1 + q2 * d2 + q3 * d3);
                    const float i1 = q0 * d1 + q1 * cm1 + (q2 * d3 - q3 * d2);
                    const float i2 = q0 * d2 + q2 * cm1 + (q3 * d1 - q1 * d3);
                    const float i3 = q0 * d3 + q3 * cm1 + (q1 * d2 - q2 * d1);
                    qf[0] = df_lead(q[0], i0); qf[1] = df_lead(q[1], i1); qf[2] = df_lead(q[2], i2); qf[3] = df_lead(q[3], i3);
                    q[0] = df_add(q[0], i0); q[1] = df_add(q[1], i1); q[2] = df_add(q[2], i2); q[3] = df_add(q[3], i3);
                } else {
                    for (int a = 0; a < 3; a++) { wh[a] = wb[a]; whf[a] = wb[a].hi; }
                }
                float ww[3];
                qrot_f(qf, whf, ww, true);
                float dr2 = 0.f;
                for (int a = 0; a < 3; a++) {
                    S.xh[tid][a] = x[a].hi;
                    S.xl[tid][a] = x[a].lo;
                    S.v[tid][a] = v[a].hi;
                    S.w[tid][a] = ww[a];
                    const float dd = (x[a].hi - S.xref[tid][a]) + x[a].lo;
                    dr2 += dd * dd;
                }
                if (mov) put_rc(P, S, tid, qf);
                moved = dr2 > 0.25f * kSkin * kSkin;
            }
            moved = __syncthreads_or(moved);
            if (moved && np > 1) {
                store_items(P, S);
                __syncthreads();
                int dummy = 0;
                build_lists(P, S, &dummy);
            }
            pair_contacts(P, S, h);
            __syncthreads();
            if (own) {
                float F[3], T[3];
                gather_contacts(P, S, tid, h, F, T);
                for (int a = 0; a < 3; a++) { S.Fc[tid][a] = F[a]; S.Tc[tid][a] = T[a]; }
                if (mov) {
                    // closing half-kick with the new contact load
                    for (int a = 0; a < 3; a++) v[a] = df_add(v[a], hh * (bg[a] + (Fh[a] + F[a]) * inv_m));
                    float qf[4] = {q[0].hi, q[1].hi, q[2].hi, q[3].hi}, Tw[3], Tb[3], dw[3];
                    for (int a = 0; a < 3; a++) Tw[a] = Th[a] + T[a];
                    qrot_f(qf, Tw, Tb, false);
                    float w1[3] = {whf[0], whf[1], whf[2]};
                    for (int it = 0; it + 1 < ROT_ITERS; it++) {
                        euler_f(iI, cI, w1, Tb, dw);
                        for (int a = 0; a < 3; a++) w1[a] = whf[a] + hh * dw[a];
                    }
                    euler_f(iI, cI, w1, Tb, dw);
                    for (int a = 0; a < 3; a++) wb[a] = df_add(wh[a], hh * dw[a]);
                }
            }
            __syncthreads();
        }
        // contact load of the end state (springs not advanced): reported by
        // lbm_get_contact_forces and the start load of the next step
        if (own) {
            float qf[4] = {q[0].hi, q[1].hi, q[2].hi, q[3].hi}, wbf[3] = {wb[0].hi, wb[1].hi, wb[2].hi}, ww[3];
            qrot_f(qf, wbf, ww, true);
            for (int a = 0; a < 3; a++) { S.v[tid][a] = v[a].hi; S.w[tid][a] = ww[a]; }
        }
        __syncthreads();
        pair_contacts(P, S, 0.f);
        __syncthreads();
        if (own) {
            float F[3], T[3];
            gather_contacts(P, S, tid, 0.f, F, T);
            for (int a = 0; a < 3; a++) { S.Fc[tid][a] = F[a]; S.Tc[tid][a] = T[a]; }
            // wall contact history back to global memory
            for (int wall = 0; wall < NWALL; wall++) {
                const int wj = tid * NWALL + wall;
                P.wall_on[wj] = S.w_on[tid][wall];
                for (int a = 0; a < 3; a++) {
                    P.wall_xcw_f[3 * wj + a] = S.w_xcw[tid][wall][a];
                    P.wall_xi_f[3 * wj + a] = S.w_xi[tid][wall][a];
                }
            }
        }
        if (np > 1) store_items(P, S);
    }

    // Write back: the compensated state, then the FP64 fields the other
    // kernels read.  q is renormalised to first order (|q|^2 - 1 is ~1e-12):
    // q <- q (1 - e/2), e = |q|^2 - 1 from exact products and a compensated sum.
    if (own) {
        DevParticle &p = P.parts[tid];
        float e_hi = -1.0f, e_lo = 0.f;
        for (int a = 0; a < 4; a++) {
            const float pr = q[a].hi * q[a].hi;
            const float er = fmaf(q[a].hi, q[a].hi, -pr) + 2.0f * q[a].hi * q[a].lo;
            const DF t = df_add({e_hi, e_lo}, pr);
            e_hi = t.hi;
            e_lo = t.lo + er;
        }
        const float e = e_hi + e_lo;
        for (int a = 0; a < 4; a++) {
            const DF t = df_add({q[a].hi, 0.f}, q[a].lo - 0.5f * e * q[a].hi);
            q[a] = t;
        }
        for (int a = 0; a < 3; a++) {
            df_store(p.sx[a], x[a]);
            df_store(p.sv[a], v[a]);
            df_store(p.swb[a], wb[a]);
        }
        for (int a = 0; a < 4; a++) df_store(p.sq[a], q[a]);
        float qf[4] = {q[0].hi, q[1].hi, q[2].hi, q[3].hi}, wbf[3] = {wb[0].hi, wb[1].hi, wb[2].hi}, ww[3];
        qrot_f(qf, wbf, ww, true);
        for (int a = 0; a < 3; a++) S.w[tid][a] = ww[a];
    }
    __syncthreads();
    // FP64 fields, one lane per component: x(3) v(3) q(4) w(3) Fc(3) Tc(3)
    for (int idx = tid; idx < np * 19; idx += blockDim.x) {
        const int k = idx / 19, c = idx % 19;
        DevParticle &p = P.parts[k];
        if (c < 3) p.x[c] = (double)p.sx[c][0] + (double)p.sx[c][1];
        else if (c < 6) p.v[c - 3] = (double)p.sv[c - 3][0] + (double)p.sv[c - 3][1];
        else if (c < 10) p.q[c - 6] = (double)p.sq[c - 6][0] + (double)p.sq[c - 6][1];
        else if (c < 13) p.w[c - 10] = (double)S.w[k][c - 10];
        else if (c < 16) P.Fc[3 * k + c - 13] = (double)S.Fc[k][c - 13];
        else P.Tc[3 * k + c - 16] = (double)S.Tc[k][c - 16];
    }
}

// ---------------------------------------------------------------------------
// k_dem64c: the active particles of k_dem64_plan (those that can meet a wall
// or another particle during the step), one thread each, one CTA.  The
// rigid-body state (x, v, q and the principal-frame angular velocity) is
// FP64 and persists in FP64 from step to step; within the step each
// component carries its change since the step began as a compensated FP32
// pair (about 48 significant bits of a change of order |v| ~ 0.1 lu: ~1e-15
// absolute), and the change is added to the FP64 value at the end of the
// step.  The sub-step increments, the contact geometry (Eqs. (5)-(13)) and
// the contact law (Eqs. (2)-(3)) are computed in FP32, as in k_dem32, from
// FP32 working copies (positions for the geometry as hi + lo pairs of the
// FP64 value plus the change).  No FP64 or FP64<->FP32 conversion runs in
// the sub-step loop: on this GPU both occupy a sub-partition for 64 cycles
// or more per warp instruction.  The sub-step sequence is k_dem's: velocity
// Verlet in kick-drift-kick form, Euler's equations in the principal frame,
// q <- q (x) exp(h w/2), the closing rotational half-kick implicit by
// ROT_ITERS sweeps.  The quaternion is renormalised once, at the end of the
// step.
// ---------------------------------------------------------------------------
// One state component within the step: the FP32 rounding of its value at
// the start (the FP64 value stays in the particle record until the end) and
// the change since then.
struct Delta {
    float bf;
    DF d;
    __device__ __forceinline__ float f() const { return bf + d.hi; }  // FP32 working value
    __device__ __forceinline__ double fin(double base) const { return base + ((double)d.hi + (double)d.lo); }
};
__device__ __forceinline__ void dl_set(Delta &a, double v) { a.bf = (float)v; a.d = {0.f, 0.f}; }
__device__ __forceinline__ void dl_add(Delta &a, float b) { a.d = df_add(a.d, b); }

// The contact groups of k_dem64_plan with more than kTinyContactGroup
// particles (the smaller ones: k_dem64t below): up to 32 one 32-thread CTA
// each, larger ones one 512-thread CTA each with the full tables; a thread
// per particle.
template <class SH, int kClass>
__global__ void __launch_bounds__(kClass == DEM_GROUP_LARGE ? kThreads : kSmallContactGroup, 1) k_dem64c(Params P) {
    static_assert(kClass != DEM_GROUP_TINY && !SH::kWarp, "groups of up to kTinyContactGroup: k_dem64t");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH &S = *reinterpret_cast<SH *>(smem_raw);
    const int tid = (int)threadIdx.x;
    const int slot = (int)blockIdx.x;
    if (slot >= P.dem_list[2 + kClass]) return;  // the whole CTA
    const int *grp = dem_groups(P, kClass) + 2 * slot;
    const int na = grp[1];
    const int *act = dem_active(P) + grp[0];
    const float h = P.h_f, hh = 0.5f * h, qh2 = 0.25f * h * h;
    const bool own = tid < na;
    const int g = own ? act[tid] : 0;
    DevParticle *pp = own ? &P.parts[g] : nullptr;

    Delta x[3], v[3], q[4], wb[3];
    float xlo[3] = {0.f, 0.f, 0.f};  // FP32 rounding error of the start position
    float Fh[3] = {0.f, 0.f, 0.f}, Th[3] = {0.f, 0.f, 0.f}, iI[3], cI[3], bg[3], inv_m = 0.f;
    bool mov = false;
    float reach = 0.f;
    if (own) {
        double wbd[3];
        rot_body(pp->q, pp->w, wbd);
        for (int a = 0; a < 3; a++) {
            dl_set(x[a], pp->x[a]);
            xlo[a] = (float)(pp->x[a] - (double)x[a].bf);
            dl_set(v[a], pp->v[a]);
            dl_set(wb[a], wbd[a]);
            Fh[a] = (float)P.Fh[3 * g + a];
            Th[a] = (float)P.Th[3 * g + a];
            iI[a] = pp->iI_f[a];
            cI[a] = pp->cI_f[a];
            bg[a] = pp->bg_f[a];
        }
        for (int a = 0; a < 4; a++) dl_set(q[a], pp->q[a]);
        inv_m = pp->inv_mass_f;
        mov = !pp->fixed;
        reach = dem_reach(P, *pp, g);
    }
    if (tid == 0) {
        int o = 0;
        for (int k = 0; k < na; k++) { S.cpo[k] = o; o += P.parts[act[k]].ncp; }
        S.cpo[na] = o;
        S.n = na;
        if (o > SH::kCps) atomicOr(&P.status[ST_ERR], ERRB_DEM_CAPACITY);
    }
    for (int k = tid; k < na; k += gdim<SH>()) S.gid[k] = act[k];
    gsync<SH>();
    if (S.cpo[na] > SH::kCps) return;

    // FP32 tables: position (hi + lo of the FP64 value), velocity, world
    // angular velocity from the body rate wf
    auto publish = [&](const float wf[3], const float qf[4]) {
        float ww[3];
        qrot_f(qf, wf, ww, true);
        for (int a = 0; a < 3; a++) {
            S.xh[tid][a] = x[a].bf;
            S.xl[tid][a] = xlo[a] + (x[a].d.hi + x[a].d.lo);
            S.v[tid][a] = v[a].f();
            S.w[tid][a] = ww[a];
        }
    };
    if (own) {
        const float qf[4] = {q[0].f(), q[1].f(), q[2].f(), q[3].f()}, wf[3] = {wb[0].f(), wb[1].f(), wb[2].f()};
        publish(wf, qf);
        S.reach[tid] = reach;
        S.brad[tid] = pp->brad_f;
        S.Rs[tid] = pp->Rs_f;
        load_cpb(P, S, tid);
        put_rc(P, S, tid, qf);
        for (int wall = 0; wall < NWALL; wall++) {
            const int wj = g * NWALL + wall;
            S.w_on[tid][wall] = P.wall_on[wj];
            for (int a = 0; a < 3; a++) {
                S.w_xcw[tid][wall][a] = P.wall_xcw_f[3 * wj + a];
                S.w_xi[tid][wall][a] = P.wall_xi_f[3 * wj + a];
            }
        }
    }
    gsync<SH>();
    int dummy = 0;
    if (na > 1) build_lists(P, S, &dummy);
    else if (tid == 0) {
        S.nup[0] = 0; S.ndn[0] = 0; S.ioff[0] = 0; S.ioff[1] = 0;
        for (int a = 0; a < 3; a++) S.xref[0][a] = S.xh[0][a] + S.xl[0][a];
    }
    gsync<SH>();
    // contact load at the start: left by the previous step's DEM (same
    // state), unless the particles were set since
    if (!P.fc_valid) {
        pair_contacts(P, S, 0.f);
        gsync<SH>();
        if (own) {
            float F[3], T[3];
            gather_contacts(P, S, tid, 0.f, F, T);
            for (int a = 0; a < 3; a++) { S.Fc[tid][a] = F[a]; S.Tc[tid][a] = T[a]; }
        }
    } else if (own) {
        for (int a = 0; a < 3; a++) {
            S.Fc[tid][a] = (float)P.Fc[3 * g + a];
            S.Tc[tid][a] = (float)P.Tc[3 * g + a];
        }
    }
    gsync<SH>();
    for (int sub = 0; sub < P.n_sub; sub++) {
        Delta wh[3] = {wb[0], wb[1], wb[2]};
        int moved = 0;
        if (own) {
            float qf[4] = {q[0].f(), q[1].f(), q[2].f(), q[3].f()};
            if (mov) {
                // first half-kick and drift
                for (int a = 0; a < 3; a++) {
                    dl_add(v[a], hh * (bg[a] + (Fh[a] + S.Fc[tid][a]) * inv_m));
                    dl_add(x[a], h * v[a].f());
                }
                // rotation: half-kick, q <- q (x) exp(h wh / 2)
                float Tw[3], Tb[3], wf[3] = {wb[0].f(), wb[1].f(), wb[2].f()}, dw[3], whf[3];
                for (int a = 0; a < 3; a++) Tw[a] = Th[a] + S.Tc[tid][a];
                qrot_f(qf, Tw, Tb, false);
                euler_f(iI, cI, wf, Tb, dw);
                for (int a = 0; a < 3; a++) {
                    dl_add(wh[a], hh * dw[a]);
                    whf[a] = wh[a].f();
                }
                float cm1, sc;
                exp_half(hh, qh2, whf, cm1, sc);
                const float d1 = sc * whf[0], d2 = sc * whf[1], d3 = sc * whf[2];
                const float q0 = qf[0], q1 = qf[1], q2 = qf[2], q3 = qf[3];
                dl_add(q[0], q0 * cm1 - (q1 * d1 + q2 * d2 + q3 * d3));
                dl_add(q[1], q0 * d1 + q1 * cm1 + (q2 * d3 - q3 * d2));
                dl_add(q[2], q0 * d2 + q2 * cm1 + (q3 * d1 - q1 * d3));
                dl_add(q[3], q0 * d3 + q3 * cm1 + (q1 * d2 - q2 * d1));
                for (int a = 0; a < 4; a++) qf[a] = q[a].f();
            }
            const float whf[3] = {wh[0].f(), wh[1].f(), wh[2].f()};
            publish(whf, qf);
            float dr2 = 0.f;
            for (int a = 0; a < 3; a++) {
                const float dd = (S.xh[tid][a] - S.xref[tid][a]) + S.xl[tid][a];
                dr2 += dd * dd;
            }
            if (mov) put_rc(P, S, tid, qf);
            moved = dr2 > 0.25f * kSkin * kSkin;
        }
        moved = gsync_or<SH>(moved);
        if (moved && na > 1) {
            store_items(P, S);
            gsync<SH>();
            build_lists(P, S, &dummy);
        }
        pair_contacts(P, S, h);
        gsync<SH>();
        if (own) {
            float F[3], T[3];
            gather_contacts(P, S, tid, h, F, T);
            for (int a = 0; a < 3; a++) { S.Fc[tid][a] = F[a]; S.Tc[tid][a] = T[a]; }
            if (mov) {
                // closing half-kick with the new contact load
                for (int a = 0; a < 3; a++) dl_add(v[a], hh * (bg[a] + (Fh[a] + F[a]) * inv_m));
                const float qf[4] = {q[0].f(), q[1].f(), q[2].f(), q[3].f()};
                float Tw[3], Tb[3], dw[3], whf[3] = {wh[0].f(), wh[1].f(), wh[2].f()}, w1[3];
                for (int a = 0; a < 3; a++) { Tw[a] = Th[a] + T[a]; w1[a] = whf[a]; }
                qrot_f(qf, Tw, Tb, false);
                for (int it = 0; it + 1 < ROT_ITERS; it++) {
                    euler_f(iI, cI, w1, Tb, dw);
                    for (int a = 0; a < 3; a++) w1[a] = whf[a] + hh * dw[a];
                }
                euler_f(iI, cI, w1, Tb, dw);
                for (int a = 0; a < 3; a++) {
                    wb[a] = wh[a];
                    dl_add(wb[a], hh * dw[a]);
                }
            }
        }
        gsync<SH>();
    }
    // the step's changes added to the FP64 state (still in the record)
    double qd[4] = {1, 0, 0, 0}, wbd[3] = {0, 0, 0}, xd[3] = {0, 0, 0}, vd[3] = {0, 0, 0};
    if (own && mov) {
        double wb0[3];
        rot_body(pp->q, pp->w, wb0);
        for (int a = 0; a < 4; a++) qd[a] = q[a].fin(pp->q[a]);
        for (int a = 0; a < 3; a++) {
            wbd[a] = wb[a].fin(wb0[a]);
            xd[a] = x[a].fin(pp->x[a]);
            vd[a] = v[a].fin(pp->v[a]);
        }
        quat_normalize(qd);
        for (int a = 0; a < 4; a++) dl_set(q[a], qd[a]);
    }
    // contact load of the end state (springs not advanced): reported by
    // lbm_get_contact_forces and the start load of the next step
    if (own) {
        const float qf[4] = {q[0].f(), q[1].f(), q[2].f(), q[3].f()}, wf[3] = {wb[0].f(), wb[1].f(), wb[2].f()};
        publish(wf, qf);
        if (mov) put_rc(P, S, tid, qf);
    }
    gsync<SH>();
    pair_contacts(P, S, 0.f);
    gsync<SH>();
    if (own) {
        float F[3], T[3];
        gather_contacts(P, S, tid, 0.f, F, T);
        for (int wall = 0; wall < NWALL; wall++) {
            const int wj = g * NWALL + wall;
            P.wall_on[wj] = S.w_on[tid][wall];
            for (int a = 0; a < 3; a++) {
                P.wall_xcw_f[3 * wj + a] = S.w_xcw[tid][wall][a];
                P.wall_xi_f[3 * wj + a] = S.w_xi[tid][wall][a];
            }
        }
        for (int a = 0; a < 3; a++) {
            P.Fc[3 * g + a] = (double)F[a];
            P.Tc[3 * g + a] = (double)T[a];
        }
        if (mov) {
            double ww[3];
            rot_world(qd, wbd, ww);
            for (int a = 0; a < 3; a++) {
                pp->x[a] = xd[a];
                pp->v[a] = vd[a];
                pp->w[a] = ww[a];
            }
            for (int a = 0; a < 4; a++) pp->q[a] = qd[a];
        }
        // the planning assumed no larger displacement (contacts with
        // inactive particles would have been missed otherwise)
        float d2 = 0.f;
        for (int a = 0; a < 3; a++) d2 += x[a].d.hi * x[a].d.hi;
        if (d2 > reach * reach) atomicOr(&P.status[ST_ERR], ERRB_DEM_REACH);
    }
    if (na > 1) store_items(P, S);
}

// ---------------------------------------------------------------------------
// Contact groups of up to four particles, one warp each (k_dem64t).  Lane
// kSegLanes * k + c works for particle k of the group (for k past the group's
// size: particle k mod size, as a mirror): the particle's lanes all hold its
// state (they integrate it from the same inputs in the same order, so they
// hold the same bits) and lane c holds its control points c and
// c + kSegLanes (a lane without one holds a point far away with weight zero,
// whose terms are exact zeros).  The metaball sums of a wall contact run over
// the particle's lanes and those of a pair contact over the whole warp
// (sixteen lanes per metaball), each reduced by an xor butterfly, after which
// every lane of the group holds the same sums; the Newton steps' decisions
// are still taken from the group's first lane, so that the lanes of a group
// stay together through every exchange.  Since every lane that writes a
// table entry writes the same bits there, the stores need no lane test (and
// the warp no branch around them); only the particles' own lanes write to
// global memory.
// ---------------------------------------------------------------------------
namespace {
constexpr int kSegLanes = 32 / kTinyContactGroup;  // lanes per particle
static_assert(2 * kSegLanes >= MAXCP, "two control points per lane of a particle");
static_assert(16 >= MAXCP, "one control point per lane in a pair solve");
constexpr unsigned kFullWarp = 0xffffffffu;
// stand-in for a missing control point: its terms vanish (K = 0) and r^2 stays
// far from zero
__device__ __forceinline__ float4 far_cp() { return make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f); }

// Butterfly sum of the metaball terms over groups of W lanes.
template <int W>
__device__ __forceinline__ void mb_bfly(MbSum &A, unsigned mask) {
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        A.M += __shfl_xor_sync(mask, A.M, o, W);
        A.g0 += __shfl_xor_sync(mask, A.g0, o, W);
        A.g1 += __shfl_xor_sync(mask, A.g1, o, W);
        A.g2 += __shfl_xor_sync(mask, A.g2, o, W);
        A.h0 += __shfl_xor_sync(mask, A.h0, o, W);
        A.h1 += __shfl_xor_sync(mask, A.h1, o, W);
        A.h2 += __shfl_xor_sync(mask, A.h2, o, W);
        A.h3 += __shfl_xor_sync(mask, A.h3, o, W);
        A.h4 += __shfl_xor_sync(mask, A.h4, o, W);
        A.h5 += __shfl_xor_sync(mask, A.h5, o, W);
    }
}
__device__ __forceinline__ void mb_unpack(const MbSum &A, float &M, float g[3], float H[6]) {
    M = A.M;
    g[0] = A.g0; g[1] = A.g1; g[2] = A.g2;
    H[0] = A.h0; H[1] = A.h1; H[2] = A.h2; H[3] = A.h3; H[4] = A.h4; H[5] = A.h5;
}

// Newton decision of one step, the same in every lane of a group: 1 singular
// Jacobian (stop before the step), 2 converged, 3 no longer shrinking, 0 go on.
__device__ __forceinline__ int newton_code(bool bad, float s2, float prev, int it) {
    return bad ? 1 : (s2 < kNewtonTol2 ? 2 : ((it >= 3 && s2 >= prev) ? 3 : 0));
}

// Wall geometry of Eqs. (10)-(13), the steps of wall_geom_f, run by the
// particle's lanes (mask); ca, cb: this lane's rotated control points.
template <int AX, class SH>
__device__ __forceinline__ bool wall_geom_seg(const Params &P, const SH &S, int k, int side, float prel, bool warm,
                                              float xcw[3], float &delta, float nv[3], float xcp[3], bool &valid,
                                              unsigned mask, const float4 ca, const float4 cb) {
    constexpr int ax = AX, t1 = (AX + 1) % 3, t2 = (AX + 2) % 3;
    const float m_ax = side ? 1.0f : -1.0f;
    float x[3];
    if (warm) {
        for (int a = 0; a < 3; a++) x[a] = xcw[a];
    } else {  // the control point nearest the plane (every lane scans the table)
        const float4 *rc = S.rc + S.cpo[k];
        const int nc = S.cpo[k + 1] - S.cpo[k];
        int kb = 0;
        float best = 3.4e38f;
        for (int c = 0; c < nc; c++) {
            const float pc = ax == 0 ? rc[c].x : (ax == 1 ? rc[c].y : rc[c].z);
            const float dd = fabsf(prel - pc);
            if (dd < best) { best = dd; kb = c; }
        }
        x[0] = rc[kb].x; x[1] = rc[kb].y; x[2] = rc[kb].z;
    }
    x[ax] = prel;
    constexpr int i11 = t1, i22 = t2, i12 = t1 + t2 == 1 ? 3 : (t1 + t2 == 2 ? 4 : 5);
    float M, g[3], H[6], xe[3];
    float prev = 3.4e38f;
    bool converged = false;
    valid = false;
    for (int it = 0;; it++) {
        MbSum A = {};
        mb_acc0(ca, x, A);
        mb_acc0(cb, x, A);
        mb_bfly<kSegLanes>(A, mask);
        mb_unpack(A, M, g, H);
        for (int a = 0; a < 3; a++) xe[a] = x[a];
        if (it == kNewtonMax) break;
        const float J00 = H[i11], J01 = H[i12], J11 = H[i22];
        const float det = J00 * J11 - J01 * J01;
        const float id = __frcp_rn(det);
        const float r0 = -g[t1], r1 = -g[t2];
        const float d0 = (J11 * r0 - J01 * r1) * id, d1 = (-J01 * r0 + J00 * r1) * id;
        const float s2 = d0 * d0 + d1 * d1;
        const int code = __shfl_sync(mask, newton_code(det == 0.f || !isfinite(det), s2, prev, it), 0, kSegLanes);
        if (code == 1) break;
        x[t1] += d0;
        x[t2] += d1;
        if (code == 2) { converged = true; break; }
        if (code == 3) break;
        prev = s2;
    }
    for (int a = 0; a < 3; a++) xcw[a] = x[a];
    if (!(g[ax] * m_ax < 0.f)) return false;
    valid = converged;
    const float qR = (1.0f - M) * __frcp_rn(dot3f(g, g));
    float dc[3];
    for (int a = 0; a < 3; a++) dc[a] = qR * g[a];
    const float dist = sqrtf(dot3f(dc, dc));
    delta = S.Rs[k] - dist;
    if (!(delta > 0.f) || dist == 0.f) return false;
    const float idist = __frcp_rn(dist);
    for (int a = 0; a < 3; a++) {
        nv[a] = dc[a] * idist;
        xcp[a] = xe[a] - 0.5f * delta * nv[a];
    }
    return true;
}

// The walls' terms of particle k added to F, T (after its pair terms), run by
// the particle's lanes (mask), which all write the contact history.
template <class SH>
__device__ void walls_seg(const Params &P, SH &S, int k, unsigned mask, float h, const float4 ca, const float4 cb,
                          float F[3], float T[3]) {
    for (int wall = 0; wall < NWALL; wall++) {
        const int ax = wall / 2, side = wall % 2;
        if (P.per[ax]) {
            S.w_on[k][wall] = 0;
            continue;
        }
        const float plane = side ? P.dim_f[ax] - 0.5f : -0.5f;
        const float prel = (plane - S.xh[k][ax]) - S.xl[k][ax];
        const int was = S.w_on[k][wall];
        float xcw[3], xi[3];
        for (int a = 0; a < 3; a++) {
            xcw[a] = S.w_xcw[k][wall][a];
            xi[a] = (was & CONTACT_ON) ? S.w_xi[k][wall][a] : 0.f;
        }
        const int go = __shfl_sync(mask, fabsf(prel) > S.brad[k] ? 0 : 1, 0, kSegLanes);
        if (!go) {
            __syncwarp(mask);
            S.w_on[k][wall] = 0;
            continue;
        }
        float delta, nv[3], xcp[3];
        bool valid;
        const bool start = (was & CONTACT_WARM) != 0;
        const bool hit =
            ax == 0   ? wall_geom_seg<0>(P, S, k, side, prel, start, xcw, delta, nv, xcp, valid, mask, ca, cb)
            : ax == 1 ? wall_geom_seg<1>(P, S, k, side, prel, start, xcw, delta, nv, xcp, valid, mask, ca, cb)
                      : wall_geom_seg<2>(P, S, k, side, prel, start, xcw, delta, nv, xcp, valid, mask, ca, cb);
        const int warm = valid ? CONTACT_WARM : 0;
        if (hit) {
            float wr[3], vi[3], Fi[3], ti[3];
            cross3f(S.w[k], xcp, wr);
            for (int a = 0; a < 3; a++) vi[a] = S.v[k][a] + wr[a];
            contact_law_f(P, delta, nv, vi, xi, h, Fi);
            cross3f(xcp, Fi, ti);
            for (int a = 0; a < 3; a++) { F[a] += Fi[a]; T[a] += ti[a]; }
        }
        __syncwarp(mask);
        for (int a = 0; a < 3; a++) S.w_xcw[k][wall][a] = xcw[a];
        S.w_on[k][wall] = hit ? (warm | CONTACT_ON) : warm;
        if (hit)
            for (int a = 0; a < 3; a++) S.w_xi[k][wall][a] = xi[a];
    }
}

// Pair geometry of Eqs. (5)-(9), the steps of pair_geom_f, run by the whole
// warp: lanes 0-15 hold the control points of particle i, lanes 16-31 those
// of particle j.
template <class SH>
__device__ bool pair_geom_w(const Params &P, const SH &S, int i, int j, const float d[3], bool warm, float xm[3],
                            float &delta, float nv[3], float xcp[3], bool &valid) {
    const int lane = threadIdx.x & 31, half = lane >> 4, cc = lane & 15;
    const int m = half ? j : i;
    const int ncm = S.cpo[m + 1] - S.cpo[m];
    const float4 cp = cc < ncm ? S.rc[S.cpo[m] + cc] : far_cp();
    const float off[3] = {half ? d[0] : 0.f, half ? d[1] : 0.f, half ? d[2] : 0.f};
    float x[3];
    if (warm) {
        for (int a = 0; a < 3; a++) x[a] = xm[a];
    } else {  // midpoint of the closest pair of control points (every lane scans the tables)
        const float4 *rci = S.rc + S.cpo[i];
        const float4 *rcj = S.rc + S.cpo[j];
        const int nci = S.cpo[i + 1] - S.cpo[i], ncj = S.cpo[j + 1] - S.cpo[j];
        float best = 3.4e38f;
        x[0] = x[1] = x[2] = 0.f;
        for (int a = 0; a < nci; a++)
            for (int b = 0; b < ncj; b++) {
                const float dd[3] = {(d[0] + rcj[b].x) - rci[a].x, (d[1] + rcj[b].y) - rci[a].y,
                                     (d[2] + rcj[b].z) - rci[a].z};
                const float d2 = dot3f(dd, dd);
                if (d2 < best) {
                    best = d2;
                    x[0] = rci[a].x + 0.5f * dd[0];
                    x[1] = rci[a].y + 0.5f * dd[1];
                    x[2] = rci[a].z + 0.5f * dd[2];
                }
            }
    }
    float M0, g0[3], H0[6], M1, g1[3], H1[6], xe[3];
    float prev = 3.4e38f;
    bool converged = false;
    valid = false;
    for (int it = 0;; it++) {
        MbSum A = {};
        mb_acc(cp, off, x, A);
        mb_bfly<16>(A, kFullWarp);
        MbSum B;  // the other particle's sums
        B.M = __shfl_xor_sync(kFullWarp, A.M, 16);
        B.g0 = __shfl_xor_sync(kFullWarp, A.g0, 16);
        B.g1 = __shfl_xor_sync(kFullWarp, A.g1, 16);
        B.g2 = __shfl_xor_sync(kFullWarp, A.g2, 16);
        B.h0 = __shfl_xor_sync(kFullWarp, A.h0, 16);
        B.h1 = __shfl_xor_sync(kFullWarp, A.h1, 16);
        B.h2 = __shfl_xor_sync(kFullWarp, A.h2, 16);
        B.h3 = __shfl_xor_sync(kFullWarp, A.h3, 16);
        B.h4 = __shfl_xor_sync(kFullWarp, A.h4, 16);
        B.h5 = __shfl_xor_sync(kFullWarp, A.h5, 16);
        mb_unpack(half ? B : A, M0, g0, H0);
        mb_unpack(half ? A : B, M1, g1, H1);
        for (int a = 0; a < 3; a++) xe[a] = x[a];
        if (it == kNewtonMax) break;
        float H[6], g[3];
        for (int a = 0; a < 6; a++) H[a] = H0[a] + H1[a];
        for (int a = 0; a < 3; a++) g[a] = -(g0[a] + g1[a]);
        const float c0 = H[1] * H[2] - H[5] * H[5];
        const float c1 = H[5] * H[4] - H[3] * H[2];
        const float c2 = H[3] * H[5] - H[1] * H[4];
        const float det = H[0] * c0 + H[3] * c1 + H[4] * c2;
        const float id = __frcp_rn(det);
        const float b11 = H[0] * H[2] - H[4] * H[4], b12 = H[4] * H[3] - H[0] * H[5];
        const float b22 = H[0] * H[1] - H[3] * H[3];
        float dx[3];
        dx[0] = (c0 * g[0] + c1 * g[1] + c2 * g[2]) * id;
        dx[1] = (c1 * g[0] + b11 * g[1] + b12 * g[2]) * id;
        dx[2] = (c2 * g[0] + b12 * g[1] + b22 * g[2]) * id;
        const float s2 = dot3f(dx, dx);
        const int code = __shfl_sync(kFullWarp, newton_code(det == 0.f || !isfinite(det), s2, prev, it), 0);
        if (code == 1) break;
        for (int a = 0; a < 3; a++) x[a] += dx[a];
        if (code == 2) { converged = true; break; }
        if (code == 3) break;
        prev = s2;
    }
    for (int a = 0; a < 3; a++) xm[a] = x[a];
    if (!(M0 > P.c_tol_f && M0 < 1.0f && M1 > P.c_tol_f && M1 < 1.0f)) return false;
    valid = converged;
    const float q0 = (1.0f - M0) * __frcp_rn(dot3f(g0, g0)), q1 = (1.0f - M1) * __frcp_rn(dot3f(g1, g1));
    float dc[3];
    for (int a = 0; a < 3; a++) dc[a] = q0 * g0[a] - q1 * g1[a];
    const float dist = sqrtf(dot3f(dc, dc));
    delta = S.Rs[i] + S.Rs[j] - dist;
    if (!(delta > 0.f) || dist == 0.f) return false;
    const float idist = __frcp_rn(dist);
    for (int a = 0; a < 3; a++) {
        nv[a] = dc[a] * idist;
        xcp[a] = (xe[a] + q0 * g0[a]) - (S.Rs[i] - 0.5f * delta) * nv[a];
    }
    return true;
}

// Pair contacts of the candidate list, one item after the other, each by the
// whole warp (every lane writes the results); results into it_res (zeros
// when not in contact), as pair_contacts.
template <class SH>
__device__ void pair_contacts_w(const Params &P, SH &S, float h) {
    const int np = S.n;
    const int total = min(S.ioff[np], SH::kItems);
    for (int it = 0; it < total; it++) {
        int i = 0;  // last i with ioff[i] <= it
        while (i + 1 < np && S.ioff[i + 1] <= it) i++;
        const int j = S.up[i][it - S.ioff[i]];
        float d[3];
        rel_vec(S, P, i, j, d);
        const float brs = S.brad[i] + S.brad[j];
        const int was = S.it_on[it];
        float xm[3], xi[3];
        for (int a = 0; a < 3; a++) {
            xm[a] = S.it_xm[it][a];
            xi[a] = (was & CONTACT_ON) ? S.it_xi[it][a] : 0.f;
        }
        const int near = __shfl_sync(kFullWarp, dot3f(d, d) > brs * brs ? 0 : 1, 0);
        float Fi[3] = {0.f, 0.f, 0.f}, ti[3] = {0.f, 0.f, 0.f}, tj[3] = {0.f, 0.f, 0.f};
        int on = 0;
        bool hit = false;
        if (near) {
            float delta, nv[3], xcp[3];
            bool valid;
            hit = pair_geom_w(P, S, i, j, d, (was & CONTACT_WARM) != 0, xm, delta, nv, xcp, valid);
            on = valid ? CONTACT_WARM : 0;
            if (hit) {
                on |= CONTACT_ON;
                float rj[3], wri[3], wrj[3], vij[3];
                for (int a = 0; a < 3; a++) rj[a] = xcp[a] - d[a];
                cross3f(S.w[i], xcp, wri);
                cross3f(S.w[j], rj, wrj);
                for (int a = 0; a < 3; a++) vij[a] = (S.v[i][a] + wri[a]) - (S.v[j][a] + wrj[a]);
                contact_law_f(P, delta, nv, vij, xi, h, Fi);
                const float Fj[3] = {-Fi[0], -Fi[1], -Fi[2]};
                cross3f(xcp, Fi, ti);
                cross3f(rj, Fj, tj);
            }
        }
        __syncwarp();
        S.it_on[it] = on;
        if (near)
            for (int a = 0; a < 3; a++) S.it_xm[it][a] = xm[a];
        if (hit)
            for (int a = 0; a < 3; a++) S.it_xi[it][a] = xi[a];
        for (int a = 0; a < 3; a++) { S.it_res[it][a] = Fi[a]; S.it_res[it][3 + a] = ti[a]; S.it_res[it][6 + a] = tj[a]; }
    }
}
}  // namespace

// A contact group of up to kTinyContactGroup particles per warp,
// kTinyGroupsPerCta warps per CTA: the sub-steps of k_dem64c with the lanes
// split by particle (above).
__global__ void __launch_bounds__(32 * kTinyGroupsPerCta, 1) k_dem64t(Params P) {
    using SH = SharedTiny;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wt = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    SH &S = reinterpret_cast<SH *>(smem_raw)[wt];
    const int slot = (int)blockIdx.x * kTinyGroupsPerCta + wt;
    if (slot >= P.dem_list[2 + DEM_GROUP_TINY]) return;  // the whole warp
    const int *grp = dem_groups(P, DEM_GROUP_TINY) + 2 * slot;
    const int na = grp[1];
    const int *act = dem_active(P) + grp[0];
    const float h = P.h_f, hh = 0.5f * h, qh2 = 0.25f * h * h;
    const int c = lane % kSegLanes;
    const unsigned seg = ((1u << kSegLanes) - 1u) << (lane - c);  // this lane's particle lanes
    const bool own = lane / kSegLanes < na;
    const int k = own ? lane / kSegLanes : lane / kSegLanes % na;  // the particle (a mirror past the group)
    const int g = act[k];
    DevParticle *pp = &P.parts[g];

    Delta x[3], v[3], q[4], wb[3];
    float xlo[3], Fh[3], Th[3], iI[3], cI[3], bg[3];
    float Fc[3] = {0.f, 0.f, 0.f}, Tc[3] = {0.f, 0.f, 0.f};  // contact load of the last evaluation
    {
        double wbd[3];
        rot_body(pp->q, pp->w, wbd);
        for (int a = 0; a < 3; a++) {
            dl_set(x[a], pp->x[a]);
            xlo[a] = (float)(pp->x[a] - (double)x[a].bf);  // FP32 rounding error of the start position
            dl_set(v[a], pp->v[a]);
            dl_set(wb[a], wbd[a]);
            Fh[a] = (float)P.Fh[3 * g + a];
            Th[a] = (float)P.Th[3 * g + a];
            iI[a] = pp->iI_f[a];
            cI[a] = pp->cI_f[a];
            bg[a] = pp->bg_f[a];
        }
        for (int a = 0; a < 4; a++) dl_set(q[a], pp->q[a]);
    }
    const float inv_m = pp->inv_mass_f;
    const bool mov = !pp->fixed;
    const float reach = dem_reach(P, *pp, g);
    const int ncp = pp->ncp;
    // this lane's control points (body frame, weight); stand-ins past ncp
    const float4 cpa = c < ncp ? make_float4(pp->cpb_f[c][0], pp->cpb_f[c][1], pp->cpb_f[c][2], pp->K_f[c]) : far_cp();
    const float4 cpb = c + kSegLanes < ncp ? make_float4(pp->cpb_f[c + kSegLanes][0], pp->cpb_f[c + kSegLanes][1],
                                                         pp->cpb_f[c + kSegLanes][2], pp->K_f[c + kSegLanes])
                                           : far_cp();
    float4 rca = cpa, rcb = cpb;  // rotated
    if (lane == 0) {
        int o = 0;
        for (int m = 0; m < na; m++) { S.cpo[m] = o; o += P.parts[act[m]].ncp; }
        S.cpo[na] = o;
        S.n = na;
        if (o > SH::kCps) atomicOr(&P.status[ST_ERR], ERRB_DEM_CAPACITY);
    }
    if (lane < na) S.gid[lane] = act[lane];
    __syncwarp();
    if (S.cpo[na] > SH::kCps) return;

    // FP32 tables: position (hi + lo of the FP64 value), velocity, world
    // angular velocity from the body rate wf
    auto publish = [&](const float wf[3], const float qf[4]) {
        float ww[3];
        qrot_f(qf, wf, ww, true);
        for (int a = 0; a < 3; a++) {
            S.xh[k][a] = x[a].bf;
            S.xl[k][a] = xlo[a] + (x[a].d.hi + x[a].d.lo);
            S.v[k][a] = v[a].f();
            S.w[k][a] = ww[a];
        }
    };
    // this lane's control points rotated by qf, into registers and the table
    // (stand-ins into the scratch row)
    const int oc = S.cpo[k];
    float4 *const dsta = c < ncp ? &S.rc[oc + c] : &S.rc_pad[lane];
    float4 *const dstb = c + kSegLanes < ncp ? &S.rc[oc + c + kSegLanes] : &S.rc_pad[lane];
    auto rotate_cps = [&](const float qf[4]) {
        float r[3];
        const float ba[3] = {cpa.x, cpa.y, cpa.z}, bb[3] = {cpb.x, cpb.y, cpb.z};
        qrot_f(qf, ba, r, true);
        rca = make_float4(r[0], r[1], r[2], cpa.w);
        qrot_f(qf, bb, r, true);
        rcb = make_float4(r[0], r[1], r[2], cpb.w);
        *dsta = rca;
        *dstb = rcb;
    };
    {
        const float qf[4] = {q[0].f(), q[1].f(), q[2].f(), q[3].f()}, wf[3] = {wb[0].f(), wb[1].f(), wb[2].f()};
        publish(wf, qf);
        S.reach[k] = reach;
        S.brad[k] = pp->brad_f;
        S.Rs[k] = pp->Rs_f;
        rotate_cps(qf);
        if (c < NWALL) {  // lane c: the history of wall c
            const int wj = g * NWALL + c;
            S.w_on[k][c] = P.wall_on[wj];
            for (int a = 0; a < 3; a++) {
                S.w_xcw[k][c][a] = P.wall_xcw_f[3 * wj + a];
                S.w_xi[k][c][a] = P.wall_xi_f[3 * wj + a];
            }
        }
    }
    __syncwarp();
    int dummy = 0;
    if (na > 1) build_lists(P, S, &dummy);
    else if (lane == 0) {
        S.nup[0] = 0; S.ndn[0] = 0; S.ioff[0] = 0; S.ioff[1] = 0;
        for (int a = 0; a < 3; a++) S.xref[0][a] = S.xh[0][a] + S.xl[0][a];
    }
    __syncwarp();
    // contact load at the start: left by the previous step's DEM (same
    // state), unless the particles were set since
    if (!P.fc_valid) {
        pair_contacts_w(P, S, 0.f);
        __syncwarp();
        gather_pairs(S, k, Fc, Tc);
        walls_seg(P, S, k, seg, 0.f, rca, rcb, Fc, Tc);
    } else {
        for (int a = 0; a < 3; a++) {
            Fc[a] = (float)P.Fc[3 * g + a];
            Tc[a] = (float)P.Tc[3 * g + a];
        }
    }
    __syncwarp();
    for (int sub = 0; sub < P.n_sub; sub++) {
        Delta wh[3] = {wb[0], wb[1], wb[2]};
        int moved = 0;
        {
            float qf[4] = {q[0].f(), q[1].f(), q[2].f(), q[3].f()};
            if (mov) {
                // first half-kick and drift
                for (int a = 0; a < 3; a++) {
                    dl_add(v[a], hh * (bg[a] + (Fh[a] + Fc[a]) * inv_m));
                    dl_add(x[a], h * v[a].f());
                }
                // rotation: half-kick, q <- q (x) exp(h wh / 2)
                float Tw[3], Tb[3], wf[3] = {wb[0].f(), wb[1].f(), wb[2].f()}, dw[3], whf[3];
                for (int a = 0; a < 3; a++) Tw[a] = Th[a] + Tc[a];
                qrot_f(qf, Tw, Tb, false);
                euler_f(iI, cI, wf, Tb, dw);
                for (int a = 0; a < 3; a++) {
                    dl_add(wh[a], hh * dw[a]);
                    whf[a] = wh[a].f();
                }
                float cm1, sc;
                exp_half(hh, qh2, whf, cm1, sc);
                const float d1 = sc * whf[0], d2 = sc * whf[1], d3 = sc * whf[2];
                const float q0 = qf[0], q1 = qf[1], q2 = qf[2], q3 = qf[3];
                dl_add(q[0], q0 * cm1 - (q1 * d1 + q2 * d2 + q3 * d3));
                dl_add(q[1], q0 * d1 + q1 * cm1 + (q2 * d3 - q3 * d2));
                dl_add(q[2], q0 * d2 + q2 * cm1 + (q3 * d1 - q1 * d3));
                dl_add(q[3], q0 * d3 + q3 * cm1 + (q1 * d2 - q2 * d1));
                for (int a = 0; a < 4; a++) qf[a] = q[a].f();
            }
            const float whf[3] = {wh[0].f(), wh[1].f(), wh[2].f()};
            publish(whf, qf);
            float dr2 = 0.f;
            for (int a = 0; a < 3; a++) {
                const float dd = (x[a].bf - S.xref[k][a]) + (xlo[a] + (x[a].d.hi + x[a].d.lo));
                dr2 += dd * dd;
            }
            if (mov) rotate_cps(qf);
            moved = dr2 > 0.25f * kSkin * kSkin;
        }
        moved = __any_sync(kFullWarp, moved);
        __syncwarp();
        if (moved && na > 1) {
            store_items(P, S);
            __syncwarp();
            build_lists(P, S, &dummy);
        }
        pair_contacts_w(P, S, h);
        __syncwarp();
        {
            float F[3], T[3];
            gather_pairs(S, k, F, T);
            walls_seg(P, S, k, seg, h, rca, rcb, F, T);
            for (int a = 0; a < 3; a++) { Fc[a] = F[a]; Tc[a] = T[a]; }
            if (mov) {
                // closing half-kick with the new contact load
                for (int a = 0; a < 3; a++) dl_add(v[a], hh * (bg[a] + (Fh[a] + F[a]) * inv_m));
                const float qf[4] = {q[0].f(), q[1].f(), q[2].f(), q[3].f()};
                float Tw[3], Tb[3], dw[3], whf[3] = {wh[0].f(), wh[1].f(), wh[2].f()}, w1[3];
                for (int a = 0; a < 3; a++) { Tw[a] = Th[a] + T[a]; w1[a] = whf[a]; }
                qrot_f(qf, Tw, Tb, false);
                for (int it = 0; it + 1 < ROT_ITERS; it++) {
                    euler_f(iI, cI, w1, Tb, dw);
                    for (int a = 0; a < 3; a++) w1[a] = whf[a] + hh * dw[a];
                }
                euler_f(iI, cI, w1, Tb, dw);
                for (int a = 0; a < 3; a++) {
                    wb[a] = wh[a];
                    dl_add(wb[a], hh * dw[a]);
                }
            }
        }
        __syncwarp();
    }
    // the step's changes added to the FP64 state (still in the record)
    double qd[4] = {1, 0, 0, 0}, wbd[3] = {0, 0, 0}, xd[3] = {0, 0, 0}, vd[3] = {0, 0, 0};
    if (mov) {
        double wb0[3];
        rot_body(pp->q, pp->w, wb0);
        for (int a = 0; a < 4; a++) qd[a] = q[a].fin(pp->q[a]);
        for (int a = 0; a < 3; a++) {
            wbd[a] = wb[a].fin(wb0[a]);
            xd[a] = x[a].fin(pp->x[a]);
            vd[a] = v[a].fin(pp->v[a]);
        }
        quat_normalize(qd);
        for (int a = 0; a < 4; a++) dl_set(q[a], qd[a]);
    }
    // contact load of the end state (springs not advanced): reported by
    // lbm_get_contact_forces and the start load of the next step
    {
        const float qf[4] = {q[0].f(), q[1].f(), q[2].f(), q[3].f()}, wf[3] = {wb[0].f(), wb[1].f(), wb[2].f()};
        publish(wf, qf);
        if (mov) rotate_cps(qf);
    }
    __syncwarp();
    pair_contacts_w(P, S, 0.f);
    __syncwarp();
    float F[3], T[3];
    gather_pairs(S, k, F, T);
    walls_seg(P, S, k, seg, 0.f, rca, rcb, F, T);
    __syncwarp();  // every lane has read the particle records (the end state is written below)
    if (own) {
        if (c < NWALL) {  // lane c: the history of wall c
            const int wj = g * NWALL + c;
            P.wall_on[wj] = S.w_on[k][c];
            for (int a = 0; a < 3; a++) {
                P.wall_xcw_f[3 * wj + a] = S.w_xcw[k][c][a];
                P.wall_xi_f[3 * wj + a] = S.w_xi[k][c][a];
            }
        }
        if (c == 0) {
            for (int a = 0; a < 3; a++) {
                P.Fc[3 * g + a] = (double)F[a];
                P.Tc[3 * g + a] = (double)T[a];
            }
            if (mov) {
                double ww[3];
                rot_world(qd, wbd, ww);
                for (int a = 0; a < 3; a++) {
                    pp->x[a] = xd[a];
                    pp->v[a] = vd[a];
                    pp->w[a] = ww[a];
                }
                for (int a = 0; a < 4; a++) pp->q[a] = qd[a];
            }
            // the planning assumed no larger displacement (contacts with
            // inactive particles would have been missed otherwise)
            float d2 = 0.f;
            for (int a = 0; a < 3; a++) d2 += x[a].d.hi * x[a].d.hi;
            if (d2 > reach * reach) atomicOr(&P.status[ST_ERR], ERRB_DEM_REACH);
        }
    }
    if (na > 1) store_items(P, S);
}

void launch_dem64c(const Params &P, cudaStream_t st) {
    // the dynamic shared memory limits are raised once per device
    static bool attr_set[64] = {};
    static_assert(sizeof(SharedSmall) <= 48 * 1024, "small contact-group tables exceed 48 KB");
    static_assert(kTinyGroupsPerCta * sizeof(SharedTiny) <= 48 * 1024, "tiny contact-group tables exceed 48 KB");
    const int big = (int)sizeof(Shared);
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev])
        attr_set[dev] = cudaFuncSetAttribute(k_dem64c<Shared, DEM_GROUP_LARGE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, big) == cudaSuccess;
    // grids for the worst case (every group tiny, or small); at most np / 33
    // groups are large.  A tiny-group CTA of 8 warps holds most of an SM's
    // registers, so few other CTAs share the SM with its latency-bound chains.
    k_dem64t<<<(P.np + kTinyGroupsPerCta - 1) / kTinyGroupsPerCta, 32 * kTinyGroupsPerCta,
               kTinyGroupsPerCta * sizeof(SharedTiny), st>>>(P);
    k_dem64c<SharedSmall, DEM_GROUP_SMALL><<<P.np / (kTinyContactGroup + 1) + 1, kSmallContactGroup,
                                             sizeof(SharedSmall), st>>>(P);
    k_dem64c<Shared, DEM_GROUP_LARGE><<<P.np / (kSmallContactGroup + 1) + 1, kThreads, big, st>>>(P);
}

// One CTA: a single warp for a few particles (the barriers between the
// sub-step phases are then nearly free), else kThreads threads.
void launch_dem32(const Params &P, cudaStream_t st) {
    // the dynamic shared memory limit is raised once per device
    static bool attr_set[64] = {};
    static_assert(sizeof(Shared) <= 227 * 1024, "k_dem32 tables exceed the shared memory of one CTA");
    const int bytes = (int)sizeof(Shared);
    int dev = 0;
    // a failure here leaves its error for the caller's cudaGetLastError()
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev])
        attr_set[dev] = cudaFuncSetAttribute(k_dem32, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    k_dem32<<<1, P.np <= 16 ? 32 : kThreads, bytes, st>>>(P);
}

}  // namespace lbmmb
