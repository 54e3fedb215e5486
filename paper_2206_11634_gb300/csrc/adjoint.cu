// Discrete adjoint of the lattice sweep around one fixed metaball (the C ABI
// of include/lbm_adjoint.h): d(mean drag)/d(control points, weights) with
// the node flags frozen.
//
// Forward step (offset form g = f - w rho0, as the main sweep): for every
// fluid node, pull g_i from x - e_i, or, on a particle link (x - e_i solid),
// take the VIBB unknown of Eqs. (19)-(25) from the node's own post-collision
// populations and those of x_ff = x + e_i (halfway bounce-back when x_ff is
// solid); collide (BGK + Guo, Eqs. (15)-(18)); the drag of the step is the
// x component of Eq. (28) summed over the links (u_w = 0; its constant part
// cancels over the closed link set, as in the main sweep).
//
// Adjoint of one step, for lambda' = dJ/dg+(t+1):
//   A1  per fluid node: recompute the pulled values, lambda_in = (dBGK/dg_in)^T
//       lambda' (the equilibrium and forcing depend on g_in only through the
//       density and momentum, so this is (1 - omega) lambda' + a + b.e_j),
//       plus the drag's direct dependence on the pulled link values;
//   A2  per fluid node y: dJ/dg+(t)_k(y) = lambda_in_k(y + e_k) (the pull,
//       transposed) plus the halfway links' and the drag's dependence on the
//       node's own populations.  A1 and A2 run as one kernel in push form:
//       node n stores lambda_in_j(n) straight into dJ/dg+(t)_j(n - e_j) when
//       n - e_j is a fluid node, and writes dJ/dg+(t) itself in the
//       directions whose neighbour is solid (its links); every entry of a
//       fluid node has exactly one writer, and lambda_in is kept only per
//       link (for A3), so lambda is read and written once per step;
//   A3  per VIBB link: the link value depends on the node's and x_ff's
//       populations through their density, momentum and one population each,
//       and on q: those 11 partial derivatives come from forward-mode dual
//       numbers through the same VIBB code as the forward step, and are
//       scattered (atomics) into dJ/dg+(t) and into dJ/dq of the link.
// The states of each segment of ceil(sqrt(T)) steps are recomputed from the
// forward run's checkpoint.  Finally dJ/dq goes through Eq. (27) and Eq. (4)
// to the control points and weights (FP64).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_adjoint.h"
#include "lbm_internal.cuh"

using namespace lbmmb;

namespace {

constexpr int Q = 19;
using L19 = Lat<19>;
constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// ---------------------------------------------------------------------------
// forward-mode dual numbers with N tangents
// ---------------------------------------------------------------------------
template <int N>
struct Dual {
    float v;
    float d[N];
};
template <int N>
__device__ __forceinline__ Dual<N> dconst(float x) {
    Dual<N> r;
    r.v = x;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = 0.f;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> dvar(float x, int k) {
    Dual<N> r = dconst<N>(x);
    r.d[k] = 1.f;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(Dual<N> a, Dual<N> b) {
    Dual<N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(Dual<N> a, Dual<N> b) {
    Dual<N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(Dual<N> a, Dual<N> b) {
    Dual<N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(Dual<N> a, Dual<N> b) {
    Dual<N> r;
    const float ib = 1.0f / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator+(Dual<N> a, float b) { return a + dconst<N>(b); }
template <int N> __device__ __forceinline__ Dual<N> operator+(float a, Dual<N> b) { return dconst<N>(a) + b; }
template <int N> __device__ __forceinline__ Dual<N> operator-(Dual<N> a, float b) { return a - dconst<N>(b); }
template <int N> __device__ __forceinline__ Dual<N> operator-(float a, Dual<N> b) { return dconst<N>(a) - b; }
template <int N>
__device__ __forceinline__ Dual<N> operator*(Dual<N> a, float b) {
    Dual<N> r;
    r.v = a.v * b;
#pragma unroll
    for (int k = 0; k < N; k++) r.d[k] = a.d[k] * b;
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(float a, Dual<N> b) { return b * a; }
template <int N> __device__ __forceinline__ Dual<N> operator/(float a, Dual<N> b) { return dconst<N>(a) / b; }
__device__ __forceinline__ float val(float x) { return x; }
template <int N> __device__ __forceinline__ float val(const Dual<N> &x) { return x.v; }

// ---------------------------------------------------------------------------
// the pieces of the step, generic in the scalar type
// ---------------------------------------------------------------------------
struct AdjConst {
    int nx, ny, nz;
    long long N;
    float rho0, omega, gfac;
    float F[3];
};

// f^eq_i - w_i rho0 for density rho = rho0 + drho, velocity u (Eq. (16))
template <typename T>
__device__ __forceinline__ T geq_t(int ex, int ey, int ez, float w, T drho, T rho, T ux, T uy, T uz) {
    const T eu = ux * (float)ex + uy * (float)ey + uz * (float)ez;
    const T uu = ux * ux + uy * uy + uz * uz;
    return (drho + rho * (eu * 3.0f + eu * eu * 4.5f - uu * 1.5f)) * w;
}

// The VIBB unknown of a link whose direction into the solid is d (index io),
// u_w = 0 (a fixed particle), from the moments and the io population of the
// fluid node x_f (post-collision: u = (m - F/2)/rho) and of x_ff.
template <typename T>
__device__ __forceinline__ T vibb_t(const AdjConst &A, int io, T q, T drf, T mfx, T mfy, T mfz, T gf, T drff, T mffx,
                                    T mffy, T mffz, T gff) {
    // io is a run-time index: packed lattice entries, no table in local memory
    const int dx = lat_e<19>(io, 0), dy = lat_e<19>(io, 1), dz = lat_e<19>(io, 2);
    const float w = (float)lat_w<19>(io);
    const T rf = drf + A.rho0, rff = drff + A.rho0;
    const T irf = 1.0f / rf, irff = 1.0f / rff;
    const T ufx = (mfx - 0.5f * A.F[0]) * irf, ufy = (mfy - 0.5f * A.F[1]) * irf, ufz = (mfz - 0.5f * A.F[2]) * irf;
    const T uffx = (mffx - 0.5f * A.F[0]) * irff, uffy = (mffy - 0.5f * A.F[1]) * irff,
            uffz = (mffz - 0.5f * A.F[2]) * irff;
    const T geqf = geq_t<T>(dx, dy, dz, w, drf, rf, ufx, ufy, ufz);
    const T geqff = geq_t<T>(dx, dy, dz, w, drff, rff, uffx, uffy, uffz);
    const T q2 = q * 2.0f, one_m2q = 1.0f - q2;
    const T fneq = q2 * (gf - geqf) + one_m2q * (gff - geqff);                 // Eq. (21)
    T drd, usx, usy, usz;
    if (val(q) <= 0.5f) {                                                       // Eqs. (22)-(23)
        drd = q2 * drf + one_m2q * drff;
        usx = q2 * ufx + one_m2q * uffx;
        usy = q2 * ufy + one_m2q * uffy;
        usz = q2 * ufz + one_m2q * uffz;
    } else {
        drd = drf;
        const T a = (1.0f - q) / q;  // + (2q - 1)/q u_w, u_w = 0
        usx = a * ufx;
        usy = a * ufy;
        usz = a * ufz;
    }
    const T b = (1.0f - q) / (1.0f + q);                                        // Eq. (24), u_w = 0
    const T udx = (usx + 2.0f * (b * uffx)) * (1.0f / 3.0f);                   // Eq. (25)
    const T udy = (usy + 2.0f * (b * uffy)) * (1.0f / 3.0f);
    const T udz = (usz + 2.0f * (b * uffz)) * (1.0f / 3.0f);
    return geq_t<T>(dx, dy, dz, w, drd, drd + A.rho0, udx, udy, udz) + fneq;  // Eqs. (20), (19)
}

// The part of the collided population i that depends on the pulled values
// only through the density offset drho and the momentum m: omega g^eq_i +
// Guo's term (Eq. (15) with Eq. (18)'s half-force shift).
template <typename T>
__device__ __forceinline__ T collide_h(const AdjConst &A, int i, T drho, T mx, T my, T mz) {
    const int ex = L19::e(i, 0), ey = L19::e(i, 1), ez = L19::e(i, 2);
    const float w = (float)L19::w(i);
    const T rho = drho + A.rho0;
    const T ir = 1.0f / rho;
    const T ux = (mx + 0.5f * A.F[0]) * ir, uy = (my + 0.5f * A.F[1]) * ir, uz = (mz + 0.5f * A.F[2]) * ir;
    const T eu = ux * (float)ex + uy * (float)ey + uz * (float)ez;
    const T uF = ux * A.F[0] + uy * A.F[1] + uz * A.F[2];
    const float eF = ex * A.F[0] + ey * A.F[1] + ez * A.F[2];
    const T g = geq_t<T>(ex, ey, ez, w, drho, rho, ux, uy, uz) * A.omega;
    return g + ((eF - uF) * 3.0f + eu * (9.0f * eF)) * (A.gfac * w);
}

// ---------------------------------------------------------------------------
// device data
// ---------------------------------------------------------------------------
struct AdjDev {
    AdjConst c;
    const uint8_t *solid;     // [N]
    const uint32_t *lmask;    // [N] particle-link directions of each node
    const int *linkid;        // [19][N] link index or -1
    const int *l_nf, *l_dir, *l_nff;  // [L] node, direction (unknown), x_ff node or -1
    float *l_q;               // [L]
    double *l_dqdMf, *l_dqdMs;  // [L] dq/dM at x_f and x_s (0 where q was clamped)
    double *l_dJdq;           // [L]
    float *l_lam;             // [L] lambda_in of the link's direction at its node (this step)
    int nlinks;
    const double *cp;         // [ncp][3] world
    const double *K;          // [ncp]
    int ncp;
    unsigned long long *J_fix;  // sum of the window's drag (2^-40 units)
    double *grad;             // [ncp][4]: dJ/dx, dJ/dy, dJ/dz, dJ/dK
    float inv_W;
};

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// The value a particle link of direction i (the unknown, arriving from the
// solid node x - e_i) takes at fluid node n: VIBB of Eqs. (19)-(25) from the
// node's moments (drho_f, m_f) and x_ff's populations, or halfway
// bounce-back when x_ff is solid.  i is a run-time index: populations are
// read from the state by address, never from an indexed local array.
__device__ __noinline__ float link_value(const AdjDev &D, const float *__restrict__ S, long long n, int i,
                                         float drho_f, float mfx, float mfy, float mfz) {
    const AdjConst &A = D.c;
    const long long N = A.N;
    const int io = L19::opp(i);
    const float gown_io = S[(long long)io * N + n];
    const int L = D.linkid[(long long)i * N + n];
    const int nff = D.l_nff[L];
    if (nff < 0) return gown_io;  // halfway bounce-back, u_w = 0
    float drff = 0.f, mff[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const float gk = S[(long long)k * N + nff];
        drff += gk;
        mff[0] += gk * L19::e(k, 0);
        mff[1] += gk * L19::e(k, 1);
        mff[2] += gk * L19::e(k, 2);
    }
    const float gff_io = S[(long long)io * N + nff];
    return vibb_t<float>(A, io, D.l_q[L], drho_f, mfx, mfy, mfz, gown_io, drff, mff[0], mff[1], mff[2], gff_io);
}

// The pulled values g_in of fluid node (x, y, z) from the state S, with the
// link values substituted on its particle links (lm).  Every array here is
// indexed by unrolled loop counters only, so it stays in registers.
__device__ __forceinline__ void gather(const AdjDev &D, const float *__restrict__ S, int x, int y, int z, long long n,
                                       uint32_t lm, float gin[Q]) {
    const AdjConst &A = D.c;
    const int N = (int)A.N;  // fewer than 2^31 nodes
    // every pull is issued at once (on a link direction its value is replaced
    // below), so the loads do not wait for the link mask
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int sx = wrapi(x - L19::e(i, 0), A.nx), sy = wrapi(y - L19::e(i, 1), A.ny),
                  sz = wrapi(z - L19::e(i, 2), A.nz);
        gin[i] = S[(long long)i * N + (sx + A.nx * (sy + A.ny * sz))];
    }
    if (!lm) return;
    float drho_f = 0.f, mf[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const float g = S[(long long)k * N + n];
        drho_f += g;
        mf[0] += g * L19::e(k, 0);
        mf[1] += g * L19::e(k, 1);
        mf[2] += g * L19::e(k, 2);
    }
#pragma unroll
    for (int i = 0; i < Q; i++)
        if ((lm >> i) & 1u) gin[i] = link_value(D, S, n, i, drho_f, mf[0], mf[1], mf[2]);
}

// Node of this thread: CTA = 32 x 4 x 2 nodes
__device__ __forceinline__ bool node_of(const AdjConst &A, int &x, int &y, int &z, long long &n) {
    x = blockIdx.x * 32 + threadIdx.x % 32;
    y = blockIdx.y * 4 + (threadIdx.x / 32) % 4;
    z = blockIdx.z * 2 + threadIdx.x / 128;
    n = x + (long long)A.nx * (y + (long long)A.ny * z);
    return x < A.nx && y < A.ny && z < A.nz;
}

__global__ void __launch_bounds__(256) k_adj_init(AdjDev D, float *S, float ux, float uy, float uz) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < D.c.N; n += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int i = 0; i < Q; i++)
            S[(long long)i * D.c.N + n] = geq_t<float>(L19::e(i, 0), L19::e(i, 1), L19::e(i, 2), (float)L19::w(i), 0.f,
                                                       D.c.rho0, ux, uy, uz);
}

// q of every link for the control points of this forward run (Eq. (27) with
// M of Eq. (4), FP64, periodic minimum image), and dq/dM for the gradient.
__global__ void k_adj_q(AdjDev D) {
    const AdjConst &A = D.c;
    for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < D.nlinks; L += gridDim.x * blockDim.x) {
        const long long n = D.l_nf[L];
        const int io = L19::opp(D.l_dir[L]);
        const int x = (int)(n % A.nx), y = (int)((n / A.nx) % A.ny), z = (int)(n / ((long long)A.nx * A.ny));
        const double pf[3] = {(double)x, (double)y, (double)z};
        const double ps[3] = {pf[0] + lat_e<19>(io, 0), pf[1] + lat_e<19>(io, 1), pf[2] + lat_e<19>(io, 2)};
        const int dims[3] = {A.nx, A.ny, A.nz};
        double Mf = 0.0, Ms = 0.0;
        for (int c = 0; c < D.ncp; c++) {
            double rf2 = 0.0, rs2 = 0.0;
            for (int a = 0; a < 3; a++) {
                double df = pf[a] - D.cp[3 * c + a], ds = ps[a] - D.cp[3 * c + a];
                df -= dims[a] * rint(df / dims[a]);
                ds -= dims[a] * rint(ds / dims[a]);
                rf2 += df * df;
                rs2 += ds * ds;
            }
            Mf += D.K[c] / rf2;
            Ms += D.K[c] / rs2;
        }
        const double den = Ms - Mf;
        double q = (1.0 - Mf) / den;  // c0 = 1 (Eq. (26) with the surface of Eq. (4))
        double dqf = (1.0 - Ms) / (den * den), dqs = -(1.0 - Mf) / (den * den);
        if (!(q > 0.0)) { q = 0.0; dqf = dqs = 0.0; }
        if (q > 1.0) { q = 1.0; dqf = dqs = 0.0; }
        D.l_q[L] = (float)q;
        D.l_dqdMf[L] = dqf;
        D.l_dqdMs[L] = dqs;
    }
}

// One forward step S -> R; accumulates the drag when in the window.
__global__ void __launch_bounds__(256) k_adj_step(AdjDev D, const float *__restrict__ S, float *__restrict__ R,
                                                   int window) {
    const AdjConst &A = D.c;
    int x, y, z;
    long long n;
    const bool in = node_of(A, x, y, z, n);
    // the node's solid mark and link mask in one round
    const bool solid = in ? D.solid[n] != 0 : true;
    const uint32_t lm = in ? D.lmask[n] : 0u;
    const bool act = in && !solid;
    float Fx = 0.f;
    if (act) {
        float gin[Q];
        gather(D, S, x, y, z, n, lm, gin);
        if (window && lm) {
#pragma unroll
            for (int i = 1; i < Q; i++) {
                if (!((lm >> i) & 1u)) continue;
                const int io = L19::opp(i);
                // Eq. (28), x component, offsets
                Fx += (float)L19::e(io, 0) * (S[(long long)io * A.N + n] + gin[i]);
            }
        }
        float drho = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            drho += gin[i];
            mx += gin[i] * L19::e(i, 0);
            my += gin[i] * L19::e(i, 1);
            mz += gin[i] * L19::e(i, 2);
        }
#pragma unroll
        for (int i = 0; i < Q; i++)
            R[(long long)i * A.N + n] = (1.0f - A.omega) * gin[i] + collide_h<float>(A, i, drho, mx, my, mz);
    }
    if (window) {
        for (int o = 16; o > 0; o >>= 1) Fx += __shfl_xor_sync(0xffffffffu, Fx, o);
        if ((threadIdx.x & 31) == 0 && Fx != 0.f)
            atomicAdd(D.J_fix, (unsigned long long)__float2ll_rn(Fx * (float)(1ull << kForceFixBits)));
    }
}

// A1 + A2 in push form (see the top of the file): lambda_in of fluid node n
// through the collision (with the drag's dependence on the pulled link
// values), pushed along the pull it came from; on a link direction i the
// node writes dJ/dg+(t) of its own opposite direction (no fluid neighbour
// pushes it): the halfway link's value and the drag's dependence on the
// node's own populations, and keeps lambda_in_i(n) for A3.  The arithmetic
// and its order are those of the two-kernel form.
__global__ void __launch_bounds__(256, 3) k_adj_back(AdjDev D, const float *__restrict__ S,
                                                    const float *__restrict__ lamN, float *__restrict__ lamT,
                                                    int window) {
    const AdjConst &A = D.c;
    int x, y, z;
    long long n;
    if (!node_of(A, x, y, z, n)) return;
    const bool solid = D.solid[n] != 0;
    const uint32_t lm = D.lmask[n];  // with the solid mark, in one round
    if (solid) return;
    float gin[Q];
    gather(D, S, x, y, z, n, lm, gin);
    float drho = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        drho += gin[i];
        mx += gin[i] * L19::e(i, 0);
        my += gin[i] * L19::e(i, 1);
        mz += gin[i] * L19::e(i, 2);
    }
    // a = sum_i lambda_i dh_i/d(drho), b = sum_i lambda_i dh_i/dm for
    // collide_h (h_i = omega g^eq_i + Guo's term, u = (m + F/2) / rho),
    // differentiated by hand: with P_i = 3 e.u + 4.5 (e.u)^2 - 1.5 u.u,
    //   dh_i/d(drho) at fixed u = omega w_i (1 + P_i),
    //   dh_i/du = omega w_i rho (3 e_i + 9 (e_i.u) e_i - 3 u)
    //             + gfac w_i (9 (e_i.F) e_i - 3 F),
    // and du/dm = I / rho, du/d(drho) = -u / rho.
    const float rho = drho + A.rho0, ir = 1.0f / rho;
    const float ux = (mx + 0.5f * A.F[0]) * ir, uy = (my + 0.5f * A.F[1]) * ir, uz = (mz + 0.5f * A.F[2]) * ir;
    const float uu = ux * ux + uy * uy + uz * uz;
    float lam[Q], sp = 0.f, sl = 0.f, v3[3] = {0.f, 0.f, 0.f}, f3[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Q; i++) {
        lam[i] = lamN[(long long)i * A.N + n];
        const int ex = L19::e(i, 0), ey = L19::e(i, 1), ez = L19::e(i, 2);
        const float lw = lam[i] * (float)L19::w(i);
        const float eu = ux * (float)ex + uy * (float)ey + uz * (float)ez;
        sp += lw * (1.0f + (eu * 3.0f + eu * eu * 4.5f - uu * 1.5f));
        sl += lw;
        const float c = lw * (3.0f + 9.0f * eu);
        const float cf = lw * (9.0f * (ex * A.F[0] + ey * A.F[1] + ez * A.F[2]));
        v3[0] += c * ex; v3[1] += c * ey; v3[2] += c * ez;
        f3[0] += cf * ex; f3[1] += cf * ey; f3[2] += cf * ez;
    }
    const float u3[3] = {ux, uy, uz};
    float b[3], gu = 0.f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float g = A.omega * rho * (v3[c] - 3.0f * u3[c] * sl) + A.gfac * (f3[c] - 3.0f * A.F[c] * sl);
        b[c] = g * ir;
        gu += g * u3[c];
    }
    const float a = A.omega * sp - gu * ir;
#pragma unroll
    for (int j = 0; j < Q; j++) {
        float v = (1.0f - A.omega) * lam[j] + a + b[0] * L19::e(j, 0) + b[1] * L19::e(j, 1) + b[2] * L19::e(j, 2);
        if ((lm >> j) & 1u) {
            // link j: x - e_j is solid; lamT_{opp j}(n) has no other writer
            if (window) v += D.inv_W * (float)L19::e(L19::opp(j), 0);
            const int L = D.linkid[(long long)j * A.N + n];
            D.l_lam[L] = v;
            const int io = L19::opp(j);
            float acc = 0.f;
            if (D.l_nff[L] < 0) acc += v;
            if (window) acc += D.inv_W * (float)L19::e(io, 0);
            lamT[(long long)io * A.N + n] = acc;
        } else {
            const int tx = wrapi(x - L19::e(j, 0), A.nx), ty = wrapi(y - L19::e(j, 1), A.ny),
                      tz = wrapi(z - L19::e(j, 2), A.nz);
            lamT[(long long)j * A.N + (tx + A.nx * (ty + (long long)A.ny * tz))] = v;
        }
    }
}

// A3: the VIBB links (x_ff fluid): 11 partial derivatives by dual numbers,
// scattered into dJ/dg+(t) at x_f and x_ff, and dJ/dq of the link.
__global__ void __launch_bounds__(128) k_adj_vibb(AdjDev D, const float *__restrict__ S, float *__restrict__ lamT) {
    const AdjConst &A = D.c;
    const long long N = A.N;
    for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < D.nlinks; L += gridDim.x * blockDim.x) {
        const int nff = D.l_nff[L];
        if (nff < 0) continue;
        const long long nf = D.l_nf[L];
        const int i = D.l_dir[L], io = L19::opp(i);
        const float lam = D.l_lam[L];
        if (lam == 0.f) continue;
        float drf = 0.f, mf[3] = {0.f, 0.f, 0.f}, gf = 0.f, drff = 0.f, mff[3] = {0.f, 0.f, 0.f}, gff = 0.f;
#pragma unroll
        for (int k = 0; k < Q; k++) {
            const float a = S[(long long)k * N + nf], b = S[(long long)k * N + nff];
            drf += a;
            drff += b;
            for (int c = 0; c < 3; c++) {
                mf[c] += a * L19::e(k, c);
                mff[c] += b * L19::e(k, c);
            }
            if (k == io) { gf = a; gff = b; }
        }
        const Dual<11> v = vibb_t<Dual<11>>(A, io, dvar<11>(D.l_q[L], 0), dvar<11>(drf, 1), dvar<11>(mf[0], 2),
                                            dvar<11>(mf[1], 3), dvar<11>(mf[2], 4), dvar<11>(gf, 5),
                                            dvar<11>(drff, 6), dvar<11>(mff[0], 7), dvar<11>(mff[1], 8),
                                            dvar<11>(mff[2], 9), dvar<11>(gff, 10));
        D.l_dJdq[L] += (double)lam * (double)v.d[0];
#pragma unroll
        for (int k = 0; k < Q; k++) {
            const float ek[3] = {(float)L19::e(k, 0), (float)L19::e(k, 1), (float)L19::e(k, 2)};
            float cf = v.d[1] + v.d[2] * ek[0] + v.d[3] * ek[1] + v.d[4] * ek[2];
            float cff = v.d[6] + v.d[7] * ek[0] + v.d[8] * ek[1] + v.d[9] * ek[2];
            if (k == io) { cf += v.d[5]; cff += v.d[10]; }
            atomicAdd(&lamT[(long long)k * N + nf], lam * cf);
            atomicAdd(&lamT[(long long)k * N + nff], lam * cff);
        }
    }
}

// dJ/dq -> dJ/d(control point position, weight) through Eq. (27) and Eq. (4).
__global__ void __launch_bounds__(256) k_adj_grad(AdjDev D) {
    __shared__ double sg[LBM_MAX_CP][4];
    const AdjConst &A = D.c;
    for (int k = threadIdx.x; k < D.ncp * 4; k += blockDim.x) sg[k / 4][k % 4] = 0.0;
    __syncthreads();
    const int dims[3] = {A.nx, A.ny, A.nz};
    for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < D.nlinks; L += gridDim.x * blockDim.x) {
        const double G = D.l_dJdq[L];
        if (G == 0.0) continue;
        const double gf = G * D.l_dqdMf[L], gs = G * D.l_dqdMs[L];
        if (gf == 0.0 && gs == 0.0) continue;
        const long long n = D.l_nf[L];
        const int io = L19::opp(D.l_dir[L]);
        const double pf[3] = {(double)(n % A.nx), (double)((n / A.nx) % A.ny), (double)(n / ((long long)A.nx * A.ny))};
        const double ps[3] = {pf[0] + lat_e<19>(io, 0), pf[1] + lat_e<19>(io, 1), pf[2] + lat_e<19>(io, 2)};
        for (int c = 0; c < D.ncp; c++) {
            double rf[3], rs[3], rf2 = 0.0, rs2 = 0.0;
            for (int a = 0; a < 3; a++) {
                rf[a] = pf[a] - D.cp[3 * c + a];
                rs[a] = ps[a] - D.cp[3 * c + a];
                rf[a] -= dims[a] * rint(rf[a] / dims[a]);
                rs[a] -= dims[a] * rint(rs[a] / dims[a]);
                rf2 += rf[a] * rf[a];
                rs2 += rs[a] * rs[a];
            }
            // M = sum K / |x - x_c|^2:  dM/dK_c = 1/r^2,  dM/dx_c = 2 K_c (x - x_c) / r^4
            atomicAdd(&sg[c][3], gf / rf2 + gs / rs2);
            const double cf = gf * 2.0 * D.K[c] / (rf2 * rf2), cs = gs * 2.0 * D.K[c] / (rs2 * rs2);
            for (int a = 0; a < 3; a++) atomicAdd(&sg[c][a], cf * rf[a] + cs * rs[a]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < D.ncp * 4; k += blockDim.x) atomicAdd(&D.grad[k], sg[k / 4][k % 4]);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct lbm_adj {
    lbm_config cfg;
    int T, W, K, C;          // steps, window, checkpoint interval, checkpoints
    int ncp, nlinks;
    long long N;
    size_t S;                // bytes of one state (19 N floats)
    char *ws;
    cudaStream_t stream;
    size_t o_state[2], o_ckpt, o_seg, o_lam[2], o_llam, o_solid, o_lmask, o_linkid, o_lnf, o_ldir, o_lnff, o_lq,
        o_dqf, o_dqs, o_dJdq, o_cp, o_K, o_J, o_grad, total;
    bool have_forward;
    char err[256];
};

namespace {

thread_local char g_adj_error[256] = "no error";

int afail(lbm_adj *a, int code, const char *fmt, ...) {
    char *buf = a ? a->err : g_adj_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}
int acheck(lbm_adj *a, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    return afail(a, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

const char *adj_check(const lbm_config *c, const lbm_particle *p, int T, int W) {
    if (!c || !p) return "config or particle is NULL";
    if (c->nx < 4 || c->ny < 4 || c->nz < 4) return "nx, ny, nz must be >= 4";
    if ((long long)c->nx * c->ny * c->nz >= (1LL << 31)) return "lattice must hold fewer than 2^31 nodes";
    if (!c->periodic[0] || !c->periodic[1] || !c->periodic[2]) return "the adjoint needs a fully periodic box";
    if (c->lattice != 19) return "the adjoint runs D3Q19";
    if (!(c->tau > 0.5)) return "tau must be > 1/2";
    if (!(c->rho0 > 0.0)) return "rho0 must be > 0";
    if (c->c0 != 1.0 && c->c0 != 0.0) return "the adjoint takes the surface M = 1 (c0 = 1)";
    if (p->n_cp < 1 || p->n_cp > LBM_MAX_CP) return "n_cp out of range";
    if (T < 1 || W < 1 || W > T) return "need T >= 1 and 1 <= W <= T";
    return nullptr;
}

// World control points of the particle (x + R(q) cp).
void world_cps(const lbm_particle *p, std::vector<double> &cp) {
    double q[4] = {p->q[0], p->q[1], p->q[2], p->q[3]};
    const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (double &v : q) v /= qn;
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                         2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    cp.assign(3 * (size_t)p->n_cp, 0.0);
    for (int k = 0; k < p->n_cp; k++)
        for (int a = 0; a < 3; a++)
            cp[3 * k + a] = p->x[a] + R[3 * a] * p->cp[k][0] + R[3 * a + 1] * p->cp[k][1] + R[3 * a + 2] * p->cp[k][2];
}

// Frozen flags (M >= 1, periodic minimum image) and the links, in node then
// direction order.
void classify_links(const lbm_config *c, const lbm_particle *p, std::vector<uint8_t> &solid,
                    std::vector<uint32_t> &lmask, std::vector<int> &nf, std::vector<int> &dir, std::vector<int> &nff) {
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    const long long N = (long long)nx * ny * nz;
    std::vector<double> cp;
    world_cps(p, cp);
    solid.assign((size_t)N, 0);
    const int dims[3] = {nx, ny, nz};
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                const double pt[3] = {(double)x, (double)y, (double)z};
                double M = 0.0;
                for (int k = 0; k < p->n_cp; k++) {
                    double r2 = 0.0;
                    for (int a = 0; a < 3; a++) {
                        double d = pt[a] - cp[3 * k + a];
                        d -= dims[a] * std::rint(d / dims[a]);
                        r2 += d * d;
                    }
                    M += p->K[k] / r2;
                }
                solid[x + (size_t)nx * (y + (size_t)ny * z)] = M >= 1.0;
            }
    lmask.assign((size_t)N, 0u);
    nf.clear();
    dir.clear();
    nff.clear();
    auto wrap = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                const long long n = x + (long long)nx * (y + (long long)ny * z);
                if (solid[(size_t)n]) continue;
                for (int i = 1; i < Q; i++) {
                    const int ex = L19::e(i, 0), ey = L19::e(i, 1), ez = L19::e(i, 2);
                    const long long s = wrap(x - ex, nx) + (long long)nx * (wrap(y - ey, ny) + (long long)ny * wrap(z - ez, nz));
                    if (!solid[(size_t)s]) continue;
                    const long long f2 = wrap(x + ex, nx) + (long long)nx * (wrap(y + ey, ny) + (long long)ny * wrap(z + ez, nz));
                    lmask[(size_t)n] |= 1u << i;
                    nf.push_back((int)n);
                    dir.push_back(i);
                    nff.push_back(solid[(size_t)f2] ? -1 : (int)f2);
                }
            }
}

void adj_layout(lbm_adj *a) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t L = (size_t)std::max(1, a->nlinks), N = (size_t)a->N;
    a->o_state[0] = take(a->S);
    a->o_state[1] = take(a->S);
    a->o_ckpt = take(a->S * (size_t)a->C);
    a->o_seg = take(a->S * (size_t)std::max(1, a->K - 1));
    a->o_lam[0] = take(a->S);
    a->o_lam[1] = take(a->S);
    a->o_llam = take(L * 4);
    a->o_solid = take(N);
    a->o_lmask = take(N * 4);
    a->o_linkid = take(N * Q * 4);
    a->o_lnf = take(L * 4);
    a->o_ldir = take(L * 4);
    a->o_lnff = take(L * 4);
    a->o_lq = take(L * 4);
    a->o_dqf = take(L * 8);
    a->o_dqs = take(L * 8);
    a->o_dJdq = take(L * 8);
    a->o_cp = take((size_t)a->ncp * 24);
    a->o_K = take((size_t)a->ncp * 8);
    a->o_J = take(8);
    a->o_grad = take((size_t)a->ncp * 32);
    a->total = o;
}

void adj_sizes(lbm_adj *a, const lbm_config *c, int T, int W, int ncp, int nlinks) {
    a->cfg = *c;
    a->T = T;
    a->W = W;
    a->K = std::max(1, (int)std::ceil(std::sqrt((double)T)));
    a->C = (T + a->K - 1) / a->K;
    a->ncp = ncp;
    a->nlinks = nlinks;
    a->N = (long long)c->nx * c->ny * c->nz;
    a->S = (size_t)Q * (size_t)a->N * 4;
}

AdjDev adj_dev(lbm_adj *a) {
    AdjDev D;
    const lbm_config &c = a->cfg;
    D.c.nx = c.nx; D.c.ny = c.ny; D.c.nz = c.nz; D.c.N = a->N;
    D.c.rho0 = (float)c.rho0;
    D.c.omega = (float)(1.0 / c.tau);
    D.c.gfac = (float)(1.0 - 0.5 / c.tau);
    for (int k = 0; k < 3; k++) D.c.F[k] = (float)c.force[k];
    char *w = a->ws;
    D.solid = reinterpret_cast<const uint8_t *>(w + a->o_solid);
    D.lmask = reinterpret_cast<const uint32_t *>(w + a->o_lmask);
    D.linkid = reinterpret_cast<const int *>(w + a->o_linkid);
    D.l_nf = reinterpret_cast<const int *>(w + a->o_lnf);
    D.l_dir = reinterpret_cast<const int *>(w + a->o_ldir);
    D.l_nff = reinterpret_cast<const int *>(w + a->o_lnff);
    D.l_q = reinterpret_cast<float *>(w + a->o_lq);
    D.l_dqdMf = reinterpret_cast<double *>(w + a->o_dqf);
    D.l_dqdMs = reinterpret_cast<double *>(w + a->o_dqs);
    D.l_dJdq = reinterpret_cast<double *>(w + a->o_dJdq);
    D.l_lam = reinterpret_cast<float *>(w + a->o_llam);
    D.nlinks = a->nlinks;
    D.cp = reinterpret_cast<const double *>(w + a->o_cp);
    D.K = reinterpret_cast<const double *>(w + a->o_K);
    D.ncp = a->ncp;
    D.J_fix = reinterpret_cast<unsigned long long *>(w + a->o_J);
    D.grad = reinterpret_cast<double *>(w + a->o_grad);
    D.inv_W = 1.0f / (float)a->W;
    return D;
}

dim3 node_grid(const lbm_adj *a) {
    return dim3((a->cfg.nx + 31) / 32, (a->cfg.ny + 3) / 4, (a->cfg.nz + 1) / 2);
}

float *state(lbm_adj *a, size_t off) { return reinterpret_cast<float *>(a->ws + off); }

}  // namespace

extern "C" {

int lbm_adj_workspace_size(const lbm_config *cfg, const lbm_particle *p, int T, int W, size_t *bytes) {
    if (const char *m = adj_check(cfg, p, T, W)) return afail(nullptr, LBM_ERR_BAD_ARG, "%s", m);
    if (!bytes) return afail(nullptr, LBM_ERR_BAD_ARG, "bytes is NULL");
    std::vector<uint8_t> solid;
    std::vector<uint32_t> lmask;
    std::vector<int> nf, dir, nff;
    classify_links(cfg, p, solid, lmask, nf, dir, nff);
    lbm_adj a;
    adj_sizes(&a, cfg, T, W, p->n_cp, (int)nf.size());
    adj_layout(&a);
    *bytes = a.total;
    return LBM_OK;
}

int lbm_adj_init(const lbm_config *cfg, const lbm_particle *p, int T, int W, void *dev_ws, size_t ws_bytes,
                 void *cuda_stream, lbm_adj **out) {
    if (!out) return afail(nullptr, LBM_ERR_BAD_ARG, "out is NULL");
    *out = nullptr;
    if (const char *m = adj_check(cfg, p, T, W)) return afail(nullptr, LBM_ERR_BAD_ARG, "%s", m);
    if (!dev_ws || reinterpret_cast<uintptr_t>(dev_ws) % kAlign)
        return afail(nullptr, LBM_ERR_BAD_ARG, "workspace NULL or not 256-byte aligned");
    std::vector<uint8_t> solid;
    std::vector<uint32_t> lmask;
    std::vector<int> nf, dir, nff;
    classify_links(cfg, p, solid, lmask, nf, dir, nff);
    lbm_adj *a = new (std::nothrow) lbm_adj();
    if (!a) return afail(nullptr, LBM_ERR_BAD_ARG, "out of host memory");
    adj_sizes(a, cfg, T, W, p->n_cp, (int)nf.size());
    adj_layout(a);
    if (ws_bytes < a->total) {
        const size_t need = a->total;
        delete a;
        return afail(nullptr, LBM_ERR_WS_TOO_SMALL, "workspace of %zu bytes, %zu needed", ws_bytes, need);
    }
    a->ws = static_cast<char *>(dev_ws);
    a->stream = static_cast<cudaStream_t>(cuda_stream);
    a->have_forward = false;
    std::snprintf(a->err, sizeof(a->err), "no error");
    std::vector<int> linkid((size_t)Q * a->N, -1);
    for (size_t L = 0; L < nf.size(); L++) linkid[(size_t)dir[L] * a->N + nf[L]] = (int)L;
    const size_t Lb = nf.size() * 4;
    int rc = acheck(a, cudaMemsetAsync(a->ws, 0, a->total, a->stream), "cudaMemsetAsync");
    auto up = [&](size_t off, const void *src, size_t bytes) {
        if (rc == LBM_OK && bytes)
            rc = acheck(a, cudaMemcpyAsync(a->ws + off, src, bytes, cudaMemcpyHostToDevice, a->stream), "cudaMemcpyAsync");
    };
    up(a->o_solid, solid.data(), solid.size());
    up(a->o_lmask, lmask.data(), lmask.size() * 4);
    up(a->o_linkid, linkid.data(), linkid.size() * 4);
    up(a->o_lnf, nf.data(), Lb);
    up(a->o_ldir, dir.data(), Lb);
    up(a->o_lnff, nff.data(), Lb);
    if (rc == LBM_OK) rc = acheck(a, cudaStreamSynchronize(a->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) {
        std::snprintf(g_adj_error, sizeof(g_adj_error), "%s", a->err);
        delete a;
        return rc;
    }
    *out = a;
    return LBM_OK;
}

int lbm_adj_forward(lbm_adj *a, const double *cp_world, const double *K, double *J) {
    if (!a) return afail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (!cp_world || !K) return afail(a, LBM_ERR_BAD_ARG, "cp_world and K are required");
    for (int c = 0; c < a->ncp; c++)
        if (!(K[c] >= 0.0)) return afail(a, LBM_ERR_BAD_ARG, "negative weight");
    int rc = acheck(a, cudaMemcpyAsync(a->ws + a->o_cp, cp_world, (size_t)a->ncp * 24, cudaMemcpyHostToDevice, a->stream),
                    "cudaMemcpyAsync");
    if (rc == LBM_OK)
        rc = acheck(a, cudaMemcpyAsync(a->ws + a->o_K, K, (size_t)a->ncp * 8, cudaMemcpyHostToDevice, a->stream),
                    "cudaMemcpyAsync");
    if (rc == LBM_OK) rc = acheck(a, cudaMemsetAsync(a->ws + a->o_J, 0, 8, a->stream), "cudaMemsetAsync");
    if (rc != LBM_OK) return rc;
    const AdjDev D = adj_dev(a);
    const int lgrid = std::max(1, std::min(1024, (a->nlinks + 255) / 256));
    if (a->nlinks > 0) k_adj_q<<<lgrid, 256, 0, a->stream>>>(D);
    float *s0 = state(a, a->o_state[0]), *s1 = state(a, a->o_state[1]);
    k_adj_init<<<1216, 256, 0, a->stream>>>(D, s0, (float)a->cfg.u0[0], (float)a->cfg.u0[1], (float)a->cfg.u0[2]);
    const dim3 grid = node_grid(a);
    for (int t = 0; t < a->T; t++) {
        if (t % a->K == 0) {
            rc = acheck(a, cudaMemcpyAsync(a->ws + a->o_ckpt + (size_t)(t / a->K) * a->S, s0, a->S,
                                           cudaMemcpyDeviceToDevice, a->stream), "cudaMemcpyAsync(checkpoint)");
            if (rc != LBM_OK) return rc;
        }
        k_adj_step<<<grid, 256, 0, a->stream>>>(D, s0, s1, t >= a->T - a->W ? 1 : 0);
        std::swap(s0, s1);
    }
    long long jfix = 0;
    rc = acheck(a, cudaGetLastError(), "forward launch");
    if (rc == LBM_OK)
        rc = acheck(a, cudaMemcpyAsync(&jfix, a->ws + a->o_J, 8, cudaMemcpyDeviceToHost, a->stream), "cudaMemcpyAsync");
    if (rc == LBM_OK) rc = acheck(a, cudaStreamSynchronize(a->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) return rc;
    if (J) *J = std::ldexp((double)jfix, -kForceFixBits) / a->W;
    a->have_forward = true;
    return LBM_OK;
}

int lbm_adj_backward(lbm_adj *a, double *dJ_dcp, double *dJ_dK) {
    if (!a) return afail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (!a->have_forward) return afail(a, LBM_ERR_BAD_ARG, "no forward run to differentiate");
    const AdjDev D = adj_dev(a);
    int rc = acheck(a, cudaMemsetAsync(a->ws + a->o_dJdq, 0, (size_t)std::max(1, a->nlinks) * 8, a->stream), "cudaMemsetAsync");
    if (rc == LBM_OK) rc = acheck(a, cudaMemsetAsync(a->ws + a->o_lam[0], 0, a->S, a->stream), "cudaMemsetAsync");
    if (rc == LBM_OK) rc = acheck(a, cudaMemsetAsync(a->ws + a->o_grad, 0, (size_t)a->ncp * 32, a->stream), "cudaMemsetAsync");
    if (rc != LBM_OK) return rc;
    float *lamN = state(a, a->o_lam[0]), *lamT = state(a, a->o_lam[1]);
    const dim3 grid = node_grid(a);
    const int lgrid = std::max(1, std::min(1024, (a->nlinks + 127) / 128));
    for (int c = a->C - 1; c >= 0; c--) {
        const int t0 = c * a->K, t1 = std::min(a->T, t0 + a->K);
        // states t0 .. t1-1 of the segment: the checkpoint, then recomputed
        std::vector<float *> seg((size_t)(t1 - t0));
        seg[0] = reinterpret_cast<float *>(a->ws + a->o_ckpt + (size_t)c * a->S);
        for (int k = 1; k < t1 - t0; k++) {
            seg[(size_t)k] = reinterpret_cast<float *>(a->ws + a->o_seg + (size_t)(k - 1) * a->S);
            k_adj_step<<<grid, 256, 0, a->stream>>>(D, seg[(size_t)k - 1], seg[(size_t)k], 0);
        }
        for (int t = t1 - 1; t >= t0; t--) {
            const int window = t >= a->T - a->W ? 1 : 0;
            const float *S = seg[(size_t)(t - t0)];
            k_adj_back<<<grid, 256, 0, a->stream>>>(D, S, lamN, lamT, window);
            if (a->nlinks > 0) k_adj_vibb<<<lgrid, 128, 0, a->stream>>>(D, S, lamT);
            std::swap(lamN, lamT);
        }
    }
    if (a->nlinks > 0) k_adj_grad<<<std::max(1, std::min(256, (a->nlinks + 255) / 256)), 256, 0, a->stream>>>(D);
    std::vector<double> g((size_t)a->ncp * 4);
    rc = acheck(a, cudaGetLastError(), "adjoint launch");
    if (rc == LBM_OK)
        rc = acheck(a, cudaMemcpyAsync(g.data(), a->ws + a->o_grad, g.size() * 8, cudaMemcpyDeviceToHost, a->stream),
                    "cudaMemcpyAsync");
    if (rc == LBM_OK) rc = acheck(a, cudaStreamSynchronize(a->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) return rc;
    for (int c = 0; c < a->ncp; c++) {
        if (dJ_dcp)
            for (int k = 0; k < 3; k++) dJ_dcp[3 * c + k] = g[4 * (size_t)c + k];
        if (dJ_dK) dJ_dK[c] = g[4 * (size_t)c + 3];
    }
    return LBM_OK;
}

int lbm_adj_info(const lbm_adj *a, int *nlinks, int *checkpoint_every) {
    if (!a) return afail(nullptr, LBM_ERR_BAD_ARG, "handle is NULL");
    if (nlinks) *nlinks = a->nlinks;
    if (checkpoint_every) *checkpoint_every = a->K;
    return LBM_OK;
}

int lbm_adj_destroy(lbm_adj *a) {
    if (!a) return LBM_OK;
    cudaStreamSynchronize(a->stream);
    delete a;
    return LBM_OK;
}

const char *lbm_adj_last_error(const lbm_adj *a) { return a ? a->err : g_adj_error; }

}  // extern "C"
