// The fused lattice sweep (one CTA per 32x4x2 brick, one node per thread).
//
// For every fluid node x (flags of this step):
//   pull    f_i(x, t+1) = f+_i(x - e_i, t) from the read array (§2.2, Eq. (14));
//   walls   a source beyond a non-periodic face: halfway bounce-back
//           f_i = f+_i'(x) (resting wall);
//   links   a source inside particle j: the unknown by VIBB, Eqs. (19)-(25),
//           with q from Eq. (27) (or Eq. (26) solved by Newton's method,
//           option q_exact), or halfway bounce-back with the moving-wall
//           term when x - d is not a fluid node (§2.3.5 item 1); the
//           Galilean-invariant momentum exchange of Eqs. (28)-(29) goes to
//           particle j;
//   collide rho, u (Eq. (18) with the half-force shift), BGK toward f^eq
//           (Eqs. (15)-(16)) plus Guo's forcing term; store to the write array.
// For every solid node the missing force points of §2.3.5 item 2 (Eqs.
// (31)-(32)) are added to the particles whose surface its links cross.
//
// Bricks with no particle in their list take the plain path: 19 coalesced
// loads and 19 coalesced stores per node, no flag reads.  Per-link force and
// torque terms are accumulated per listed particle.  FP64 lattices reduce them
// across the CTA in a fixed order (warp butterfly, then warps in order) into
// FP64 partials per (brick, particle) that k_force_reduce sums in brick order;
// lattices below FP64 turn every term into 64-bit fixed point, sum it per warp
// in shared memory and add the warp's sums to the totals per particle, all
// with integer atomics (exact, so the order does not matter).
#pragma once

#include "k_flags.cuh"
#include "k_plain.cuh"

namespace lbmmb {
// Resident CTAs per SM of the near sweep: its link evaluation needs more than
// the 64 registers per thread that four 256-thread CTAs leave (it spilled to
// local memory there, and one brick's latency sets the step when few bricks
// are near), so it is compiled for two.
constexpr int kNearCtasPerSm = 2;

template <typename C>
__device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Listed slot of particle id (the list is short and ascending).
__device__ __forceinline__ int slot_of(const SmemParticles &sp, int id) {
    for (int s = 0; s < sp.n; s++)
        if (sp.id[s] == id) return s;
    return -1;
}

// Whether world node (x,y,z) + brick offset lies inside listed particle s,
// decided exactly: FP32 outside the error band, FP64 inside it.  Mval gets a
// value of M (FP32 or FP64) usable for q.
template <typename C>
__device__ __forceinline__ bool inside_exact(const Params &P, const SmemParticles &sp, int s, int lx, int ly, int lz,
                                             int bx0, int by0, int bz0, C &Mval) {
    if (sizeof(C) == 4) {
        bool unsure;
        const float M = metaball32(P, sp, s, (float)lx, (float)ly, (float)lz, unsure);
        Mval = (C)M;
        if (!unsure) return M >= P.c0_f;
    }
    const double M = metaball64(P, P.parts[sp.id[s]], (double)(bx0 + lx), (double)(by0 + ly), (double)(bz0 + lz));
    if (sizeof(C) == 8) Mval = (C)M;
    return M >= P.c0;
}

// M value for the link fraction (no exactness needed beyond the working
// precision).
template <typename C>
__device__ __forceinline__ C m_value(const Params &P, const SmemParticles &sp, int s, int lx, int ly, int lz, int bx0,
                                     int by0, int bz0) {
    if (sizeof(C) == 4) {
        bool unsure;
        return (C)metaball32(P, sp, s, (float)lx, (float)ly, (float)lz, unsure);
    }
    return (C)metaball64(P, P.parts[sp.id[s]], (double)(bx0 + lx), (double)(by0 + ly), (double)(bz0 + lz));
}

template <typename C> __device__ __forceinline__ C c0_of(const Params &P) { return sizeof(C) == 4 ? (C)P.c0_f : (C)P.c0; }

// 1 / x in the working precision: the approximate FP32 reciprocal (a link's
// arithmetic is FP32 throughout below FP64), the IEEE quotient in FP64.
template <typename C> __device__ __forceinline__ C rcp_w(C x) {
    if (sizeof(C) == 4) return (C)__fdividef(1.0f, (float)x);
    return C(1) / x;
}

// FP32 M of listed particle s at the brick-local fluid node (lx,ly,lz) and at
// the solid node one link d further, in one pass over the control points
// (minimum image taken at the fluid node; a particle spans far less than half
// the box), for the link fraction of Eq. (27), which needs no exact M.
__device__ __forceinline__ void m_link_f(const Params &P, const SmemParticles &sp, int s, int lx, int ly, int lz,
                                         int dx, int dy, int dz, float &Mf, float &Ms) {
    const float Lx = (float)P.nx, Ly = (float)P.ny, Lz = (float)P.nz;
    float a = 0.f, b = 0.f;
    const int nc = sp.ncp[s];
    for (int k = 0; k < nc; k++) {
        float ox = (float)lx - sp.crel[s][k][0];
        float oy = (float)ly - sp.crel[s][k][1];
        float oz = (float)lz - sp.crel[s][k][2];
        if (P.per[0]) { if (ox > 0.5f * Lx) ox -= Lx; else if (ox < -0.5f * Lx) ox += Lx; }
        if (P.per[1]) { if (oy > 0.5f * Ly) oy -= Ly; else if (oy < -0.5f * Ly) oy += Ly; }
        if (P.per[2]) { if (oz > 0.5f * Lz) oz -= Lz; else if (oz < -0.5f * Lz) oz += Lz; }
        const float sx = ox + (float)dx, sy = oy + (float)dy, sz = oz + (float)dz;
        const float K = sp.K[s][k];
        a += K * __fdividef(1.0f, ox * ox + oy * oy + oz * oz);
        b += K * __fdividef(1.0f, sx * sx + sy * sy + sz * sz);
    }
    Mf = a;
    Ms = b;
}

// M of listed particle s and its derivative along d at x_b + q d, x_b the
// brick-local node (lx,ly,lz): M = sum K/r^2, dM/dq = -2 sum K (r.d)/r^4.
// FP32 works on brick-relative offsets, minimum image taken at the node.
template <typename C>
__device__ __forceinline__ void m_line(const Params &P, const SmemParticles &sp, int s, int lx, int ly, int lz,
                                       int dx, int dy, int dz, int bx0, int by0, int bz0, C q, C &M, C &dM) {
    M = 0;
    dM = 0;
    if (sizeof(C) == 8) {
        const DevParticle &p = P.parts[sp.id[s]];
        for (int k = 0; k < p.ncp; k++) {
            const double r0 = minimg_d(P, 0, (double)(bx0 + lx) - p.cpw[k][0]) + (double)q * dx;
            const double r1 = minimg_d(P, 1, (double)(by0 + ly) - p.cpw[k][1]) + (double)q * dy;
            const double r2 = minimg_d(P, 2, (double)(bz0 + lz) - p.cpw[k][2]) + (double)q * dz;
            const double inv = 1.0 / (r0 * r0 + r1 * r1 + r2 * r2);
            const double t = p.K[k] * inv;
            M += (C)t;
            dM += (C)(-2.0 * t * inv * (r0 * dx + r1 * dy + r2 * dz));
        }
        return;
    }
    const float Ls[3] = {(float)P.nx, (float)P.ny, (float)P.nz};
    const int l[3] = {lx, ly, lz}, d[3] = {dx, dy, dz};
    for (int k = 0; k < sp.ncp[s]; k++) {
        float r[3];
        for (int a = 0; a < 3; a++) {
            float b = (float)l[a] - sp.crel[s][k][a];
            if (P.per[a]) { if (b > 0.5f * Ls[a]) b -= Ls[a]; else if (b < -0.5f * Ls[a]) b += Ls[a]; }
            r[a] = b + (float)q * (float)d[a];
        }
        const float inv = 1.0f / (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        const float t = sp.K[s][k] * inv;
        M += (C)t;
        dM += (C)(-2.0f * t * inv * (r[0] * d[0] + r[1] * d[1] + r[2] * d[2]));
    }
}

// Exact link fraction (§2.3.1): the root of Eq. (26), M(x_b + q d) = c0, in
// [0,1] (M(x_b) < c0 <= M(x_b + d) brackets it), by Newton's method started
// from Eq. (27)'s value q, with the tolerance 1e-7 and the cap of 100
// iterations the paper states: a Newton correction below the tolerance is
// taken and ends the iteration; a larger step that would leave the current
// bracket bisects it instead.  Below FP64 the residual is FP32, so near the
// root its sign is noise; the bracket then shrinks by bisection and the loop
// still ends within the cap.
template <typename C>
__device__ __noinline__ C q_root(const Params &P, const SmemParticles &sp, int s, int lx, int ly, int lz, int dx,
                                 int dy, int dz, int bx0, int by0, int bz0, C q) {
    const C c0 = c0_of<C>(P);
    C lo = 0, hi = 1;
    for (int it = 0; it < 100; it++) {
        C M, dM;
        m_line<C>(P, sp, s, lx, ly, lz, dx, dy, dz, bx0, by0, bz0, q, M, dM);
        const C r = M - c0;
        if (r < C(0)) lo = q; else hi = q;
        if (dM != C(0) && fabs(r / dM) < C(1e-7)) return q - r / dM;
        C qn = dM != C(0) ? q - r / dM : C(0.5) * (lo + hi);
        if (!(qn > lo && qn < hi)) qn = C(0.5) * (lo + hi);
        const C dq = qn - q;
        q = qn;
        if (fabs(dq) < C(1e-7)) break;
    }
    return q;
}

// Lever arm from particle s's centroid to the brick-local point p (minimum
// image), in the working precision.
template <typename C>
__device__ __forceinline__ void lever(const Params &P, const SmemParticles &sp, int s, int bx0, int by0, int bz0,
                                      C px, C py, C pz, C r[3]) {
    if (sizeof(C) == 8) {
        const DevParticle &p = P.parts[sp.id[s]];
        r[0] = (C)minimg_d(P, 0, bx0 + (double)px - p.x[0]);
        r[1] = (C)minimg_d(P, 1, by0 + (double)py - p.x[1]);
        r[2] = (C)minimg_d(P, 2, bz0 + (double)pz - p.x[2]);
        return;
    }
    C d[3] = {px - (C)sp.prel[s][0], py - (C)sp.prel[s][1], pz - (C)sp.prel[s][2]};
    const int Ls[3] = {P.nx, P.ny, P.nz};
    for (int a = 0; a < 3; a++) {
        if (P.per[a]) {
            const C L = (C)Ls[a];
            if (d[a] > C(0.5) * L) d[a] -= L;
            else if (d[a] < C(-0.5) * L) d[a] += L;
        }
        r[a] = d[a];
    }
}

template <typename C>
__device__ __forceinline__ void particle_velocity(const Params &P, const SmemParticles &sp, int s, const C r[3],
                                                  C uw[3]) {
    C v[3], w[3];
    if (sizeof(C) == 8) {
        const DevParticle &p = P.parts[sp.id[s]];
        for (int a = 0; a < 3; a++) { v[a] = (C)p.v[a]; w[a] = (C)p.w[a]; }
    } else {
        for (int a = 0; a < 3; a++) { v[a] = (C)sp.v[s][a]; w[a] = (C)sp.w[s][a]; }
    }
    uw[0] = v[0] + w[1] * r[2] - w[2] * r[1];
    uw[1] = v[1] + w[2] * r[0] - w[0] * r[2];
    uw[2] = v[2] + w[0] * r[1] - w[1] * r[0];
}

// Where a thread's force and torque terms go.  FP64 lattices add them to a
// per-thread array [MAXPB][6] that the CTA reduces in a fixed order.
// Lattices below FP64 turn each term into 64-bit fixed point (2^-40 lu; the
// FP32 value is kept exactly down to that unit) and add it to the warp's
// totals in shared memory with integer atomics: exact, so the result does
// not depend on the order, and no per-thread array lives in local memory.
// One link's force and torque terms in fixed point, handed back to the
// warp's link round, which sums them over the warp with integer reductions
// (exact, like the atomics) before one lane adds them to the warp's totals.
struct LinkTerms {
    int s;            // listed slot, -1: none
    long long t[6];
};
template <typename C>
struct ForceSink {
    C (*acc)[6];
    unsigned long long (*fix)[6];
    LinkTerms *defer;  // set: the terms go to *defer instead
};

// Force and torque (r x dP) of one term, and the same in 64-bit fixed point.
template <typename C>
__device__ __forceinline__ void force_terms(const C dP[3], const C r[3], C t[6]) {
    t[0] = dP[0];
    t[1] = dP[1];
    t[2] = dP[2];
    t[3] = r[1] * dP[2] - r[2] * dP[1];
    t[4] = r[2] * dP[0] - r[0] * dP[2];
    t[5] = r[0] * dP[1] - r[1] * dP[0];
}
template <typename C>
__device__ __forceinline__ unsigned long long to_fixed(C v) {
    return (unsigned long long)__float2ll_rn((float)v * (float)(1ull << kForceFixBits));
}

template <typename C>
__device__ __forceinline__ void add_term(ForceSink<C> sink, int s, const C dP[3], const C r[3]) {
    C t[6];
    force_terms<C>(dP, r, t);
    if (sizeof(C) == 8) {
#pragma unroll
        for (int c = 0; c < 6; c++) sink.acc[s][c] += t[c];
    } else if (sink.defer) {
        sink.defer->s = s;
#pragma unroll
        for (int c = 0; c < 6; c++) sink.defer->t[c] = (long long)to_fixed<C>(t[c]);
    } else {
#pragma unroll
        for (int c = 0; c < 6; c++)
            if (t[c] != C(0)) atomicAdd(&sink.fix[s][c], to_fixed<C>(t[c]));
    }
}

// The warp's link terms of one round added to its totals per listed slot:
// each 64-bit term split into 21 + 21 + 22 bits, summed over the warp with
// 32-bit reductions and put back together, which is the exact 64-bit sum
// (modulo 2^64, as the atomics).
__device__ __forceinline__ void warp_add_terms(unsigned long long (*fix)[6], int cnt, const LinkTerms &lt,
                                               int lane) {
    for (int s = 0; s < cnt; s++) {
        const bool mine = lt.s == s;
        if (!__any_sync(0xffffffffu, mine)) continue;
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const long long v = mine ? lt.t[c] : 0ll;
            const unsigned lo = (unsigned)v & 0x1FFFFFu, mid = (unsigned)(v >> 21) & 0x1FFFFFu;
            const int hi = (int)(v >> 42);
            const unsigned long long sum =
                (unsigned long long)__reduce_add_sync(0xffffffffu, lo) +
                ((unsigned long long)__reduce_add_sync(0xffffffffu, mid) << 21) +
                ((unsigned long long)(long long)__reduce_add_sync(0xffffffffu, hi) << 42);
            if (lane == 0) fix[s][c] += sum;
        }
    }
}

// The second fluid node x_ff = x - d of a link (d = e_io, into the solid):
// whether it is a fluid node inside the box, and, for VIBB, the density
// offset, momentum and the io population of its post-collision state.  Its
// flag and populations are fetched together (beyond a wall the address is
// clamped to x itself, whose values are then not used).
template <typename C>
struct FFData {
    C drho, m[3], g_io;
    bool ok;
};
template <typename S, int Q>
__device__ __forceinline__ FFData<typename Codec<S>::C> ff_fetch(const Params &P, int x, int y, int z, int io) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const int dx = lat_e<Q>(io, 0), dy = lat_e<Q>(io, 1), dz = lat_e<Q>(io, 2);
    int fx = x - dx, fy = y - dy, fz = z - dz;
    bool ff_in = true;
    if (fx < 0 || fx >= P.nx) { if (P.per[0]) fx = (fx + P.nx) % P.nx; else ff_in = false; }
    if (fy < 0 || fy >= P.ny) { if (P.per[1]) fy = (fy + P.ny) % P.ny; else ff_in = false; }
    if (fz < 0 || fz >= P.nz) { if (P.per[2]) fz = (fz + P.nz) % P.nz; else ff_in = false; }
    const int nff = ff_in ? fx + P.nx * (fy + P.ny * fz) : x + P.nx * (y + P.ny * z);
    const uint16_t flag_ff = P.flag_new[nff];
    FFData<C> f;
    f.drho = 0;
    f.m[0] = f.m[1] = f.m[2] = 0;
    f.g_io = 0;
    if (P.vibb) {
        const S *A = (const S *)P.fA;
        const C rho0 = Prm<C>::rho0(P);
#pragma unroll
        for (int k = 0; k < Q; k++) {
            const C fk = Cd::ld(A + (long long)k * P.N + nff, (C)L::w(k), rho0);
            f.drho += fk;
            f.m[0] += fk * L::e(k, 0);
            f.m[1] += fk * L::e(k, 1);
            f.m[2] += fk * L::e(k, 2);
            if (k == io) f.g_io = fk;
        }
    }
    f.ok = ff_in && flag_ff == 0;
    return f;
}

// Geometry of one particle link (direction i arrives at x from the solid node
// x + d, d = -e_i, of listed particle slot s): the link fraction q of Eq. (27)
// (clamped to [0,1]: rounding can push it past the ends; or Eq. (26) by
// Newton with q_exact), the lever arm r from the particle's centroid to the
// wall point x_w = x + q d and the wall velocity u_w there.  M_j(x_f) is
// shared by all links of the node to the same particle (Mf_cache).
template <typename C>
struct LinkGeom {
    C q, r[3], uw[3];
};
template <typename S, int Q>
__device__ __forceinline__ LinkGeom<typename Codec<S>::C> link_geometry(const Params &P, const SmemParticles &sp,
                                                                       int i, int s, int lx, int ly, int lz, int bx0,
                                                                       int by0, int bz0,
                                                                       typename Codec<S>::C *Mf_cache,
                                                                       int *Mf_slot) {
    using L = Lat<Q>;
    using C = typename Codec<S>::C;
    const int io = L::opp(i);
    const int dx = lat_e<Q>(io, 0), dy = lat_e<Q>(io, 1), dz = lat_e<Q>(io, 2);  // d, into the solid
    C Mf, Ms;
    if (sizeof(C) == 4) {
        float mf, ms;
        m_link_f(P, sp, s, lx, ly, lz, dx, dy, dz, mf, ms);
        Mf = (C)mf;
        Ms = (C)ms;
    } else {
        if (*Mf_slot != s) {
            *Mf_cache = m_value<C>(P, sp, s, lx, ly, lz, bx0, by0, bz0);
            *Mf_slot = s;
        }
        Mf = *Mf_cache;
        Ms = m_value<C>(P, sp, s, lx + dx, ly + dy, lz + dz, bx0, by0, bz0);
    }
    LinkGeom<C> g;
    C q = sizeof(C) == 4 ? (c0_of<C>(P) - Mf) * rcp_w<C>(Ms - Mf) : (c0_of<C>(P) - Mf) / (Ms - Mf);
    q = q > C(0) ? (q < C(1) ? q : C(1)) : C(0);  // (a NaN from Ms == Mf becomes 0)
    if (P.q_exact) q = q_root<C>(P, sp, s, lx, ly, lz, dx, dy, dz, bx0, by0, bz0, q);
    g.q = q;
    lever<C>(P, sp, s, bx0, by0, bz0, (C)lx + q * dx, (C)ly + q * dy, (C)lz + q * dz, g.r);
    particle_velocity<C>(P, sp, s, g.r, g.uw);
    return g;
}

// The unknown population of a particle link of geometry g and its
// momentum-exchange term dP, in offset form: fown_io is the node's
// post-collision offset g = f - w rho0 along d, drho_f = rho_f - rho0, u_f its
// velocity, ff the second fluid node x_ff = x - d, and the unknown is
// returned as an offset.  Eq. (28)'s term is (d - u_w) f+_d + (d + u_w) f_-d =
// 2 d w rho0 + (d - u_w) g+_d + (d + u_w) g_-d; the constant 2 d w rho0 sums
// to exactly zero over all links that cross a particle's surface (those of
// Eq. (28) and the missing force points of §2.3.5 together: every pair of
// solid nodes of the particle cancels), and so does its torque
// (x_s - x_p) x 2 d w rho0, so both are left out unless the missing force
// points are switched off.
template <typename S, int Q>
__device__ __forceinline__ typename Codec<S>::C link_update(const Params &P, int i,
                                                           const LinkGeom<typename Codec<S>::C> &g,
                                                           const FFData<typename Codec<S>::C> &ff,
                                                           typename Codec<S>::C fown_io,
                                                           typename Codec<S>::C drho_f,
                                                           const typename Codec<S>::C *u_f,
                                                           typename Codec<S>::C dP[3]) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const int io = L::opp(i);
    const int dx = lat_e<Q>(io, 0), dy = lat_e<Q>(io, 1), dz = lat_e<Q>(io, 2);  // d, into the solid
    const C w_io = (C)lat_w<Q>(io);
    const C rho0 = Prm<C>::rho0(P);
    const C q = g.q;
    const C *uw = g.uw;
    const C eu_w = -(dx * uw[0] + dy * uw[1] + dz * uw[2]);  // e_i . u_w with e_i = -d
    const C rho_f = rho0 + drho_f;
    const C drho_ff = ff.drho, m_ff[3] = {ff.m[0], ff.m[1], ff.m[2]}, fff_io = ff.g_io;
    const bool ff_ok = ff.ok;
    C fin;
    if (!P.vibb || !ff_ok) {
        fin = fown_io + C(6) * w_io * rho_f * eu_w;
    } else {
        C u_ff[3];
        const C rho_ff = rho0 + drho_ff;
        const C inv_rho_ff = rcp_w<C>(rho_ff);
        for (int a = 0; a < 3; a++) u_ff[a] = (m_ff[a] - C(0.5) * Prm<C>::F(P, a)) * inv_rho_ff;
        const C feq_f = geq_i<C>(dx, dy, dz, w_io, drho_f, rho_f, u_f[0], u_f[1], u_f[2]);
        const C feq_ff = geq_i<C>(dx, dy, dz, w_io, drho_ff, rho_ff, u_ff[0], u_ff[1], u_ff[2]);
        // Eq. (21): non-equilibrium part, interpolated (q <= 1/2) or
        // extrapolated (q > 1/2) from x_f and x_ff
        const C fneq_d = C(2) * q * (fown_io - feq_f) + (C(1) - C(2) * q) * (fff_io - feq_ff);
        C drho_d, us[3], uss[3], ud[3];
        if (q <= C(0.5)) {  // Eqs. (22)-(23), first branches
            drho_d = C(2) * q * drho_f + (C(1) - C(2) * q) * drho_ff;
            for (int a = 0; a < 3; a++) us[a] = C(2) * q * u_f[a] + (C(1) - C(2) * q) * u_ff[a];
        } else {            // second branches
            drho_d = drho_f;
            const C inv_q = rcp_w<C>(q);
            const C a_f = (C(1) - q) * inv_q, a_w = (C(2) * q - C(1)) * inv_q;
            for (int a = 0; a < 3; a++) us[a] = a_f * u_f[a] + a_w * uw[a];
        }
        const C inv_1q = rcp_w<C>(C(1) + q);
        const C b_ff = (C(1) - q) * inv_1q, b_w = C(2) * q * inv_1q;
        for (int a = 0; a < 3; a++) uss[a] = b_ff * u_ff[a] + b_w * uw[a];                 // (24)
        for (int a = 0; a < 3; a++) ud[a] = (us[a] + C(2) * uss[a]) * C(1.0 / 3.0);        // (25)
        const C fplus_d = geq_i<C>(dx, dy, dz, w_io, drho_d, rho0 + drho_d, ud[0], ud[1], ud[2]) + fneq_d;        // (20)
        fin = fplus_d + C(6) * w_io * rho_f * eu_w;                                                              // (19)
    }
    // Eq. (28): (e_i' - u_w) f+_i'(x,t) - (e_i - u_w) f_i(x,t+1), e_i' = d,
    // in offsets (the constant part left out, see above)
    dP[0] = (C(dx) - uw[0]) * fown_io + (C(dx) + uw[0]) * fin;
    dP[1] = (C(dy) - uw[1]) * fown_io + (C(dy) + uw[1]) * fin;
    dP[2] = (C(dz) - uw[2]) * fown_io + (C(dz) + uw[2]) * fin;
    if (!P.missing_force) {
        const C c = C(2) * w_io * rho0;
        dP[0] += c * dx; dP[1] += c * dy; dP[2] += c * dz;
    }
    return fin;
}

// One particle link of listed particle j at node x: its geometry, its
// unknown and its momentum-exchange term added to the sink.
template <typename S, int Q>
__device__ __forceinline__ typename Codec<S>::C particle_link(const Params &P, const SmemParticles &sp, int i, int x,
                                                             int y, int z, int lx, int ly, int lz, int bx0, int by0,
                                                             int bz0, int j, const FFData<typename Codec<S>::C> &ff,
                                                             typename Codec<S>::C fown_io,
                                                             typename Codec<S>::C drho_f,
                                                             const typename Codec<S>::C *u_f,
                                                             ForceSink<typename Codec<S>::C> sink,
                                                             typename Codec<S>::C *Mf_cache, int *Mf_slot) {
    using C = typename Codec<S>::C;
    const int s = slot_of(sp, j);
    if (s < 0) {  // cannot happen for a consistent brick list; bounce back plainly
        atomicOr(&P.status[ST_ERR], ERRB_BRICK_OVERFLOW);
        return fown_io;
    }
    const LinkGeom<C> g = link_geometry<S, Q>(P, sp, i, s, lx, ly, lz, bx0, by0, bz0, Mf_cache, Mf_slot);
    C dP[3];
    const C fin = link_update<S, Q>(P, i, g, ff, fown_io, drho_f, u_f, dP);
    add_term<C>(sink, s, dP, g.r);
    return fin;
}

// Missing force points at a solid node (§2.3.5 item 2).  Reading: a link
// y -> x_s = y + d crossing particle j's surface (M_j(y) < c0 <= M_j(x_s))
// is seen by Eq. (28) when y is a fluid node and x_s is owned by j; every
// other crossing link (y covered by another particle or beyond a wall, or
// x_s inside j but owned by another particle) is a missing force point and
// gets Eqs. (31)-(32) with f^eq(rho0, u_w).  The caller passes the candidate
// directions of listed particle s (those whose neighbour y = x - d is not a
// fluid node of j's or j's own node): this evaluates them.
template <typename S, int Q>
__device__ __noinline__ int solid_links(const Params &P, const SmemParticles &sp, int s, bool owner, uint32_t cand,
                                        int lx, int ly, int lz, int bx0, int by0, int bz0,
                                        ForceSink<typename Codec<S>::C> sink) {
    using C = typename Codec<S>::C;
    const C rho0 = Prm<C>::rho0(P);
    int terms = 0;
    C Ms;
    if (owner) {
        Ms = m_value<C>(P, sp, s, lx, ly, lz, bx0, by0, bz0);
    } else if (!inside_exact<C>(P, sp, s, lx, ly, lz, bx0, by0, bz0, Ms)) {
        return 0;
    }
    while (cand) {
        const int i = __ffs(cand) - 1;
        cand &= cand - 1;
        const int dx = lat_e<Q>(i, 0), dy = lat_e<Q>(i, 1), dz = lat_e<Q>(i, 2);
        C My;
        if (inside_exact<C>(P, sp, s, lx - dx, ly - dy, lz - dz, bx0, by0, bz0, My)) continue;
        C q = (c0_of<C>(P) - My) / (Ms - My);
        q = q < C(0) ? C(0) : (q > C(1) ? C(1) : q);
        if (P.q_exact) q = q_root<C>(P, sp, s, lx - dx, ly - dy, lz - dz, dx, dy, dz, bx0, by0, bz0, q);
        C r[3], uw[3];
        lever<C>(P, sp, s, bx0, by0, bz0, (C)(lx - dx) + q * dx, (C)(ly - dy) + q * dy, (C)(lz - dz) + q * dz, r);
        particle_velocity<C>(P, sp, s, r, uw);
        const C w = (C)lat_w<Q>(i);
        // Eqs. (31)-(32) in offsets; the constant 2 d w rho0 cancels
        // with those of the other crossing links (see particle_link)
        const C fi = geq_i<C>(dx, dy, dz, w, C(0), rho0, uw[0], uw[1], uw[2]);
        const C fo = geq_i<C>(-dx, -dy, -dz, w, C(0), rho0, uw[0], uw[1], uw[2]);
        C dP[3];
        dP[0] = (C(dx) - uw[0]) * fi + (C(dx) + uw[0]) * fo;
        dP[1] = (C(dy) - uw[1]) * fi + (C(dy) + uw[1]) * fo;
        dP[2] = (C(dz) - uw[2]) * fi + (C(dz) + uw[2]) * fo;
        add_term<C>(sink, s, dP, r);
        terms++;
    }
    return terms;
}

// The unknown of one particle link, computed by any lane of the warp: the
// node's (brick-local lx,ly,lz) own post-collision populations, the owner of
// the solid node and x_ff's flag and populations are all fetched in one
// round, then the link is evaluated as in particle_link.
template <typename S, int Q>
__device__ __noinline__ typename Codec<S>::C link_coop(const Params &P, const SmemParticles &sp, int i, int lx, int ly,
                                                      int lz, int bx0, int by0, int bz0,
                                                      ForceSink<typename Codec<S>::C> sink) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const int x = bx0 + lx, y = by0 + ly, z = bz0 + lz;
    const int n = x + P.nx * (y + P.ny * z);
    const S *A = (const S *)P.fA;
    const long long N = P.N;
    const C rho0 = Prm<C>::rho0(P);
    // the solid source x - e_i (inside the domain: the link exists) and its
    // owner; x_ff
    int sx = x - lat_e<Q>(i, 0), sy = y - lat_e<Q>(i, 1), sz = z - lat_e<Q>(i, 2);
    if (sx < 0) sx += P.nx; else if (sx >= P.nx) sx -= P.nx;
    if (sy < 0) sy += P.ny; else if (sy >= P.ny) sy -= P.ny;
    if (sz < 0) sz += P.nz; else if (sz >= P.nz) sz -= P.nz;
    const int j = (int)P.flag_new[sx + P.nx * (sy + P.ny * sz)] - 1;
    const int io = L::opp(i);
    const FFData<C> ff = ff_fetch<S, Q>(P, x, y, z, io);
    // moments of the node's post-collision populations, and the one along
    // d = -e_i (picked in the unrolled loop, so nothing is indexed at run time)
    C fown_io = 0;
    C drho_f = 0, m_f[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const C fk = Cd::ld(A + (long long)k * N + n, (C)L::w(k), rho0);
        drho_f += fk;
        m_f[0] += fk * L::e(k, 0);
        m_f[1] += fk * L::e(k, 1);
        m_f[2] += fk * L::e(k, 2);
        if (k == io) fown_io = fk;
    }
    C u_f[3];
    const C inv_rho_f = rcp_w<C>(rho0 + drho_f);
    for (int a = 0; a < 3; a++) u_f[a] = (m_f[a] - C(0.5) * Prm<C>::F(P, a)) * inv_rho_f;
    C Mf_cache = 0;
    int Mf_slot = -1;
    return particle_link<S, Q>(P, sp, i, x, y, z, lx, ly, lz, bx0, by0, bz0, j, ff, fown_io, drho_f, u_f, sink,
                               &Mf_cache, &Mf_slot);
}

// Shared scratch of the warp-cooperative link evaluation: per warp a queue of
// (lane, direction) link entries and their results.
constexpr int kLinkQueue = 32 * 18;
struct LinkScratch {
    unsigned short entry[BRICK / 32][kLinkQueue];
    float result[BRICK / 32][kLinkQueue];
    unsigned long long fix[BRICK / 32][MAXPB][6];  // the warp's fixed-point force/torque terms
};

// A fluid node with at least one particle link, in a brick some particle
// reaches: pull, walls, VIBB / halfway bounce-back on the particle links with
// their momentum exchange, collide, store.
template <typename S, int Q, bool kForce>
__device__ __noinline__ void boundary_node(const Params &P, const SmemParticles &sp, int x, int y, int z, int lx,
                                           int ly, int lz, int bx0, int by0, int bz0, int n,
                                           ForceSink<typename Codec<S>::C> sink, int *nlinks) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const S *A = (const S *)P.fA;
    S *B = (S *)P.fB;
    const long long N = P.N;
    const C rho0 = Prm<C>::rho0(P);
    int xs[3], ys[3], zs[3];
    neighbour_coords(P, x, y, z, xs, ys, zs);
    C fown[Q];
    C drho_f = 0, m_f[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < Q; k++) {
        fown[k] = Cd::ld(A + (long long)k * N + n, (C)L::w(k), rho0);
        drho_f += fown[k];
        m_f[0] += fown[k] * L::e(k, 0);
        m_f[1] += fown[k] * L::e(k, 1);
        m_f[2] += fown[k] * L::e(k, 2);
    }
    C u_f[3];
    const C inv_rho_f = C(1) / (rho0 + drho_f);
    for (int a = 0; a < 3; a++) u_f[a] = (m_f[a] - C(0.5) * Prm<C>::F(P, a)) * inv_rho_f;
    C fin[Q];
    int srcs[Q];
    uint32_t links = 0;
    fin[0] = fown[0];
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const int sx = xs[1 - L::e(i, 0)], sy = ys[1 - L::e(i, 1)], sz = zs[1 - L::e(i, 2)];
        if ((sx | sy | sz) < 0) {
            fin[i] = fown[L::opp(i)];  // box wall: halfway bounce-back
            srcs[i] = n;
            continue;
        }
        const int src = sx + P.nx * (sy + P.ny * sz);
        srcs[i] = src;
        fin[i] = Cd::ld(A + (long long)i * N + src, (C)L::w(i), rho0);
        if (P.flag_new[src] != 0) links |= 1u << i;
    }
    // each thread visits its own links only, so a warp runs as many link
    // updates as its busiest node has links
    C Mf_cache = 0;
    int Mf_slot = -1;
    while (links) {
        const int i = __ffs(links) - 1;
        links &= links - 1;
        const FFData<C> ff = ff_fetch<S, Q>(P, x, y, z, L::opp(i));
        fin[i] = particle_link<S, Q>(P, sp, i, x, y, z, lx, ly, lz, bx0, by0, bz0, (int)P.flag_new[srcs[i]] - 1, ff,
                                     fown[L::opp(i)], drho_f, u_f, sink, &Mf_cache, &Mf_slot);
        (*nlinks)++;
    }
#pragma unroll
    for (int i = 0; i < Q; i++) fin[i] = Cd::g_to_v(fin[i], (C)L::w(i));
    collide_store<S, Q, kForce>(P, fin, B, N, n);
}

// Bricks some particle reaches: nodes without particle links take the plain
// path (plus 19 flag reads); boundary and solid nodes go out of line; then
// the deterministic reduction of the per-particle terms.
template <typename S, int Q, bool kForce>
__device__ __noinline__ void near_brick(const Params &P, SmemParticles &sp, double (*red)[6], int *s_links,
                                        LinkScratch *ls, int b, int bx0, int by0, int bz0, int cnt) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lx = tid % BX, ly = (tid / BX) % BY, lz = tid / (BX * BY);
    const int x = bx0 + lx, y = by0 + ly, z = bz0 + lz;
    const bool active = x < P.nx && y < P.ny && z < P.nz;
    const long long N = P.N;
    const int n = x + P.nx * (y + P.ny * z);
    const S *A = (const S *)P.fA;
    S *B = (S *)P.fB;
    const C rho0 = Prm<C>::rho0(P);

    C acc[MAXPB][6];  // FP64 only
    const ForceSink<C> sink{acc, ls->fix[warp]};
    if (sizeof(C) == 8) {
        for (int s = 0; s < cnt; s++)
            for (int c = 0; c < 6; c++) acc[s][c] = 0;
    } else {
        for (int e = lane; e < cnt * 6; e += 32) ls->fix[warp][e / 6][e % 6] = 0ull;
        __syncwarp();
    }
    int nlinks = 0;

    // the node's flag and its neighbours' (y = x - e_i; kWall beyond a wall),
    // read in one round by fluid and solid nodes alike and issued before the
    // brick's particles are loaded, so the two latencies overlap
    constexpr uint32_t kWall = 0xFFFFFFFFu;
    uint32_t nf[Q];
    C fin[Q];
    {
        int xs[3], ys[3], zs[3];
        neighbour_coords(P, x, y, z, xs, ys, zs);
        nf[0] = active ? (uint32_t)P.flag_new[n] : 1u;
#pragma unroll
        for (int i = 1; i < Q; i++) {
            const int sx = xs[1 - L::e(i, 0)], sy = ys[1 - L::e(i, 1)], sz = zs[1 - L::e(i, 2)];
            const bool wall = (sx | sy | sz) < 0;
            nf[i] = (!active || wall) ? kWall : (uint32_t)P.flag_new[sx + P.nx * (sy + P.ny * sz)];
        }
        if (sizeof(C) == 8 && active) {  // FP64: the pulls in the same round
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const int sx = xs[1 - L::e(i, 0)], sy = ys[1 - L::e(i, 1)], sz = zs[1 - L::e(i, 2)];
                const bool wall = (sx | sy | sz) < 0;
                const S *ptr = wall ? A + (long long)L::opp(i) * N + n
                                    : A + (long long)i * N + (sx + P.nx * (sy + P.ny * sz));
                fin[i] = Cd::ld(ptr, (C)L::w(i), rho0);
            }
        }
    }
    load_particle_records(P, sp, cnt, bx0, by0, bz0);  // ids staged by the caller
    const bool fluid = active && nf[0] == 0;
    uint32_t links = 0;
    if (fluid) {
#pragma unroll
        for (int i = 1; i < Q; i++)
            if (nf[i] != 0 && nf[i] != kWall) links |= 1u << i;
    }
    int nterms = 0;  // missing-force-point terms this thread added
    if (active && !fluid && P.missing_force) {
        // per listed particle j, the directions whose neighbour is neither a
        // fluid node next to j's own node nor a node of j
        const int owner = (int)nf[0] - 1;
        for (int s = 0; s < sp.n; s++) {
            const int j = sp.id[s];
            // a node outside another particle's bounding sphere is not inside
            // it: solid_links would find nothing
            if (j != owner && !in_bound(P, sp, s, lx, ly, lz)) continue;
            uint32_t cand = 0;
#pragma unroll
            for (int i = 1; i < Q; i++) {
                const bool seen = (nf[i] == 0 && j == owner) || nf[i] == (uint32_t)(j + 1);
                if (!seen) cand |= 1u << i;
            }
            if (cand) nterms += solid_links<S, Q>(P, sp, s, j == owner, cand, lx, ly, lz, bx0, by0, bz0, sink);
        }
    }
    if (sizeof(C) == 8) {
        // FP64 storage: every node evaluates its own links
        if (links) boundary_node<S, Q, kForce>(P, sp, x, y, z, lx, ly, lz, bx0, by0, bz0, n, sink, &nlinks);
        else if (fluid) {
#pragma unroll
            for (int i = 0; i < Q; i++) fin[i] = Cd::g_to_v(fin[i], (C)L::w(i));
            collide_store<S, Q, kForce>(P, fin, B, N, n);
        }
    } else {
        // the warp's links in a queue (lane order, then direction order);
        // all 32 lanes evaluate them, then each node takes its results back
        const int mine = __popc(links);
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int first = incl - mine;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        {
            uint32_t m = links;
            for (int k = first; m; k++) {
                const int i = __ffs(m) - 1;
                m &= m - 1;
                ls->entry[warp][k] = (unsigned short)((lane << 5) | i);
            }
        }
        __syncwarp();
        // rounds of 32 links; each round's force terms are summed over the
        // warp (no per-link atomics on the warp's totals)
        for (int r = 0; r < total; r += 32) {
            const int e = r + lane;
            LinkTerms lt;
            lt.s = -1;
            if (e < total) {
                const int ent = ls->entry[warp][e];
                const int L_ = ent >> 5, i = ent & 31;
                const int t = warp * 32 + L_;  // the node's thread index in the brick
                ForceSink<C> ds = sink;
                ds.defer = &lt;
                ls->result[warp][e] = (float)link_coop<S, Q>(P, sp, i, t % BX, (t / BX) % BY, t / (BX * BY), bx0,
                                                             by0, bz0, ds);
                nlinks++;
            }
            warp_add_terms(ls->fix[warp], cnt, lt, lane);
        }
        __syncwarp();
        if (fluid) {
            // pull after the link evaluation: populations held across the
            // out-of-line link calls would be spilled around them
            int xs[3], ys[3], zs[3];
            neighbour_coords(P, x, y, z, xs, ys, zs);
            int k = first;
#pragma unroll
            for (int i = 0; i < Q; i++) {
                if (links & (1u << i)) {  // link results are offsets g
                    fin[i] = Cd::g_to_v((C)ls->result[warp][k], (C)L::w(i));
                    k++;
                } else {
                    const int sx = xs[1 - L::e(i, 0)], sy = ys[1 - L::e(i, 1)], sz = zs[1 - L::e(i, 2)];
                    const bool wall = (sx | sy | sz) < 0;
                    const S *ptr = wall ? A + (long long)L::opp(i) * N + n
                                        : A + (long long)i * N + (sx + P.nx * (sy + P.ny * sz));
                    fin[i] = Cd::ldv(ptr, (C)L::w(i), rho0);
                }
            }
            collide_store<S, Q, kForce>(P, fin, B, N, n);  // collide-space values
        }
    }

    if (sizeof(C) == 4) {
        // the warp's fixed-point totals go to the particles' totals with
        // integer atomics (exact, order-independent, no barrier); a warp that
        // evaluated no link and no missing force point has nothing to add
        if (__any_sync(0xffffffffu, nlinks > 0 || nterms > 0)) {
            __syncwarp();
            for (int e = lane; e < cnt * 6; e += 32) {
                const unsigned long long v = ls->fix[warp][e / 6][e % 6];
                if (v) atomicAdd(&P.Ffix[sp.id[e / 6] * 6 + e % 6], v);
            }
        }
        const int nl = __reduce_add_sync(0xffffffffu, (unsigned)nlinks);
        if (lane == 0 && nl) atomicAdd(&P.counters[CNT_NLINKS], nl);
    } else {
        // deterministic CTA reduction of the per-particle terms
        for (int s = 0; s < cnt; s++) {
            for (int c = 0; c < 6; c++) {
                C v = acc[s][c];
                v = warp_sum<C>(v);
                if (lane == 0) red[warp][c] = (double)v;
            }
            __syncthreads();
            if (tid < 6) {
                double t = 0.0;
                for (int w = 0; w < BRICK / 32; w++) t += red[w][tid];
                P.partial[((long long)b * MAXPB + s) * 6 + tid] = t;
            }
            __syncthreads();
        }
        const int nl = __reduce_add_sync(0xffffffffu, (unsigned)nlinks);
        if (lane == 0 && nl) atomicAdd(s_links, nl);
        __syncthreads();
        if (tid == 0 && *s_links) atomicAdd(&P.counters[CNT_NLINKS], *s_links);
    }
}

// Whether a brick of the near set can hold a particle link or a missing
// force point: it needs a solid node in the brick or a solid neighbour of one
// of its nodes -- the brick's own mark, and for each of the 26 bricks around
// it the faces turned towards it (all of them, for an edge or corner brick).
// Called by every thread of the CTA (a barrier); the same answer in all.
__device__ __forceinline__ bool brick_near_solid(const Params &P, int bxi, int byi, int bzi) {
    const int tid = threadIdx.x;
    bool near_solid = false;
    if (tid < 27) {
        const int o[3] = {tid % 3 - 1, (tid / 3) % 3 - 1, tid / 9 - 1};
        int q[3] = {bxi + o[0], byi + o[1], bzi + o[2]};
        const int nbs[3] = {P.nbx, P.nby, P.nbz};
        bool in = true;
        for (int a = 0; a < 3; a++) {
            if (q[a] < 0 || q[a] >= nbs[a]) {
                if (P.per[a]) q[a] = (q[a] + nbs[a]) % nbs[a];
                else in = false;
            }
        }
        const uint32_t m = in ? (uint32_t)P.brick_solid[q[0] + P.nbx * (q[1] + P.nby * q[2])] : 0u;
        near_solid = (m & kSolidAny) != 0;
        for (int a = 0; a < 3; a++)  // a brick below faces us with its high face, and so on
            if (o[a] != 0) near_solid = near_solid && (m & (1u << (2 * a + (o[a] < 0 ? 1 : 0)))) != 0;
    }
    return __syncthreads_or(near_solid) != 0;
}

// The sweep of the bricks listed this step (exactly those some particle's
// grown search box meets) and of the predicted-near bricks that are not
// listed: every brick k_sweep_plain leaves.  A brick of this set that can
// hold no particle link (no particle listed, or no solid node next to it)
// takes the plain path, here (kSplit false: the batched sweep), or (kSplit
// true) it is appended to the step's list for k_sweep_near_plain, which runs
// after this kernel on the plain sweep's stream at the plain sweep's
// occupancy, while this kernel keeps its CTAs for the link bricks.
// Persistent grid;
// the CTAs take the bricks one at a time from a per-step counter (a brick
// with particle links costs about ten times one on the plain path, and a
// fixed split left the busiest CTA near 1.45 times the mean).  Thread 0
// fetches the next entry while the current brick runs; s_next holds it,
// alternating between two slots so that a slot is rewritten only after
// every thread has passed the barrier that follows its last read.
template <typename S, int Q, bool kForce, bool kSplit = false>
__device__ __forceinline__ void near_work(const Params &P, SmemParticles &sp, double (*red)[6], int &s_links,
                                          LinkScratch &ls, int *s_next) {
    const int tid = threadIdx.x;
    const int t = P.step;
    const int c_exact = P.counters[CNT_LISTED];
    const int c_pred = P.pred_stamp_cur ? P.pred_count[t % 3] : 0;
    const int total = c_exact + c_pred;
    int done = 0;
    int nxt = 0;
    if (tid == 0) nxt = atomicAdd(&P.counters[CNT_NEAR_NEXT], 1);
    for (int k = 0;; k ^= 1) {
        if (tid == 0) s_next[k] = nxt;
        __syncthreads();  // the previous brick is done with the shared state
        const int w = s_next[k];
        if (w >= total) break;
        if (tid == 0) nxt = atomicAdd(&P.counters[CNT_NEAR_NEXT], 1);
        int b;
        if (w < c_exact) {
            b = P.wl_list[(t % 3) * P.nbricks + w];
        } else {
            b = P.pred_list_cur[w - c_exact];
            if (P.stamp[b] == t) continue;  // listed: taken above
        }
        int bxi, byi, bzi;
        brick_coords(P, b, bxi, byi, bzi);
        const int bx0 = bxi * BX, by0 = byi * BY, bz0 = bzi * BZ;
        int cnt = min(P.bcount[b], MAXPB);
        // the brick's particle ids, staged with the neighbourhood check below
        // (made visible by its barrier)
        if (tid >= 32 && tid < 32 + cnt) sp.id[tid - 32] = P.blist[b * MAXPB + (tid - 32)];
        if (tid == 0) sp.n = cnt;
        if (cnt > 0 && P.brick_solid) {
            if (!brick_near_solid(P, bxi, byi, bzi)) cnt = 0;
        } else {
            __syncthreads();
        }
        done++;
        if (cnt == 0) {
            if (kSplit) {  // k_sweep_near_plain takes it (each brick is listed once a step)
                if (tid == 0) P.np_list[atomicAdd(P.np_count, 1)] = b;
                continue;
            }
            const int x = bx0 + tid % BX, y = by0 + (tid / BX) % BY, z = bz0 + tid / (BX * BY);
            if (x < P.nx && y < P.ny && z < P.nz) plain_node<S, Q, kForce>(P, x, y, z, x + P.nx * (y + P.ny * z));
            continue;
        }
        if (tid == 0) s_links = 0;
        near_brick<S, Q, kForce>(P, sp, red, &s_links, &ls, b, bx0, by0, bz0, cnt);
    }
    if (tid == 0 && done) atomicAdd(&P.counters[CNT_NEAR], done);
}
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, kNearCtasPerSm) k_sweep_near(Params P) {
    __shared__ SmemParticles sp;
    __shared__ double red[BRICK / 32][6];
    __shared__ int s_links;
    __shared__ LinkScratch ls;
    __shared__ int s_next[2];
    near_work<S, Q, kForce, true>(P, sp, red, s_links, ls, s_next);
}

// The bricks of the near set that hold no particle link, as the near sweep
// listed them (np_list, np_count: this step's parity): the plain path, one
// brick per CTA at a time over a persistent grid, on the plain sweep's stream
// after the near sweep.  It reads nothing else of the step's lists, so the
// next step's binning and flag pass (which rewrite them) may run beside it.
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, 4) k_sweep_near_plain(Params P) {
    const int tid = threadIdx.x;
    const int total = *P.np_count;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int b = P.np_list[w];
        int bxi, byi, bzi;
        brick_coords(P, b, bxi, byi, bzi);
        const int x = bxi * BX + tid % BX, y = byi * BY + (tid / BX) % BY, z = bzi * BZ + tid / (BX * BY);
        if (x < P.nx && y < P.ny && z < P.nz) plain_node<S, Q, kForce>(P, x, y, z, x + P.nx * (y + P.ny * z));
    }
}

}  // namespace lbmmb
