// The plain path of the lattice sweep (§2.2, Eqs. (14)-(18)): bricks that no
// particle reaches.  One CTA per 32x4x2 brick, one node per thread: 19
// coalesced pulls (a source beyond a non-periodic face gives halfway
// bounce-back, the node's own opposite population), BGK toward f^eq with
// Guo's forcing term, 19 coalesced stores.  No flags are read.  Populations
// are held as offsets g = f - w rho0 (see the codecs), and loads and stores
// carry evict-first hints: the arrays cannot stay in L2 until the next step.
// The near sweep (k_sweep.cuh) reuses collide_store and plain_node.
#pragma once

#include "lbm_internal.cuh"

namespace lbmmb {

// e . v over the nonzero components of a lattice direction, taken in x, y, z
// order.  The zero components are left out rather than multiplied: x * 0 is
// not folded away under IEEE rules, and for D3Q19 that is 27 of the 57 terms
// of each sum over directions.  The sum is the same (up to the sign of a zero
// result) as e_x v_x + e_y v_y + e_z v_z evaluated left to right.
template <typename C>
__device__ __forceinline__ C dot_e(int ex, int ey, int ez, C vx, C vy, C vz) {
    C s = C(0);
    bool any = false;
    if (ex != 0) { s = ex > 0 ? vx : -vx; any = true; }
    if (ey != 0) { s = any ? (ey > 0 ? s + vy : s - vy) : (ey > 0 ? vy : -vy); any = true; }
    if (ez != 0) { s = any ? (ez > 0 ? s + vz : s - vz) : (ez > 0 ? vz : -vz); }
    return s;
}

// acc + e v for a component e in {-1, 0, 1}
template <typename C>
__device__ __forceinline__ C add_e(C acc, int e, C v) {
    return e > 0 ? acc + v : (e < 0 ? acc - v : acc);
}

// Collide one node: moments (Eq. (18)) with the half-force shift, BGK toward
// f^eq (Eqs. (15)-(16)) plus Guo's forcing term (compiled out when the body
// force is zero).  fin and out hold collide-space values (Codec::ldv): the
// offsets g = f - w rho0 for FP32/FP64 storage, the stored h = g / w for the
// scaled 16-bit forms, so neither side multiplies by the weights.
//
// Per direction, with c = omega drho - 1.5 omega rho u.u,
//   g_out_i = (1 - omega) g_i + w_i (c + 3 omega rho e_i.u + 4.5 omega rho (e_i.u)^2)
//             + w_i gfac (3 (e_i.F - u.F) + 9 (e_i.u)(e_i.F)),
// which is omega g^eq_i (offset form) plus the forcing term (h_out_i =
// g_out_i / w_i is the same without the w_i).  Opposite directions share w_i
// and |e_i.u|, so each pair (i, i+1) evaluates the even part once and adds or
// subtracts the odd part.
template <typename S, int Q, bool kForce>
__device__ __forceinline__ void collide_values(const Params &P, const typename Codec<S>::C (&fin)[Q],
                                               typename Codec<S>::C (&out)[Q]) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    static_assert(L::opp(1) == 2 && L::opp(Q - 2) == Q - 1, "directions come in opposite pairs (i, i+1), i odd");
    const C rho0 = Prm<C>::rho0(P);
    // offsets: rho = rho0 + sum g, momentum = sum g e
    C drho = 0, mx = 0, my = 0, mz = 0;
    if constexpr (Cd::kScaled) {
        // g = w h: sums per weight class (rest, i = 1..6, i = 7..Q-1), then weighted
        C s1 = 0, x1 = 0, y1 = 0, z1 = 0, s2 = 0, x2 = 0, y2 = 0, z2 = 0;
#pragma unroll
        for (int i = 1; i <= 6; i++) {
            s1 += fin[i];
            x1 = add_e(x1, L::e(i, 0), fin[i]);
            y1 = add_e(y1, L::e(i, 1), fin[i]);
            z1 = add_e(z1, L::e(i, 2), fin[i]);
        }
#pragma unroll
        for (int i = 7; i < Q; i++) {
            s2 += fin[i];
            x2 = add_e(x2, L::e(i, 0), fin[i]);
            y2 = add_e(y2, L::e(i, 1), fin[i]);
            z2 = add_e(z2, L::e(i, 2), fin[i]);
        }
        const C w0 = (C)L::w(0), w1 = (C)L::w(1), w2 = (C)L::w(Q - 1);
        drho = w0 * fin[0] + w1 * s1 + w2 * s2;
        mx = w1 * x1 + w2 * x2;
        my = w1 * y1 + w2 * y2;
        mz = w1 * z1 + w2 * z2;
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            drho += fin[i];
            mx = add_e(mx, L::e(i, 0), fin[i]);
            my = add_e(my, L::e(i, 1), fin[i]);
            mz = add_e(mz, L::e(i, 2), fin[i]);
        }
    }
    const C rho = rho0 + drho;
    const C Fx = kForce ? Prm<C>::F(P, 0) : C(0), Fy = kForce ? Prm<C>::F(P, 1) : C(0),
            Fz = kForce ? Prm<C>::F(P, 2) : C(0);
    C inv_rho;
    if (sizeof(C) == 4) inv_rho = (C)__frcp_rn((float)rho);
    else inv_rho = C(1) / rho;
    C ux, uy, uz;
    if (kForce) {
        ux = (mx + C(0.5) * Fx) * inv_rho; uy = (my + C(0.5) * Fy) * inv_rho; uz = (mz + C(0.5) * Fz) * inv_rho;
    } else {
        ux = mx * inv_rho; uy = my * inv_rho; uz = mz * inv_rho;
    }
    const C omega = Prm<C>::omega(P), om1 = C(1) - omega;
    const C uu = ux * ux + uy * uy + uz * uz;
    const C om_rho = omega * rho;
    const C c = omega * drho - C(1.5) * om_rho * uu;
    const C k3 = C(3) * om_rho, k45 = C(4.5) * om_rho;
    C gfac = C(0), uF3 = C(0);
    if (kForce) {
        gfac = Prm<C>::gfac(P);
        uF3 = C(3) * (ux * Fx + uy * Fy + uz * Fz);
    }
    {
        C e = c;
        if (kForce) e -= gfac * uF3;
        if constexpr (Cd::kScaled) out[0] = om1 * fin[0] + e;
        else out[0] = om1 * fin[0] + (C)L::w(0) * e;
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
        const C eu = dot_e(ex, ey, ez, ux, uy, uz);
        C even = c + k45 * eu * eu;  // equal for i and its opposite
        C odd = k3 * eu;             // opposite signs
        if (kForce) {
            const C eF = dot_e(ex, ey, ez, Fx, Fy, Fz);
            even += gfac * (C(9) * eu * eF - uF3);
            odd += gfac * C(3) * eF;
        }
        if constexpr (!Cd::kScaled) {
            const C w = (C)L::w(i);
            even *= w;
            odd *= w;
        }
        out[i] = om1 * fin[i] + (even + odd);
        out[i + 1] = om1 * fin[i + 1] + (even - odd);
    }
}

// Collide one node (collide-space values, see collide_values) and store it.
template <typename S, int Q, bool kForce, bool kStream = false>
__device__ __forceinline__ void collide_store(const Params &P, typename Codec<S>::C (&fin)[Q], S *B, long long N,
                                              int n) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const C rho0 = Prm<C>::rho0(P);
    C out[Q];
    collide_values<S, Q, kForce>(P, fin, out);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const C w = (C)L::w(i);
        if (kStream) Cd::stv_s(B + (long long)i * N + n, out[i], w, rho0);
        else Cd::stv(B + (long long)i * N + n, out[i], w, rho0);
    }
}

// Neighbour coordinates of a node along each axis (index 0: -1, 1: 0, 2: +1),
// wrapped on periodic axes, -1 beyond a wall.
__device__ __forceinline__ void neighbour_coords(const Params &P, int x, int y, int z, int xs[3], int ys[3], int zs[3]) {
    xs[1] = x; ys[1] = y; zs[1] = z;
    xs[0] = x - 1; xs[2] = x + 1; ys[0] = y - 1; ys[2] = y + 1; zs[0] = z - 1; zs[2] = z + 1;
    if (xs[0] < 0) xs[0] = P.per[0] ? P.nx - 1 : -1;
    if (xs[2] >= P.nx) xs[2] = P.per[0] ? 0 : -1;
    if (ys[0] < 0) ys[0] = P.per[1] ? P.ny - 1 : -1;
    if (ys[2] >= P.ny) ys[2] = P.per[1] ? 0 : -1;
    if (zs[0] < 0) zs[0] = P.per[2] ? P.nz - 1 : -1;
    if (zs[2] >= P.nz) zs[2] = P.per[2] ? 0 : -1;
}

// The pull of a node no particle link reaches: f_i from x - e_i, halfway
// bounce-back at walls (the node's own opposite population), as collide-space
// values (Codec::ldv).  No flags are read.  A row off the y and z faces (one warp of a brick) takes the source
// n - e_i . (1, nx, nx ny) as a 32-bit index, corrected only on its two
// x-face lanes (wrap or bounce-back); other rows, and lattices whose
// population indices need more than 31 bits, resolve each neighbour's
// coordinates.
template <typename S, int Q, bool kStream>
__device__ __forceinline__ void plain_pull(const Params &P, int x, int y, int z, int n,
                                           typename Codec<S>::C (&fin)[Q]) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const S *A = (const S *)P.fA;
    const C rho0 = Prm<C>::rho0(P);
    if (P.idx32 && y > 0 && y < P.ny - 1 && z > 0 && z < P.nz - 1) {
        const int N = (int)P.N, nx = P.nx, nxy = P.nx * P.ny;
        int cm = 0, cp = 0;        // source x - 1 (e_x = +1) and x + 1 (e_x = -1) wrapped
        bool wm = false, wp = false;  // ... or beyond a wall
        if (x == 0) { if (P.per[0]) cm = nx; else wm = true; }
        if (x == nx - 1) { if (P.per[0]) cp = -nx; else wp = true; }
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const int ex = L::e(i, 0);
            int idx = i * N + n - (ex + nx * L::e(i, 1) + nxy * L::e(i, 2));
            if (ex > 0) idx = wm ? L::opp(i) * N + n : idx + cm;
            if (ex < 0) idx = wp ? L::opp(i) * N + n : idx + cp;
            const S *src = A + (unsigned)idx;
            fin[i] = kStream ? Cd::ldv_s(src, (C)L::w(i), rho0) : Cd::ldv(src, (C)L::w(i), rho0);
        }
        return;
    }
    const long long N = P.N;
    int xs[3], ys[3], zs[3];
    neighbour_coords(P, x, y, z, xs, ys, zs);
    int row[3][3];  // nx * (y' + ny * z') for the neighbour rows
#pragma unroll
    for (int b = 0; b < 3; b++)
#pragma unroll
        for (int c = 0; c < 3; c++) row[b][c] = P.nx * (ys[b] + P.ny * zs[c]);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int bx = 1 - L::e(i, 0), by = 1 - L::e(i, 1), bz = 1 - L::e(i, 2);
        const bool wall = (xs[bx] | ys[by] | zs[bz]) < 0;
        // wall: f_i = f+_i'(x), the node's own opposite population
        const S *src = wall ? A + (long long)L::opp(i) * N + n : A + (long long)i * N + (xs[bx] + row[by][bz]);
        fin[i] = kStream ? Cd::ldv_s(src, (C)L::w(i), rho0) : Cd::ldv(src, (C)L::w(i), rho0);
    }
}

// A node of a brick no particle reaches: pull, collide, store.
template <typename S, int Q, bool kForce, bool kStream = false>
__device__ __forceinline__ void plain_node(const Params &P, int x, int y, int z, int n) {
    typename Codec<S>::C fin[Q];
    plain_pull<S, Q, kStream>(P, x, y, z, n, fin);
    collide_store<S, Q, kForce, kStream>(P, fin, (S *)P.fB, P.N, n);
}

// The sweep of every brick outside this step's predicted near set: the plain
// path only.  Runs on its own stream, concurrently with the particle kernels.
// With few near bricks expected (plain_spec) the pulls are issued together
// with the brick's skip entry and only the stores wait for it, so a CTA does
// not start with a lone dependent load; a skipped brick then costs its reads.
template <typename S, int Q, bool kForce>
__device__ __forceinline__ void plain_brick(const Params &P, int b) {
    const int tid = threadIdx.x;
    int bxi, byi, bzi;
    brick_coords(P, b, bxi, byi, bzi);
    const int x = bxi * BX + tid % BX, y = byi * BY + (tid / BX) % BY, z = bzi * BZ + tid / (BX * BY);
    const bool inside = x < P.nx && y < P.ny && z < P.nz;
    const int n = x + P.nx * (y + P.ny * z);
    if (P.plain_spec) {
        const bool skipped = P.skip && P.skip[(P.step % 3) * P.nbricks + b] == P.step;
        if (!inside) return;
        typename Codec<S>::C fin[Q];
        plain_pull<S, Q, true>(P, x, y, z, n, fin);
        if (!skipped) collide_store<S, Q, kForce, true>(P, fin, (S *)P.fB, P.N, n);
        return;
    }
    if (P.skip && P.skip[(P.step % 3) * P.nbricks + b] == P.step) return;  // the near sweep takes it
    if (inside) plain_node<S, Q, kForce, true>(P, x, y, z, n);
}
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, 4) k_sweep_plain(Params P) {
    // persistent over the bricks when the grid is smaller than the brick
    // count (it then leaves CTA slots to the particle kernels running beside)
    for (int b = blockIdx.x; b < P.nbricks; b += gridDim.x) plain_brick<S, Q, kForce>(P, b);
}

}  // namespace lbmmb
