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

// Collide one node: moments (Eq. (18)) with the half-force shift, BGK toward
// f^eq (Eqs. (15)-(16)) plus Guo's forcing term (compiled out when the body
// force is zero); out receives the post-collision offsets.
template <typename S, int Q, bool kForce>
__device__ __forceinline__ void collide_values(const Params &P, const typename Codec<S>::C (&fin)[Q],
                                               typename Codec<S>::C (&out)[Q]) {
    using L = Lat<Q>;
    using C = typename Codec<S>::C;
    const C rho0 = Prm<C>::rho0(P);
    // offsets: rho = rho0 + sum g, momentum = sum g e
    C drho = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        drho += fin[i];
        mx += fin[i] * L::e(i, 0);
        my += fin[i] * L::e(i, 1);
        mz += fin[i] * L::e(i, 2);
    }
    const C rho = rho0 + drho;
    const C Fx = kForce ? Prm<C>::F(P, 0) : C(0), Fy = kForce ? Prm<C>::F(P, 1) : C(0),
            Fz = kForce ? Prm<C>::F(P, 2) : C(0);
    C inv_rho;
    if (sizeof(C) == 4) inv_rho = (C)__frcp_rn((float)rho);
    else inv_rho = C(1) / rho;
    const C ux = (mx + C(0.5) * Fx) * inv_rho, uy = (my + C(0.5) * Fy) * inv_rho, uz = (mz + C(0.5) * Fz) * inv_rho;
    const C omega = Prm<C>::omega(P);
    const C uu = ux * ux + uy * uy + uz * uz;
    const C om_rho = omega * rho, om_drho = omega * drho;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
        const C w = (C)L::w(i);
        const C eu = ex * ux + ey * uy + ez * uz;
        // omega g^eq = w (omega drho + omega rho (3 eu + 4.5 eu^2 - 1.5 uu))
        const C geq_om = w * (om_drho + om_rho * (C(3) * eu + C(4.5) * eu * eu - C(1.5) * uu));
        C o = fin[i] - omega * fin[i] + geq_om;
        if (kForce) {
            const C gfac = Prm<C>::gfac(P);
            const C uF = ux * Fx + uy * Fy + uz * Fz;
            const C eF = ex * Fx + ey * Fy + ez * Fz;
            o += gfac * w * (C(3) * (eF - uF) + C(9) * eu * eF);
        }
        out[i] = o;
    }
}

// Collide one node and store it.
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
        if (kStream) Cd::st_s(B + (long long)i * N + n, out[i], w, rho0);
        else Cd::st(B + (long long)i * N + n, out[i], w, rho0);
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
// bounce-back at walls (the node's own opposite population).  No flags are
// read.  Node indices are 32-bit (the lattice holds fewer than 2^31 nodes).
template <typename S, int Q, bool kStream>
__device__ __forceinline__ void plain_pull(const Params &P, int x, int y, int z, int n,
                                           typename Codec<S>::C (&fin)[Q]) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const S *A = (const S *)P.fA;
    const long long N = P.N;
    const C rho0 = Prm<C>::rho0(P);
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
        fin[i] = kStream ? Cd::ld_s(src, (C)L::w(i), rho0) : Cd::ld(src, (C)L::w(i), rho0);
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
template <typename S, int Q, bool kForce>
__device__ __forceinline__ void plain_brick(const Params &P, int b) {
    if (P.skip && P.skip[(P.step % 3) * P.nbricks + b] == P.step) return;  // the near sweep takes it
    const int tid = threadIdx.x;
    int bxi, byi, bzi;
    brick_coords(P, b, bxi, byi, bzi);
    const int x = bxi * BX + tid % BX, y = byi * BY + (tid / BX) % BY, z = bzi * BZ + tid / (BX * BY);
    if (x < P.nx && y < P.ny && z < P.nz) plain_node<S, Q, kForce, true>(P, x, y, z, x + P.nx * (y + P.ny * z));
}
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, 4) k_sweep_plain(Params P) {
    // persistent over the bricks when the grid is smaller than the brick
    // count (it then leaves CTA slots to the particle kernels running beside)
    for (int b = blockIdx.x; b < P.nbricks; b += gridDim.x) plain_brick<S, Q, kForce>(P, b);
}

}  // namespace lbmmb
