// The fixed-geometry sweep.
//
// When every particle is fixed (fixed = 1) the node flags, the particle links
// and their geometry (q of Eq. (27), the lever arm from the centroid to the
// wall point x_w and the wall velocity there) cannot change.  Once the flag
// pass has run for three steps, k_static_build records them: per node whether
// the plain path may take it (sskip), and for every fluid node with particle
// links its link directions and each link's geometry.  The missing force
// points (§2.3.5 item 2, Eqs. (31)-(32)) depend on the geometry only, so their
// fixed-point force/torque totals are summed once (smf).  Every later step is
// two kernels that run concurrently on disjoint nodes: k_static_plain over the
// nodes the plain path takes (the pull, BGK and stores of k_sweep_plain, over
// aligned 256-node spans, no brick lists) and k_static_links over the link
// nodes (VIBB of Eqs. (19)-(25) and the momentum exchange of Eqs. (28)-(29)
// with the recorded geometry).  The arithmetic is the near sweep's
// (link_geometry, link_update, solid_links, collide_store), so a step gives
// the same bits either way.  Lattices below FP64 only (the force totals are
// the fixed-point ones).
#pragma once

#include "k_sweep.cuh"

namespace lbmmb {

// ---------------------------------------------------------------------------
// build: one CTA per brick listed this step (no other brick holds a solid
// node or a node next to one), after sskip, scount and smf were cleared
// ---------------------------------------------------------------------------
struct StaticBuildScratch {
    uint32_t nf[BRICK][19];  // the node's flag and its neighbours' (index i: y = x - e_i)
    unsigned long long fix[BRICK / 32][MAXPB][6];  // each warp's missing-force terms
};

template <typename S, int Q>
__device__ __forceinline__ void static_build_brick(const Params &P, SmemParticles &sp, StaticBuildScratch &bs,
                                                   int b) {
    using L = Lat<Q>;
    using C = typename Codec<S>::C;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int bxi, byi, bzi;
    brick_coords(P, b, bxi, byi, bzi);
    const int bx0 = bxi * BX, by0 = byi * BY, bz0 = bzi * BZ;
    const int lx = tid % BX, ly = (tid / BX) % BY, lz = tid / (BX * BY);
    const int x = bx0 + lx, y = by0 + ly, z = bz0 + lz;
    const bool active = x < P.nx && y < P.ny && z < P.nz;
    const int n = x + P.nx * (y + P.ny * z);
    const int cnt = min(P.bcount[b], MAXPB);
    __syncthreads();  // the previous brick is done with the shared state
    load_smem_particles(P, sp, b, bx0, by0, bz0);
    for (int e = lane; e < cnt * 6; e += 32) bs.fix[warp][e / 6][e % 6] = 0ull;
    __syncwarp();

    constexpr uint32_t kWall = 0xFFFFFFFFu;
    {
        int xs[3], ys[3], zs[3];
        neighbour_coords(P, x, y, z, xs, ys, zs);
        bs.nf[tid][0] = active ? (uint32_t)P.flag_new[n] : 1u;
#pragma unroll
        for (int i = 1; i < Q; i++) {
            const int sx = xs[1 - L::e(i, 0)], sy = ys[1 - L::e(i, 1)], sz = zs[1 - L::e(i, 2)];
            const bool wall = (sx | sy | sz) < 0;
            bs.nf[tid][i] = (!active || wall) ? kWall : (uint32_t)P.flag_new[sx + P.nx * (sy + P.ny * sz)];
        }
    }
    const uint32_t own = bs.nf[tid][0];
    const bool fluid = active && own == 0;
    uint32_t links = 0;
    if (fluid) {
        for (int i = 1; i < Q; i++)
            if (bs.nf[tid][i] != 0 && bs.nf[tid][i] != kWall) links |= 1u << i;
    }
    if (active) P.sskip[n] = (uint8_t)((!fluid || links) ? 1 : 0);

    if (links) {
        const int k = __popc(links);
        const int node = atomicAdd(&P.scount[0], 1);
        const int base = atomicAdd(&P.scount[1], k);
        if (node >= P.snode_cap || base + k > P.slink_cap) {
            atomicOr(&P.status[ST_ERR], ERRB_STATIC_CAPACITY);
        } else {
            StaticNode sn;
            sn.n = n;
            sn.mask = links;
            sn.base = base;
            P.snodes[node] = sn;
            C Mf_cache = 0;
            int Mf_slot = -1;
            int r = 0;
            uint32_t m = links;
            while (m) {
                const int i = __ffs(m) - 1;
                m &= m - 1;
                const int j = (int)bs.nf[tid][i] - 1;
                const int s = slot_of(sp, j);
                StaticLink rec;
                if (s < 0) {  // cannot happen for a consistent brick list
                    atomicOr(&P.status[ST_ERR], ERRB_BRICK_OVERFLOW);
                    rec.q = 0.f;
                    for (int a = 0; a < 3; a++) rec.r[a] = rec.uw[a] = 0.f;
                } else {
                    const LinkGeom<C> g = link_geometry<S, Q>(P, sp, i, s, lx, ly, lz, bx0, by0, bz0, &Mf_cache,
                                                              &Mf_slot);
                    rec.q = (float)g.q;
                    for (int a = 0; a < 3; a++) {
                        rec.r[a] = (float)g.r[a];
                        rec.uw[a] = (float)g.uw[a];
                    }
                }
                // x_ff = x - d = x + e_i is the neighbour on the far side
                const bool ff_ok = bs.nf[tid][L::opp(i)] == 0;
                rec.jf = (j & 0xFFFF) | (ff_ok ? (int)0x80000000u : 0);
                P.slinks[base + r] = rec;
                r++;
            }
        }
    }

    // missing force points of the solid nodes: their totals once
    if (active && !fluid && P.missing_force) {
        const int owner = (int)own - 1;
        const ForceSink<C> sink{nullptr, bs.fix[warp]};
        for (int s = 0; s < sp.n; s++) {
            const int j = sp.id[s];
            uint32_t cand = 0;
            for (int i = 1; i < Q; i++) {
                const uint32_t f = bs.nf[tid][i];
                const bool seen = (f == 0 && j == owner) || f == (uint32_t)(j + 1);
                if (!seen) cand |= 1u << i;
            }
            if (cand) solid_links<S, Q>(P, sp, s, j == owner, cand, lx, ly, lz, bx0, by0, bz0, sink);
        }
    }
    __syncwarp();
    for (int e = lane; e < cnt * 6; e += 32) {
        const unsigned long long v = bs.fix[warp][e / 6][e % 6];
        if (v) atomicAdd(&P.smf[sp.id[e / 6] * 6 + e % 6], v);
    }
}

template <typename S, int Q>
__global__ void __launch_bounds__(BRICK) k_static_build(Params P) {
    if (sizeof(typename Codec<S>::C) == 8) return;  // FP64 lattices keep the near sweep
    __shared__ SmemParticles sp;
    __shared__ StaticBuildScratch bs;
    const int listed = P.counters[CNT_LISTED];
    for (int w = blockIdx.x; w < listed; w += gridDim.x)
        static_build_brick<S, Q>(P, sp, bs, P.wl_list[(P.step % 3) * P.nbricks + w]);
}

// ---------------------------------------------------------------------------
// plain nodes: one CTA per 256 consecutive nodes
// ---------------------------------------------------------------------------
// The node's skip mark is loaded together with its pulls (which stay in the
// box either way), so the two latencies overlap; a skipped node stores
// nothing.
template <typename S, int Q, bool kForce>
__device__ __forceinline__ void static_plain_node(const Params &P, int n) {
    if (n >= P.N) return;
    const bool skip = P.sskip[n] != 0;
    const int nxy = P.nx * P.ny;
    const int z = n / nxy, r = n - z * nxy;
    const int y = r / P.nx, x = r - y * P.nx;
    typename Codec<S>::C fin[Q];
    plain_pull<S, Q, true>(P, x, y, z, n, fin);
    if (!skip) collide_store<S, Q, kForce, true>(P, fin, (S *)P.fB, P.N, n);
}
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, 4) k_static_plain(Params P) {
    static_plain_node<S, Q, kForce>(P, blockIdx.x * BRICK + (int)threadIdx.x);
}

// ---------------------------------------------------------------------------
// link nodes: one warp per kStaticNodesPerWarp listed link nodes
// ---------------------------------------------------------------------------
constexpr int kStaticSlots = 4;  // particles per warp with shared-memory force sums
struct StaticScratch {
    unsigned short entry[BRICK / 32][kLinkQueue];  // (lane << 5) | direction
    int rec[BRICK / 32][kLinkQueue];               // link record, then (as float bits) its result
    int node[BRICK / 32][32];                      // node index of each lane
    int ids[BRICK / 32][kStaticSlots];
    unsigned long long fix[BRICK / 32][kStaticSlots][6];
};

// One link of node n (direction i, record r): the node's own populations and
// x_ff's fetched in one round, the unknown and the momentum exchange with the
// recorded geometry; the force/torque terms go to the warp's table.
template <typename S, int Q>
__device__ __noinline__ float static_link(const Params &P, StaticScratch &ss, int warp, int n, int i, int r) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const S *A = (const S *)P.fA;
    const long long N = P.N;
    const C rho0 = Prm<C>::rho0(P);
    const StaticLink rec = P.slinks[r];
    const int nxy = P.nx * P.ny;
    const int z = n / nxy, rr = n - z * nxy;
    const int y = rr / P.nx, x = rr - y * P.nx;
    const int io = L::opp(i);
    const bool ok = rec.jf < 0;  // bit 31
    // x_ff = x - d = x + e_i (inside the box when ok)
    int fx = x + lat_e<Q>(i, 0), fy = y + lat_e<Q>(i, 1), fz = z + lat_e<Q>(i, 2);
    if (fx < 0) fx += P.nx; else if (fx >= P.nx) fx -= P.nx;
    if (fy < 0) fy += P.ny; else if (fy >= P.ny) fy -= P.ny;
    if (fz < 0) fz += P.nz; else if (fz >= P.nz) fz -= P.nz;
    const int nff = ok ? fx + P.nx * (fy + P.ny * fz) : n;
    FFData<C> ff;
    ff.drho = 0;
    ff.m[0] = ff.m[1] = ff.m[2] = 0;
    ff.g_io = 0;
    ff.ok = ok;
    C fown_io = 0, drho_f = 0, m_f[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const C fk = Cd::ld(A + (long long)k * N + n, (C)L::w(k), rho0);
        drho_f += fk;
        m_f[0] += fk * L::e(k, 0);
        m_f[1] += fk * L::e(k, 1);
        m_f[2] += fk * L::e(k, 2);
        if (k == io) fown_io = fk;
        if (P.vibb && ok) {
            const C gk = Cd::ld(A + (long long)k * N + nff, (C)L::w(k), rho0);
            ff.drho += gk;
            ff.m[0] += gk * L::e(k, 0);
            ff.m[1] += gk * L::e(k, 1);
            ff.m[2] += gk * L::e(k, 2);
            if (k == io) ff.g_io = gk;
        }
    }
    C u_f[3];
    const C inv_rho_f = rcp_w<C>(rho0 + drho_f);  // as the near sweep's link_coop
    for (int a = 0; a < 3; a++) u_f[a] = (m_f[a] - C(0.5) * Prm<C>::F(P, a)) * inv_rho_f;
    LinkGeom<C> g;
    g.q = (C)rec.q;
    for (int a = 0; a < 3; a++) {
        g.r[a] = (C)rec.r[a];
        g.uw[a] = (C)rec.uw[a];
    }
    C dP[3];
    const C fin = link_update<S, Q>(P, i, g, ff, fown_io, drho_f, u_f, dP);
    C t[6];
    force_terms<C>(dP, g.r, t);
    const int j = rec.jf & 0xFFFF;
    int slot = -1;
    for (int k = 0; k < kStaticSlots && slot < 0; k++) {
        const int id = ss.ids[warp][k];
        if (id == j) {
            slot = k;
        } else if (id < 0) {
            const int old = atomicCAS(&ss.ids[warp][k], -1, j);
            if (old == -1 || old == j) slot = k;
        }
    }
    for (int c = 0; c < 6; c++) {
        if (t[c] == C(0)) continue;
        if (slot >= 0) atomicAdd(&ss.fix[warp][slot][c], to_fixed<C>(t[c]));
        else atomicAdd(&P.Ffix[j * 6 + c], to_fixed<C>(t[c]));
    }
    return (float)fin;
}

template <typename S, int Q, bool kForce>
__device__ __forceinline__ void static_links_warp(const Params &P, StaticScratch &ss, int wg) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const S *A = (const S *)P.fA;
    S *B = (S *)P.fB;
    const long long N = P.N;
    const C rho0 = Prm<C>::rho0(P);
    if (lane < kStaticSlots) ss.ids[warp][lane] = -1;
    for (int e = lane; e < kStaticSlots * 6; e += 32) ss.fix[warp][e / 6][e % 6] = 0ull;
    const int idx = wg * kStaticNodesPerWarp + lane;
    const bool has = lane < kStaticNodesPerWarp && idx < P.snodes_n;
    StaticNode sn;
    sn.n = 0;
    sn.mask = 0u;
    sn.base = 0;
    if (has) sn = P.snodes[idx];
    ss.node[warp][lane] = sn.n;
    const uint32_t links = sn.mask;
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
        for (int k = 0; m; k++) {
            const int i = __ffs(m) - 1;
            m &= m - 1;
            ss.entry[warp][first + k] = (unsigned short)((lane << 5) | i);
            ss.rec[warp][first + k] = sn.base + k;
        }
    }
    __syncwarp();
    for (int e = lane; e < total; e += 32) {
        const int ent = ss.entry[warp][e];
        ss.rec[warp][e] =
            __float_as_int(static_link<S, Q>(P, ss, warp, ss.node[warp][ent >> 5], ent & 31, ss.rec[warp][e]));
    }
    __syncwarp();
    if (has) {
        const int n = sn.n;
        const int nxy = P.nx * P.ny;
        const int z = n / nxy, rr = n - z * nxy;
        const int y = rr / P.nx, x = rr - y * P.nx;
        int xs[3], ys[3], zs[3];
        neighbour_coords(P, x, y, z, xs, ys, zs);
        C fin[Q];
        int k = first;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            if (links & (1u << i)) {  // link results are offsets g
                fin[i] = Cd::g_to_v((C)__int_as_float(ss.rec[warp][k]), (C)L::w(i));
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
    __syncwarp();
    for (int e = lane; e < kStaticSlots * 6; e += 32) {
        const int id = ss.ids[warp][e / 6];
        const unsigned long long v = ss.fix[warp][e / 6][e % 6];
        if (id >= 0 && v) atomicAdd(&P.Ffix[id * 6 + e % 6], v);
    }
}

// The step's constant parts: the missing-force-point totals and the link
// count (one thread).
__device__ __forceinline__ void static_constants(const Params &P) {
    for (int k = 0; k < P.np * 6; k++)
        if (P.smf[k]) atomicAdd(&P.Ffix[k], P.smf[k]);
    atomicAdd(&P.counters[CNT_NLINKS], P.scount[1]);
}

template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, kNearCtasPerSm) k_static_links(Params P) {
    if (sizeof(typename Codec<S>::C) == 8) return;
    __shared__ StaticScratch ss;
    if (blockIdx.x == 0 && threadIdx.x == 0) static_constants(P);
    const int warps = (P.snodes_n + kStaticNodesPerWarp - 1) / kStaticNodesPerWarp;
    for (int wg = blockIdx.x * (BRICK / 32) + (threadIdx.x >> 5); wg < warps; wg += gridDim.x * (BRICK / 32))
        static_links_warp<S, Q, kForce>(P, ss, wg);
}

// ---------------------------------------------------------------------------
// batched lattices: the same two kernels over all cases
// ---------------------------------------------------------------------------

// plain_chunk spans per CTA as k_sweep_plain_batch; the CTA holding a case's
// first span also clears that case's per-step region for the next step (the
// binning, which clears it otherwise, does not run in fixed-geometry steps).
// Compiled for five CTAs per SM (48 registers, 8 bytes spilled): no particle
// kernel needs the SM slots here, and it measured 1 % faster than four on the
// 64-case batch (six spilled 88 bytes and was 2-6 % slower).
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, 5) k_static_plain_batch(BatchArgs B) {
    const int total = B.span_off[B.ncases];
    const unsigned step = *(volatile const unsigned *)(B.ctr + 1);
    const Params *row = B.tab + (size_t)(step & 1) * B.ncases;
    const int g0 = blockIdx.x * B.plain_chunk;
    const int g1 = min(total, g0 + B.plain_chunk);
    // the case's parameters in shared memory (re-read when the CTA's spans
    // cross into the next case): loads from there cannot alias the stores
    // to the populations, so they stay in registers
    __shared__ Params sP;
    int cur = -1;
    for (int g = g0; g < g1; g++) {
        const int c = B.span_case[g];
        if (c != cur) {
            __syncthreads();
            const int *src = reinterpret_cast<const int *>(row + c);
            int *dst = reinterpret_cast<int *>(&sP);
            for (int k = threadIdx.x; k < (int)(sizeof(Params) / 4); k += blockDim.x) dst[k] = src[k];
            __syncthreads();
            cur = c;
        }
        const Params &P = sP;
        if (g == B.span_off[c]) {
            int4 *zp = static_cast<int4 *>(P.bin_next);
            const long long n16 = P.bin_next_bytes / 16;
            for (long long k = threadIdx.x; k < n16; k += blockDim.x) zp[k] = make_int4(0, 0, 0, 0);
        }
        static_plain_node<S, Q, kForce>(P, (g - B.span_off[c]) * BRICK + (int)threadIdx.x);
    }
    advance_step_when_last(B.ctr + 3, B.ctr + 1);
}

// One warp per kStaticNodesPerWarp link nodes of a case (each case at least one warp, whose
// first also adds the case's constant parts); the last CTA advances the
// particle chain's step counter.
template <typename S, int Q, bool kForce>
__global__ void __launch_bounds__(BRICK, kNearCtasPerSm) k_static_links_batch(BatchArgs B) {
    __shared__ StaticScratch ss;
    const unsigned step = *(volatile const unsigned *)B.ctr;
    const Params *row = B.tab + (size_t)(step & 1) * B.ncases;
    const int warps = B.swarp_off[B.ncases];
    const int gw = blockIdx.x * (BRICK / 32) + (int)(threadIdx.x >> 5);
    if (gw < warps) {
        int lo = 0, hi = B.ncases - 1;  // the case whose warp range holds gw
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (B.swarp_off[mid] <= gw) lo = mid;
            else hi = mid - 1;
        }
        const Params &P = row[lo];
        const int wl = gw - B.swarp_off[lo];
        if (wl == 0 && (threadIdx.x & 31) == 0) static_constants(P);
        if (wl * kStaticNodesPerWarp < P.snodes_n) static_links_warp<S, Q, kForce>(P, ss, wl);
    }
    advance_step_when_last(B.ctr + 2, B.ctr);
}

}  // namespace lbmmb
