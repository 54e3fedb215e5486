// Node classification and local refilling (templated on storage and lattice).
//
// k_flags (one CTA per brick): sorts the brick's list, classifies its nodes
// (§2.3.1: solid when M_j >= c0, Eq. (26), owner = largest M_j, ties to the
// lower index), and refills the nodes the particles uncovered since the last
// step (§2.3.3, Eq. (30)).  M is evaluated in FP32 against a certified
// error band and re-evaluated in FP64 inside it, so the flags equal those of
// an exact FP64 evaluation.
#pragma once

#include "lbm_internal.cuh"

namespace lbmmb {

__device__ __forceinline__ void quat_rot(const double q[4], const double v[3], double r[3]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double R00 = 1 - 2 * (y * y + z * z), R01 = 2 * (x * y - w * z), R02 = 2 * (x * z + w * y);
    const double R10 = 2 * (x * y + w * z), R11 = 1 - 2 * (x * x + z * z), R12 = 2 * (y * z - w * x);
    const double R20 = 2 * (x * z - w * y), R21 = 2 * (y * z + w * x), R22 = 1 - 2 * (x * x + y * y);
    r[0] = R00 * v[0] + R01 * v[1] + R02 * v[2];
    r[1] = R10 * v[0] + R11 * v[1] + R12 * v[2];
    r[2] = R20 * v[0] + R21 * v[1] + R22 * v[2];
}

template <typename C>
__device__ __forceinline__ C feq_i(int ex, int ey, int ez, C w, C rho, C ux, C uy, C uz) {
    const C eu = ex * ux + ey * uy + ez * uz;
    const C uu = ux * ux + uy * uy + uz * uz;
    return w * rho * (C(1) + C(3) * eu + C(4.5) * eu * eu - C(1.5) * uu);
}
// The same equilibrium in offset form: f^eq_i - w_i rho0 for density
// rho = rho0 + drho.
template <typename C>
__device__ __forceinline__ C geq_i(int ex, int ey, int ez, C w, C drho, C rho, C ux, C uy, C uz) {
    const C eu = ex * ux + ey * uy + ez * uz;
    const C uu = ux * ux + uy * uy + uz * uz;
    return w * (drho + rho * (C(3) * eu + C(4.5) * eu * eu - C(1.5) * uu));
}

// Per-brick solid marks written by the flag pass (brick_solid): bit 7 when
// the brick holds a solid node, bits 0-5 when one lies on its low-x, high-x,
// low-y, high-y, low-z or high-z face.
constexpr uint32_t kSolidAny = 0x80u;

template <typename S, int Q>
__device__ __forceinline__ void flags_brick(const Params &P, SmemParticles &sp, int b) {
    using L = Lat<Q>;
    using Cd = Codec<S>;
    using C = typename Cd::C;
    constexpr bool kF64 = sizeof(C) == 8;
    const int tid = threadIdx.x;
    int cnt = P.bcount[b];
    // the list's slots are read in the same round as its count (slots past
    // the count hold stale ids and are not used)
    const int raw_id = tid < MAXPB ? P.blist[b * MAXPB + tid] : 0;
    if (cnt > MAXPB) cnt = MAXPB;
    __syncthreads();  // the previous brick's use of sp and of the list is over
    // ascending particle order makes the list, and hence every sum over it,
    // independent of the scatter's atomic order: lane s of warp 0 places its
    // id at its rank (ids are distinct)
    if (tid < 32) {
        const int id = tid < cnt ? raw_id : 0x7fffffff;
        int rank = 0;
        for (int o = 0; o < cnt; o++) rank += __shfl_sync(0xffffffffu, id, o) < id;
        if (tid < cnt) P.blist[b * MAXPB + rank] = id;
        if (tid == 0) P.bcount[b] = cnt;
    }
    __shared__ unsigned s_faces;
    if (tid == 0) s_faces = 0u;
    __syncthreads();
    int bxi, byi, bzi;
    brick_coords(P, b, bxi, byi, bzi);
    const int bx0 = bxi * BX, by0 = byi * BY, bz0 = bzi * BZ;
    const int lx = tid % BX, ly = (tid / BX) % BY, lz = tid / (BX * BY);
    const int x = bx0 + lx, y = by0 + ly, z = bz0 + lz;
    const bool active = x < P.nx && y < P.ny && z < P.nz;
    const long long n = (long long)x + (long long)P.nx * ((long long)y + (long long)P.ny * z);
    // the previous flag (the refill below needs it), issued with the
    // particles' loads so that the two latencies overlap
    const uint16_t old = active ? P.flag_old[n] : (uint16_t)0;
    if (cnt > 0) load_smem_particles(P, sp, b, bx0, by0, bz0);

    // owner: the covering particle with the largest M, ties to the lower
    // index (the list is ascending); with one cover its FP32 decision is
    // enough, several covers compare their M in FP64.  Kept as running
    // values, so no per-thread array is indexed at run time.
    int own = -1;
    if (active && cnt > 0) {
        int own_s = -1;
        double own_M = -1.0;  // FP64 M of the current owner, < 0 until computed
        for (int s = 0; s < cnt; s++) {
            if (!in_bound(P, sp, s, lx, ly, lz)) continue;  // outside s: M < c0 there
            bool unsure;
            const float M = metaball32(P, sp, s, (float)lx, (float)ly, (float)lz, unsure);
            bool inside;
            double Md = -1.0;
            if (kF64 || unsure) {
                Md = metaball64(P, P.parts[sp.id[s]], (double)x, (double)y, (double)z);
                inside = Md >= P.c0;
            } else {
                inside = M >= P.c0_f;
            }
            if (!inside) continue;
            if (own_s < 0) {
                own_s = s;
                own_M = Md;
                continue;
            }
            if (own_M < 0.0) own_M = metaball64(P, P.parts[sp.id[own_s]], (double)x, (double)y, (double)z);
            if (Md < 0.0) Md = metaball64(P, P.parts[sp.id[s]], (double)x, (double)y, (double)z);
            if (Md > own_M) {
                own_s = s;
                own_M = Md;
            }
        }
        if (own_s >= 0) own = sp.id[own_s];
    }
    const uint16_t fl = own >= 0 ? (uint16_t)(own + 1) : (uint16_t)0;
    if (active) P.flag_new[n] = fl;
    // where the brick holds solid nodes now: bit 7 anywhere, bits 0-5 on its
    // faces (low x, high x, low y, high y, low z, high z; a high face is the
    // last node inside the box on a ragged edge).  The near sweep takes the
    // plain path for a brick none of whose nodes has a solid neighbour.
    {
        uint32_t m = 0;
        if (active && fl != 0) {
            m = kSolidAny;
            if (lx == 0) m |= 1u;
            if (lx == BX - 1 || x == P.nx - 1) m |= 2u;
            if (ly == 0) m |= 4u;
            if (ly == BY - 1 || y == P.ny - 1) m |= 8u;
            if (lz == 0) m |= 16u;
            if (lz == BZ - 1 || z == P.nz - 1) m |= 32u;
        }
        m = __reduce_or_sync(0xffffffffu, m);
        if ((tid & 31) == 0 && m) atomicOr(&s_faces, m);
        __syncthreads();
        if (tid == 0 && P.brick_solid) P.brick_solid[b] = (uint8_t)s_faces;
    }

    // Local refilling, §2.3.3.  Reading: f_i' at x_new counts as known
    // (Eq. (30)) when it streams in from x_new + e_i and that node was a fluid
    // node of the previous step; then f_i = f_i'(x_new+e_i) + 6 w_i rho0
    // e_i.u_w, else f_i = f^eq_i(rho0, u_new); u_w = u_new is the surface
    // velocity at x_new of the particle that uncovered it.  The values become
    // the node's post-collision populations.
    if (active && fl == 0) {
        if (old != 0) {
            const DevParticle &pj = P.parts[old - 1];
            double r[3] = {minimg_d(P, 0, (double)x - pj.x[0]), minimg_d(P, 1, (double)y - pj.x[1]),
                           minimg_d(P, 2, (double)z - pj.x[2])};
            const C ux = (C)(pj.v[0] + pj.w[1] * r[2] - pj.w[2] * r[1]);
            const C uy = (C)(pj.v[1] + pj.w[2] * r[0] - pj.w[0] * r[2]);
            const C uz = (C)(pj.v[2] + pj.w[0] * r[1] - pj.w[1] * r[0]);
            const C rho0 = (C)P.rho0;
            S *A = (S *)P.fA;
            const long long N = P.N;
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
                int sx = x + ex, sy = y + ey, sz = z + ez;
                bool in = true;
                if (sx < 0 || sx >= P.nx) { if (P.per[0]) sx = (sx + P.nx) % P.nx; else in = false; }
                if (sy < 0 || sy >= P.ny) { if (P.per[1]) sy = (sy + P.ny) % P.ny; else in = false; }
                if (sz < 0 || sz >= P.nz) { if (P.per[2]) sz = (sz + P.nz) % P.nz; else in = false; }
                const C w = (C)L::w(i);
                // offset form (g = f - w rho0; opposite directions share w)
                C g;
                const long long nb = (long long)sx + (long long)P.nx * ((long long)sy + (long long)P.ny * sz);
                if (i != 0 && in && P.flag_old[nb] == 0) {
                    const int io = L::opp(i);
                    g = Cd::ld_plain(A + (long long)io * N + nb, w, rho0) +
                        C(6) * w * rho0 * (ex * ux + ey * uy + ez * uz);
                } else {
                    g = geq_i<C>(ex, ey, ez, w, C(0), rho0, ux, uy, uz);
                }
                Cd::st(A + (long long)i * N + n, g, w, rho0);
            }
            atomicAdd(&P.counters[CNT_NREFILL], 1);
        }
    }
}

// Persistent grid over the bricks listed this step and in the two steps
// before; a brick listed in several of these lists is visited once (its most
// recent listing).
// The bricks are handed out one at a time from a per-step counter, as in the
// near sweep (thread 0 fetches the next entry while the current brick runs;
// s_next alternates between two slots).
template <typename S, int Q>
__device__ __forceinline__ void flags_work(const Params &P, SmemParticles &sp, int *s_next, int blk) {
    const int t = P.step;
    const int r0 = t % 3, r1 = (t + 2) % 3, r2 = (t + 1) % 3;
    const int c0 = P.counters[CNT_LISTED];
    const int c1 = t >= 1 ? P.wl_count[r1] : 0;
    const int c2 = t >= 2 ? P.wl_count[r2] : 0;
    if (blk == 0 && threadIdx.x == 0) P.wl_count[r0] = c0;  // read by the next two steps
    const int total = c0 + c1 + c2;
    int nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(&P.counters[CNT_FLAGS_NEXT], 1);
    for (int k = 0;; k ^= 1) {
        if (threadIdx.x == 0) s_next[k] = nxt;
        __syncthreads();
        const int w = s_next[k];
        if (w >= total) break;
        if (threadIdx.x == 0) nxt = atomicAdd(&P.counters[CNT_FLAGS_NEXT], 1);
        int b;
        if (w < c0) {
            b = P.wl_list[r0 * P.nbricks + w];
        } else if (w < c0 + c1) {
            b = P.wl_list[r1 * P.nbricks + (w - c0)];
            if (P.stamp[b] == t) continue;      // also listed this step
        } else {
            b = P.wl_list[r2 * P.nbricks + (w - c0 - c1)];
            if (P.stamp[b] >= t - 1) continue;  // listed again since
        }
        flags_brick<S, Q>(P, sp, b);
    }
}
template <typename S, int Q>
__global__ void __launch_bounds__(BRICK) k_flags(Params P) {
    __shared__ SmemParticles sp;
    __shared__ int s_next[2];
    flags_work<S, Q>(P, sp, s_next, blockIdx.x);
}

// Every node to f^eq(rho0, u0).
template <typename S, int Q>
__global__ void k_init(Params P, S *f) {
    using L = Lat<Q>;
    using C = typename Codec<S>::C;
    const C rho0 = (C)P.rho0, ux = (C)P.u0[0], uy = (C)P.u0[1], uz = (C)P.u0[2];
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const C w = (C)L::w(i);
            Codec<S>::st(f + (long long)i * P.N + n, geq_i<C>(L::e(i, 0), L::e(i, 1), L::e(i, 2), w, C(0), rho0, ux, uy, uz),
                         w, rho0);
        }
    }
}

// Stored populations -> FP64 [Q][N] (and back).
template <typename S, int Q>
__global__ void k_get_pop(Params P, const S *f, double *out) {
    using L = Lat<Q>;
    using C = typename Codec<S>::C;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < Q; i++)
            out[(long long)i * P.N + n] =
                (double)Codec<S>::ldf(f + (long long)i * P.N + n, (C)L::w(i), (C)P.rho0);
    }
}
template <typename S, int Q>
__global__ void k_set_pop(Params P, S *f, const double *in) {
    using L = Lat<Q>;
    using C = typename Codec<S>::C;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < Q; i++)
            Codec<S>::stf(f + (long long)i * P.N + n, (C)in[(long long)i * P.N + n], (C)L::w(i), (C)P.rho0);
    }
}

// Macroscopic fields of the stored populations: rho = sum f, u = (sum f e -
// F/2)/rho (the velocity of the collision that produced them).
template <typename S, int Q>
__global__ void k_fields(Params P, const S *f, const uint16_t *flags, double *rho, double *u, uint16_t *fl_out) {
    using L = Lat<Q>;
    using C = typename Codec<S>::C;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += (long long)gridDim.x * blockDim.x) {
        const uint16_t fl = flags[n];
        if (fl_out) fl_out[n] = fl;
        double r = 0, mx = 0, my = 0, mz = 0;
        if (fl == 0) {
            // offsets: rho = rho0 + sum g, momentum = sum g e
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const double gi = (double)Codec<S>::ld_plain(f + (long long)i * P.N + n, (C)L::w(i), (C)P.rho0);
                r += gi;
                mx += gi * L::e(i, 0);
                my += gi * L::e(i, 1);
                mz += gi * L::e(i, 2);
            }
            r += P.rho0;
        }
        if (rho) rho[n] = r;
        if (u) {
            const bool ok = fl == 0;
            u[n] = ok ? (mx - 0.5 * P.F[0]) / r : 0.0;
            u[P.N + n] = ok ? (my - 0.5 * P.F[1]) / r : 0.0;
            u[2 * P.N + n] = ok ? (mz - 0.5 * P.F[2]) / r : 0.0;
        }
    }
}

// Health scan: non-finite populations or |u| > 0.5 at a fluid node.
template <typename S, int Q>
__global__ void k_check(Params P, const S *f, const uint16_t *flags) {
    using L = Lat<Q>;
    using C = typename Codec<S>::C;
    bool bad = false;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += (long long)gridDim.x * blockDim.x) {
        if (flags[n] != 0) continue;
        float r = P.rho0_f, mx = 0, my = 0, mz = 0;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const float gi = (float)Codec<S>::ld_plain(f + (long long)i * P.N + n, (C)L::w(i), (C)P.rho0);
            r += gi;
            mx += gi * L::e(i, 0);
            my += gi * L::e(i, 1);
            mz += gi * L::e(i, 2);
        }
        const float u2 = (mx * mx + my * my + mz * mz) / (r * r);
        if (!(r > 0.f) || !isfinite(r) || !(u2 <= 0.25f)) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&P.status[ST_ERR], ERRB_DIVERGED);
}

}  // namespace lbmmb
