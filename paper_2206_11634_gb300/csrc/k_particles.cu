// Particle-side kernels, all FP64:
//   k_bin          world control points, search boxes, scatter into bricks;
//   k_force_reduce per-particle totals of the sweep's brick partials;
//   k_dem          n_sub DEM sub-steps (§2.3.4) with the hydrodynamic load
//                  frozen: metaball-metaball and metaball-wall contacts
//                  (§2.1.3-2.1.4), contact law (§2.1.1), velocity Verlet and
//                  Euler's equations in the body frame (Eq. (1)).
#include "k_flags.cuh"
#include "dem_fp64.cuh"

namespace lbmmb {

// ---------------------------------------------------------------------------
// k_bin: one CTA per particle.  The search box AABB(x_i) -+ sqrt(sum K / c0)
// holds every node with M >= c0 (M >= c0 forces min |x - x_i|^2 <= sum K /
// c0); grown by one node it also holds every fluid node with a link into
// the particle.  The particle is appended to the list of each brick the grown
// box meets (k_flags sorts the lists).
// ---------------------------------------------------------------------------
__device__ void bin_particle(const Params &P, int j) {
    const int t = threadIdx.x;
    DevParticle &p = P.parts[j];
    if (t < p.ncp) {
        double r[3];
        quat_rot(p.q, p.cpb[t], r);
        for (int a = 0; a < 3; a++) {
            const double c = p.x[a] + r[a];
            p.cpw[t][a] = c;
            // the FP32 pair the sweeps form brick-relative positions from
            const float hi = (float)c;
            p.cpw_hl[t][a][0] = hi;
            p.cpw_hl[t][a][1] = (float)(c - (double)hi);
        }
    } else if (t >= 32 && t < 35) {
        const int a = t - 32;
        const float hi = (float)p.x[a];
        p.x_hl[a][0] = hi;
        p.x_hl[a][1] = (float)(p.x[a] - (double)hi);
    } else if (t >= 64 && t < 70) {
        const int a = t - 64;
        p.vw_f[a] = (float)(a < 3 ? p.v[a] : p.w[a - 3]);
    }
    __syncthreads();
    if (t == 0) {
        const double bound = sqrt(p.sumK / P.c0);
        for (int a = 0; a < 3; a++) {
            double mn = p.cpw[0][a], mx = p.cpw[0][a];
            for (int k = 1; k < p.ncp; k++) {
                mn = fmin(mn, p.cpw[k][a]);
                mx = fmax(mx, p.cpw[k][a]);
            }
            p.lo[a] = mn - bound;
            p.hi[a] = mx + bound;
        }
    }
    __syncthreads();
    const BrickRange rx = brick_range(P, p, 0), ry = brick_range(P, p, 1), rz = brick_range(P, p, 2);
    const int nxb = rx.hi - rx.lo + 1, nyb = ry.hi - ry.lo + 1, nzb = rz.hi - rz.lo + 1;
    if (nxb <= 0 || nyb <= 0 || nzb <= 0) return;
    const int total = nxb * nyb * nzb;
    for (int k = t; k < total; k += blockDim.x) {
        const int bxi = (rx.lo + k % nxb) % P.nbx;
        const int byi = (ry.lo + (k / nxb) % nyb) % P.nby;
        const int bzi = (rz.lo + k / (nxb * nyb)) % P.nbz;
        const int b = bxi + P.nbx * (byi + P.nby * bzi);
        const int slot = atomicAdd(&P.bcount[b], 1);
        if (slot < MAXPB) P.blist[b * MAXPB + slot] = j;
        else atomicOr(&P.status[ST_ERR], ERRB_BRICK_OVERFLOW);
        if (slot == 0) {  // first particle of this brick: list it for k_flags
            const int pos = atomicAdd(&P.counters[CNT_LISTED], 1);
            P.wl_list[(P.step % 3) * P.nbricks + pos] = b;
            P.stamp[b] = P.step;
            if (P.skip) P.skip[(P.step % 3) * P.nbricks + b] = P.step;
        }
    }
    if (!P.pred_stamp_next) return;
    // bricks the next step's near sweep takes: the box grown by two nodes (a
    // link, plus one node of motion); every node the next refill writes and
    // every node next to one lies inside
    const BrickRange gx = brick_range(P, p, 0, 2.0), gy = brick_range(P, p, 1, 2.0), gz = brick_range(P, p, 2, 2.0);
    const int gxb = gx.hi - gx.lo + 1, gyb = gy.hi - gy.lo + 1, gzb = gz.hi - gz.lo + 1;
    if (gxb <= 0 || gyb <= 0 || gzb <= 0) return;
    const int gtotal = gxb * gyb * gzb;
    const int next = P.step + 1;
    for (int k = t; k < gtotal; k += blockDim.x) {
        const int bxi = (gx.lo + k % gxb) % P.nbx;
        const int byi = (gy.lo + (k / gxb) % gyb) % P.nby;
        const int bzi = (gz.lo + k / (gxb * gyb)) % P.nbz;
        const int b = bxi + P.nbx * (byi + P.nby * bzi);
        if (atomicExch(&P.pred_stamp_next[b], next) != next) {
            const int pos = atomicAdd(&P.pred_count[next % 3], 1);
            P.pred_list_next[pos] = b;
            if (P.skip) P.skip[(next % 3) * P.nbricks + b] = next;
        }
    }
}

__global__ void __launch_bounds__(256) k_bin(Params P) {
    // predicted-near counts, ring of three by step: slot step+1 is filled by
    // the binning; slot step+2 (consumed by the near sweep of step-1) is
    // cleared for the next binning
    if (blockIdx.x == 0 && threadIdx.x == 0 && P.pred_count) P.pred_count[(P.step + 2) % 3] = 0;
    // this step's list of the near set's link-free bricks, filled by the near
    // sweep (its reader two steps back finished before the last near sweep)
    if (blockIdx.x == 0 && threadIdx.x == 0 && P.np_count) *P.np_count = 0;
    if (P.bin_next && blockIdx.x == gridDim.x - 1) {
        // the region of step + 1 (that of step - 1, whose readers are done:
        // they ran before this kernel on the same stream)
        int4 *z = static_cast<int4 *>(P.bin_next);
        const long long n16 = P.bin_next_bytes / 16;
        for (long long k = threadIdx.x; k < n16; k += blockDim.x) z[k] = make_int4(0, 0, 0, 0);
        return;
    }
    if ((int)blockIdx.x < P.np) bin_particle(P, blockIdx.x);
}

// Batched binning: one CTA per (case, particle), at least one per case.  The
// first CTA of a case also clears the other parity's per-step region for the
// next step (the forces of this step's predecessor stay readable until then).
__global__ void __launch_bounds__(256) k_bin_batch(BatchArgs B) {
    __shared__ Params sP;
    const int item = blockIdx.x;
    const int c = case_of(B.item_off, B.ncases, item);
    const int j = item - B.item_off[c];
    load_case_params(B, c, B.ctr, sP);
    if (j == 0) {
        if (threadIdx.x == 0 && sP.pred_count) sP.pred_count[(sP.step + 2) % 3] = 0;
        int4 *z = static_cast<int4 *>(sP.bin_next);
        const long long n16 = sP.bin_next_bytes / 16;
        for (long long k = threadIdx.x; k < n16; k += blockDim.x) z[k] = make_int4(0, 0, 0, 0);
    }
    if (j < sP.np) bin_particle(sP, j);
}

void launch_bin_batch(const BatchArgs &B, int grid, cudaStream_t st) { k_bin_batch<<<grid, 256, 0, st>>>(B); }

// ---------------------------------------------------------------------------
// k_force_reduce: one CTA per particle; each thread sums the partials of a
// fixed subset of the particle's bricks, then the CTA reduces in a fixed
// order, so the FP64 totals are reproducible run to run.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_force_reduce(Params P) {
    const int j = blockIdx.x;
    const DevParticle &p = P.parts[j];
    const int t = threadIdx.x;
    const BrickRange rx = brick_range(P, p, 0), ry = brick_range(P, p, 1), rz = brick_range(P, p, 2);
    const int nxb = rx.hi - rx.lo + 1, nyb = ry.hi - ry.lo + 1, nzb = rz.hi - rz.lo + 1;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (nxb > 0 && nyb > 0 && nzb > 0) {
        const int total = nxb * nyb * nzb;
        for (int k = t; k < total; k += blockDim.x) {
            const int bxi = (rx.lo + k % nxb) % P.nbx;
            const int byi = (ry.lo + (k / nxb) % nyb) % P.nby;
            const int bzi = (rz.lo + k / (nxb * nyb)) % P.nbz;
            const int b = bxi + P.nbx * (byi + P.nby * bzi);
            const int c = min(P.bcount[b], MAXPB);
            for (int s = 0; s < c; s++) {
                if (P.blist[b * MAXPB + s] == j) {
                    for (int q = 0; q < 6; q++) acc[q] += P.partial[((long long)b * MAXPB + s) * 6 + q];
                    break;
                }
            }
        }
    }
    __shared__ double red[8][6];
    const int lane = t & 31, warp = t >> 5;
    for (int q = 0; q < 6; q++) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (t < 6) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); w++) s += red[w][t];
        if (t < 3) P.Fh[3 * j + t] = s;
        else P.Th[3 * j + t - 3] = s;
    }
}

// ---------------------------------------------------------------------------
// DEM.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rotm(const double q[4], double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
__device__ __forceinline__ void mv(const double A[9], const double v[3], double r[3]) {
    r[0] = A[0] * v[0] + A[1] * v[1] + A[2] * v[2];
    r[1] = A[3] * v[0] + A[4] * v[1] + A[5] * v[2];
    r[2] = A[6] * v[0] + A[7] * v[1] + A[8] * v[2];
}
__device__ __forceinline__ void mtv(const double A[9], const double v[3], double r[3]) {
    r[0] = A[0] * v[0] + A[3] * v[1] + A[6] * v[2];
    r[1] = A[1] * v[0] + A[4] * v[1] + A[7] * v[2];
    r[2] = A[2] * v[0] + A[5] * v[1] + A[8] * v[2];
}

// M, grad M and Hessian of Eq. (4) at x (world, minimum image).
__device__ void mb_dd(const Params &P, const DevParticle &p, const double x[3], double &M, double g[3], double H[9]) {
    M = 0.0;
    for (int a = 0; a < 3; a++) g[a] = 0.0;
    for (int a = 0; a < 9; a++) H[a] = 0.0;
    for (int k = 0; k < p.ncp; k++) {
        double r[3];
        for (int a = 0; a < 3; a++) r[a] = minimg_d(P, a, x[a] - p.cpw[k][a]);
        const double r2 = dot3(r, r);
        const double K = p.K[k];
        const double i2 = 1.0 / (r2 * r2);
        M += K / r2;
        for (int a = 0; a < 3; a++) g[a] += -2.0 * K * r[a] * i2;
        const double i3 = 8.0 * K / (r2 * r2 * r2);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) H[3 * a + b] += i3 * r[a] * r[b] - (a == b ? 2.0 * K * i2 : 0.0);
    }
}

__device__ bool solve_sym3(const double H[9], const double b[3], double x[3]) {
    const double c0 = H[4] * H[8] - H[5] * H[7];
    const double c1 = H[5] * H[6] - H[3] * H[8];
    const double c2 = H[3] * H[7] - H[4] * H[6];
    const double det = H[0] * c0 + H[1] * c1 + H[2] * c2;
    if (det == 0.0 || !isfinite(det)) return false;
    const double id = 1.0 / det;
    const double B[9] = {c0 * id, (H[2] * H[7] - H[1] * H[8]) * id, (H[1] * H[5] - H[2] * H[4]) * id,
                         c1 * id, (H[0] * H[8] - H[2] * H[6]) * id, (H[2] * H[3] - H[0] * H[5]) * id,
                         c2 * id, (H[1] * H[6] - H[0] * H[7]) * id, (H[0] * H[4] - H[1] * H[3]) * id};
    mv(B, b, x);
    return true;
}

// Contact law of §2.1.1 (Eqs. (2)-(3)) at contact point velocities vi, vj;
// xi is the tangential spring (advanced by v_t h, kept in the tangent plane,
// reset on sliding); returns the force on body i.  F_n >= 0.
__device__ void contact_law(const Params &P, double delta, const double n[3], const double vi[3], const double vj[3],
                            double xi[3], double h, double F[3]) {
    const double vij[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
    const double vn = dot3(vij, n);
    double Fn = P.kn * delta - P.eta_n * vn;
    if (Fn < 0.0) Fn = 0.0;
    double vt[3];
    for (int a = 0; a < 3; a++) vt[a] = vij[a] - vn * n[a];
    const double xn = dot3(xi, n);
    for (int a = 0; a < 3; a++) xi[a] = xi[a] - xn * n[a] + vt[a] * h;
    double Ft[3];
    for (int a = 0; a < 3; a++) Ft[a] = -P.kt * xi[a] - P.eta_t * vt[a];
    const double ft = sqrt(dot3(Ft, Ft));
    if (ft > P.mu_s * Fn) {
        const double sc = ft > 0.0 ? P.mu_s * Fn / ft : 0.0;
        for (int a = 0; a < 3; a++) {
            Ft[a] *= sc;
            xi[a] = P.kt > 0.0 ? -(Ft[a] + P.eta_t * vt[a]) / P.kt : 0.0;
        }
    }
    for (int a = 0; a < 3; a++) F[a] = Fn * n[a] + Ft[a];
}

__device__ void point_vel(const Params &P, const DevParticle &p, const double x[3], double v[3]) {
    double r[3], wr[3];
    for (int a = 0; a < 3; a++) r[a] = minimg_d(P, a, x[a] - p.x[a]);
    cross3(p.w, r, wr);
    for (int a = 0; a < 3; a++) v[a] = p.v[a] + wr[a];
}

// Pair geometry, Eqs. (5)-(9): Newton on grad(M_i + M_j) = 0 from the warm
// start or the midpoint of the closest control-point pair; a contact needs
// c_tol < M < 1 for both; closest points by the first-order Taylor step of
// Eqs. (7)-(8); contact point in the middle of the overlap.  `valid`: Newton
// converged to a point within those bounds (the next solve may start there).
__device__ bool pair_geometry(const Params &P, const DevParticle &pi, const DevParticle &pj, bool warm,
                              double xm[3], double &delta, double nv[3], double xcp[3], bool &valid) {
    double x[3];
    if (warm) {
        for (int a = 0; a < 3; a++) x[a] = xm[a];
    } else {
        double best = 1e300;
        for (int a = 0; a < pi.ncp; a++)
            for (int b = 0; b < pj.ncp; b++) {
                double dd[3];
                for (int c = 0; c < 3; c++) dd[c] = minimg_d(P, c, pj.cpw[b][c] - pi.cpw[a][c]);
                const double d2 = dot3(dd, dd);
                if (d2 < best) {
                    best = d2;
                    for (int c = 0; c < 3; c++) x[c] = pi.cpw[a][c] + 0.5 * dd[c];
                }
            }
    }
    bool converged = false;
    valid = false;
    for (int it = 0; it < 50; it++) {
        double M0, g0[3], H0[9], M1, g1[3], H1[9];
        mb_dd(P, pi, x, M0, g0, H0);
        mb_dd(P, pj, x, M1, g1, H1);
        double g[3], H[9], dx[3];
        for (int a = 0; a < 3; a++) g[a] = -(g0[a] + g1[a]);
        for (int a = 0; a < 9; a++) H[a] = H0[a] + H1[a];
        if (!solve_sym3(H, g, dx)) break;
        for (int a = 0; a < 3; a++) x[a] += dx[a];
        if (sqrt(dot3(dx, dx)) < 1e-12) { converged = true; break; }
    }
    for (int a = 0; a < 3; a++) xm[a] = x[a];
    double M0, g0[3], H0[9], M1, g1[3], H1[9];
    mb_dd(P, pi, x, M0, g0, H0);
    mb_dd(P, pj, x, M1, g1, H1);
    if (!(M0 > P.c_tol && M0 < 1.0 && M1 > P.c_tol && M1 < 1.0)) return false;
    valid = converged;
    const double q0 = (1.0 - M0) / dot3(g0, g0), q1 = (1.0 - M1) / dot3(g1, g1);
    double xc0[3], dc[3];
    for (int a = 0; a < 3; a++) {
        xc0[a] = x[a] + q0 * g0[a];
        dc[a] = xc0[a] - (x[a] + q1 * g1[a]);
    }
    const double dist = sqrt(dot3(dc, dc));
    delta = pi.Rs + pj.Rs - dist;
    if (!(delta > 0.0) || dist == 0.0) return false;
    for (int a = 0; a < 3; a++) {
        nv[a] = dc[a] / dist;
        xcp[a] = xc0[a] - (pi.Rs - 0.5 * delta) * nv[a];
    }
    return true;
}

// Wall geometry, Eqs. (10)-(13): Newton on the two tangential components of
// grad M on the wall plane, dM/dm < 0 along the outward normal m; start from
// the warm start or the projection of the control point nearest the plane.
// `valid`: Newton converged and dM/dm < 0 there.
__device__ bool wall_geometry(const Params &P, const DevParticle &p, int wall, bool warm, double xcw[3],
                              double &delta, double nv[3], double xcp[3], bool &valid) {
    const int ax = wall / 2, side = wall % 2;
    const double plane = side ? dim_of(P, ax) - 0.5 : -0.5;
    const double m_ax = side ? 1.0 : -1.0;
    const int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
    double x[3];
    if (warm) {
        for (int a = 0; a < 3; a++) x[a] = xcw[a];
    } else {
        int kb = 0;
        double best = 1e300;
        for (int k = 0; k < p.ncp; k++) {
            const double dd = fabs(plane - p.cpw[k][ax]);
            if (dd < best) { best = dd; kb = k; }
        }
        for (int a = 0; a < 3; a++) x[a] = p.cpw[kb][a];
    }
    x[ax] = plane;
    bool converged = false;
    valid = false;
    for (int it = 0; it < 50; it++) {
        double M, g[3], H[9];
        mb_dd(P, p, x, M, g, H);
        const double J00 = H[3 * t1 + t1], J01 = H[3 * t1 + t2], J10 = H[3 * t2 + t1], J11 = H[3 * t2 + t2];
        const double det = J00 * J11 - J01 * J10;
        if (det == 0.0 || !isfinite(det)) break;
        const double r0 = -g[t1], r1 = -g[t2];
        const double d0 = (J11 * r0 - J01 * r1) / det, d1 = (-J10 * r0 + J00 * r1) / det;
        x[t1] += d0;
        x[t2] += d1;
        if (sqrt(d0 * d0 + d1 * d1) < 1e-12) { converged = true; break; }
    }
    for (int a = 0; a < 3; a++) xcw[a] = x[a];
    double M, g[3], H[9];
    mb_dd(P, p, x, M, g, H);
    if (!(g[ax] * m_ax < 0.0)) return false;
    valid = converged;
    const double qR = (1.0 - M) / dot3(g, g);
    double dc[3];
    for (int a = 0; a < 3; a++) dc[a] = qR * g[a];
    const double dist = sqrt(dot3(dc, dc));
    delta = p.Rs - dist;
    if (!(delta > 0.0) || dist == 0.0) return false;
    for (int a = 0; a < 3; a++) {
        nv[a] = dc[a] / dist;
        xcp[a] = x[a] - 0.5 * delta * nv[a];
    }
    return true;
}

__device__ double bounding_radius(const DevParticle &p) { return p.brad; }

// All contact forces at the current state: pairs (strided over the CTA),
// then per particle the pair terms in index order followed by the walls.
__device__ void contacts(const Params &P, double h) {
    const int np = P.np;
    const int t = threadIdx.x;
    for (int idx = t; idx < np * np; idx += blockDim.x) {
        const int i = idx / np, j = idx % np;
        if (j <= i) continue;
        double *out = P.pairF + (long long)idx * 9;
        for (int a = 0; a < 9; a++) out[a] = 0.0;
        const DevParticle &pi = P.parts[i], &pj = P.parts[j];
        double dx[3];
        for (int a = 0; a < 3; a++) dx[a] = minimg_d(P, a, pj.x[a] - pi.x[a]);
        if (sqrt(dot3(dx, dx)) > pi.brad + pj.brad) {
            P.pair_on[idx] = 0;
            continue;
        }
        double xm[3], delta, nv[3], xcp[3];
        const int was = P.pair_on[idx];
        bool valid;
        for (int a = 0; a < 3; a++) xm[a] = P.pair_xm[3 * idx + a];
        const bool hit = pair_geometry(P, pi, pj, (was & CONTACT_WARM) != 0, xm, delta, nv, xcp, valid);
        for (int a = 0; a < 3; a++) P.pair_xm[3 * idx + a] = xm[a];
        const int warm = valid ? CONTACT_WARM : 0;
        if (!hit) {
            P.pair_on[idx] = warm;
            continue;
        }
        double xi[3];
        for (int a = 0; a < 3; a++) xi[a] = (was & CONTACT_ON) ? P.pair_xi[3 * idx + a] : 0.0;
        P.pair_on[idx] = warm | CONTACT_ON;
        double vi[3], vj[3], Fi[3];
        point_vel(P, pi, xcp, vi);
        point_vel(P, pj, xcp, vj);
        contact_law(P, delta, nv, vi, vj, xi, h, Fi);
        for (int a = 0; a < 3; a++) P.pair_xi[3 * idx + a] = xi[a];
        double ri[3], rj[3], Fj[3], ti[3], tj[3];
        for (int a = 0; a < 3; a++) {
            ri[a] = minimg_d(P, a, xcp[a] - pi.x[a]);
            rj[a] = minimg_d(P, a, xcp[a] - pj.x[a]);
            Fj[a] = -Fi[a];
        }
        cross3(ri, Fi, ti);
        cross3(rj, Fj, tj);
        for (int a = 0; a < 3; a++) { out[a] = Fi[a]; out[3 + a] = ti[a]; out[6 + a] = tj[a]; }
    }
    __syncthreads();
    for (int k = t; k < np; k += blockDim.x) {
        double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
        for (int m = 0; m < np; m++) {
            if (m < k) {
                const double *o = P.pairF + ((long long)m * np + k) * 9;
                for (int a = 0; a < 3; a++) { F[a] += -o[a]; T[a] += o[6 + a]; }
            } else if (m > k) {
                const double *o = P.pairF + ((long long)k * np + m) * 9;
                for (int a = 0; a < 3; a++) { F[a] += o[a]; T[a] += o[3 + a]; }
            }
        }
        const DevParticle &p = P.parts[k];
        for (int wall = 0; wall < NWALL; wall++) {
            const int ax = wall / 2, side = wall % 2;
            const int wj = k * NWALL + wall;
            if (P.per[ax]) { P.wall_on[wj] = 0; continue; }
            const double plane = side ? dim_of(P, ax) - 0.5 : -0.5;
            if (fabs(plane - p.x[ax]) > p.brad) { P.wall_on[wj] = 0; continue; }
            double xcw[3], delta, nv[3], xcp[3];
            const int was = P.wall_on[wj];
            bool valid;
            for (int a = 0; a < 3; a++) xcw[a] = P.wall_xcw[3 * wj + a];
            const bool hit = wall_geometry(P, p, wall, (was & CONTACT_WARM) != 0, xcw, delta, nv, xcp, valid);
            for (int a = 0; a < 3; a++) P.wall_xcw[3 * wj + a] = xcw[a];
            const int warm = valid ? CONTACT_WARM : 0;
            if (!hit) { P.wall_on[wj] = warm; continue; }
            double xi[3];
            for (int a = 0; a < 3; a++) xi[a] = (was & CONTACT_ON) ? P.wall_xi[3 * wj + a] : 0.0;
            P.wall_on[wj] = warm | CONTACT_ON;
            double vi[3], vw[3] = {0, 0, 0}, Fi[3], ri[3], ti[3];
            point_vel(P, p, xcp, vi);
            contact_law(P, delta, nv, vi, vw, xi, h, Fi);
            for (int a = 0; a < 3; a++) P.wall_xi[3 * wj + a] = xi[a];
            for (int a = 0; a < 3; a++) ri[a] = minimg_d(P, a, xcp[a] - p.x[a]);
            cross3(ri, Fi, ti);
            for (int a = 0; a < 3; a++) { F[a] += Fi[a]; T[a] += ti[a]; }
        }
        for (int a = 0; a < 3; a++) { P.Fc[3 * k + a] = F[a]; P.Tc[3 * k + a] = T[a]; }
    }
    __syncthreads();
}

// One rotational sub-step: half-kick, rotate with the half-step rate, then
// the closing half-kick solved by ROT_ITERS fixed-point sweeps; wb and Tb are
// body-frame (principal) quantities, Tb is refreshed for the new orientation.
__device__ __forceinline__ void rotate_substep(const DevParticle &p, double q[4], double wb[3], double Tb[3],
                                               const double Tw[3], double h) {
    double dw[3], wh[3];
    euler_rate(p, wb, Tb, dw);
    for (int a = 0; a < 3; a++) wh[a] = wb[a] + 0.5 * h * dw[a];
    quat_step(q, wh, h);
    rot_body(q, Tw, Tb);
    double w1[3] = {wh[0], wh[1], wh[2]};
    for (int it = 0; it < ROT_ITERS; it++) {
        euler_rate(p, w1, Tb, dw);
        for (int a = 0; a < 3; a++) w1[a] = wh[a] + 0.5 * h * dw[a];
    }
    for (int a = 0; a < 3; a++) wb[a] = w1[a];
}

__device__ void refresh_cpw(const Params &P) {
    for (int idx = threadIdx.x; idx < P.np * MAXCP; idx += blockDim.x) {
        DevParticle &p = P.parts[idx / MAXCP];
        const int k = idx % MAXCP;
        if (k < p.ncp) {
            double r[3];
            quat_rot(p.q, p.cpb[k], r);
            for (int a = 0; a < 3; a++) p.cpw[k][a] = p.x[a] + r[a];
        }
    }
    __syncthreads();
}

constexpr int kFastMaxParticles = 256;

// Whether some contact can occur during this LBM step.  Without contacts a
// particle moves by at most |v| + |a| over the unit step (a = the frozen
// acceleration), so when every bounding-sphere gap to a wall exceeds the
// particle's bound, every gap between two particles exceeds the sum of their
// bounds, and no contact is active, none starts during the step (the first
// one would need a larger displacement first).  Tested in FP32 with a margin
// of 1e-2 that covers its rounding; a doubtful case counts as "possible".
__device__ bool contact_possible(const Params &P) {
    __shared__ float xs[kFastMaxParticles][3], reach[kFastMaxParticles], br[kFastMaxParticles];
    __shared__ int s_possible;
    const int np = P.np;
    if (np > kFastMaxParticles) return true;
    if (threadIdx.x == 0) s_possible = 0;
    __syncthreads();
    int possible = 0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const DevParticle &p = P.parts[k];
        double D = 0.0;
        if (!p.fixed) {
            double a2 = 0.0;
            for (int a = 0; a < 3; a++) {
                const double acc = p.buoy * P.g[a] + P.Fh[3 * k + a] * p.inv_mass;
                a2 += acc * acc;
            }
            D = sqrt(dot3(p.v, p.v)) + sqrt(a2);
        }
        const float Df = (float)D * 1.0001f + 1e-4f;
        for (int a = 0; a < 3; a++) xs[k][a] = (float)p.x[a];
        reach[k] = Df;
        br[k] = (float)p.brad;
        for (int wall = 0; wall < NWALL; wall++) {
            if (P.wall_on[k * NWALL + wall] & CONTACT_ON) possible = 1;
            const int ax = wall / 2, side = wall % 2;
            if (P.per[ax]) continue;
            const float plane = side ? (float)dim_of(P, ax) - 0.5f : -0.5f;
            if (fabsf(plane - (float)p.x[ax]) - br[k] <= Df + 1e-2f) possible = 1;
        }
    }
    __syncthreads();
    // warp w takes rows w, w + nwarp, ..., its lanes the columns j > i
    const int lane = threadIdx.x & 31, nwarp = (blockDim.x + 31) >> 5;
    for (int i = threadIdx.x >> 5; i < np && !possible; i += nwarp)
        for (int j = i + 1 + lane; j < np; j += 32) {
            if (P.pair_on[i * np + j] & CONTACT_ON) { possible = 1; break; }
            float d2 = 0.f;
            for (int a = 0; a < 3; a++) {
                float d = xs[j][a] - xs[i][a];
                if (P.per[a]) {
                    const float L = (float)dim_of(P, a);
                    d -= L * rintf(d / L);
                }
                d2 += d * d;
            }
            const float lim = br[i] + br[j] + reach[i] + reach[j] + 1e-2f;
            if (d2 <= lim * lim) { possible = 1; break; }
        }
    if (possible) atomicOr(&s_possible, 1);
    __syncthreads();
    return s_possible != 0;
}

// ---------------------------------------------------------------------------
// Rotation of a contact-free particle, four lanes per particle.  Lane 0 holds
// the quaternion's scalar part, lanes 1..3 its vector part and the x,y,z
// components of every vector (lane 0's vector slot is unused), so the cross
// products, the quaternion product and Euler's equations run one component
// per lane with width-4 shuffles.  FP64 throughout.
// ---------------------------------------------------------------------------
// lanes of the quads that take part (whole quads); set by the caller
__device__ __forceinline__ double qget(unsigned mask, double v, int lane) { return __shfl_sync(mask, v, lane, 4); }

// (a x b) for this lane's axis m = lane - 1 (lanes 1..3)
// Per-lane shuffle sources, fixed for the whole sub-step loop.
struct QuadLanes {
    int lane;      // 0..3
    int l1, l2;    // lanes of the next two axes (cyclic) of this lane's axis
    int p1, p2, p3;        // quaternion product: lanes of d paired with q1, q2, q3
    double s1, s2, s3;     // and their signs
};

__device__ __forceinline__ QuadLanes quad_lanes() {
    QuadLanes L;
    L.lane = threadIdx.x & 3;
    const int m = L.lane == 0 ? 0 : L.lane - 1;
    L.l1 = 1 + (m + 1) % 3;
    L.l2 = 1 + (m + 2) % 3;
    // r = q (x) d:  r_k = q0 d_k + s1 q1 d_p1 + s2 q2 d_p2 + s3 q3 d_p3
    const int P1[4] = {1, 0, 3, 2}, P2[4] = {2, 3, 0, 1}, P3[4] = {3, 2, 1, 0};
    const double S1[4] = {-1, 1, -1, 1}, S2[4] = {-1, 1, 1, -1}, S3[4] = {-1, -1, 1, 1};
    L.p1 = P1[L.lane]; L.p2 = P2[L.lane]; L.p3 = P3[L.lane];
    L.s1 = S1[L.lane]; L.s2 = S2[L.lane]; L.s3 = S3[L.lane];
    return L;
}

// (a x b), this lane's axis (lanes 1..3)
__device__ __forceinline__ double qcross(unsigned mk, const QuadLanes &L, double a, double b) {
    const double a1 = qget(mk, a, L.l1), a2 = qget(mk, a, L.l2), b1 = qget(mk, b, L.l1), b2 = qget(mk, b, L.l2);
    return a1 * b2 - a2 * b1;
}
// sum over lanes 1..3
__device__ __forceinline__ double qsum3(unsigned mk, const QuadLanes &L, double v) {
    double t = L.lane == 0 ? 0.0 : v;
    t += __shfl_xor_sync(mk, t, 1, 4);
    t += __shfl_xor_sync(mk, t, 2, 4);
    return t;
}
// Euler's equations in the principal frame, this lane's axis
__device__ __forceinline__ double qeuler(unsigned mk, const QuadLanes &L, double w, double Tb, double iI, double cI) {
    const double w1 = qget(mk, w, L.l1), w2 = qget(mk, w, L.l2);
    return fma(cI * w1, w2, iI * Tb);
}
// R(q)^T v (body components of a world vector), R(q) v when toward_world
__device__ __forceinline__ double qrotate(unsigned mk, const QuadLanes &L, double q, double v, bool toward_world) {
    const double c = qcross(mk, L, q, v);      // u x v
    const double uc = qcross(mk, L, q, c);     // u x (u x v)
    const double w = qget(mk, q, 0);
    return v + 2.0 * (toward_world ? fma(w, c, uc) : fma(-w, c, uc));
}

// Rotation sub-steps of one free particle by its quad of lanes; mk holds the
// lanes of every quad of this warp that takes part.  FP64 throughout.
//
// On this GPU an FP64 warp instruction occupies its sub-partition for 64
// cycles, so the sub-step is written for few of them (26 per sub-step, for
// every quad of the warp at once); shuffles, sign flips and compares run on
// other pipes.  It is the same sub-step as rotate_substep and the oracle's,
// rearranged:
// - half-kick  wh = wb + hh f(wb, Tb) as fma(hh cI w_{l+1}, w_{l+2}, wb + hh iI Tb);
// - exp(h wh / 2) = (c, sc wh) with c and sc from their Taylor series in
//   s2 = |wh|^2, two terms past the leading one (truncation below 1e-18 while
//   a2 = (h/2)^2 s2 <= 1e-5, i.e. |w| h <= 6e-3; larger a2 takes the longer
//   series or sincos);
// - the body-frame torque of the new orientation, R(q (x) d)^T T_w =
//   R(d)^T R(q)^T T_w, from the previous one: Tb' = Tb - 2 c X + 2 s x X,
//   X = s x Tb, (c, s) = d (the same rotation; the rounding differs from
//   rebuilding it from q by ~1e-16 per sub-step, and Tb is rebuilt from q at
//   every LBM step);
// - the closing half-kick's ROT_ITERS = 2 fixed-point sweeps with the
//   constants hh cI, hh iI folded in;
// - q <- q (x) d with the signs of the quaternion product applied as sign
//   flips of the shuffled q.
__device__ __forceinline__ double dneg_if(double v, bool neg) {
    return __longlong_as_double(__double_as_longlong(v) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}

// Tw_lane: this lane's component of the world-frame torque (lane 0: not
// used); the new attitude and world angular velocity go to q_out[4] and
// w_out[3] (which may be p's own).
__device__ void rotate_free_quad(unsigned mk, const DevParticle &p, double Tw_lane, double h, int n_sub,
                                 double *q_out, double *w_out) {
    const QuadLanes L = quad_lanes();
    const int lane = L.lane;
    const int m = lane == 0 ? 0 : lane - 1;
    double q = p.q[lane];
    const double Tw = lane == 0 ? 0.0 : Tw_lane;
    double wb = qrotate(mk, L, q, lane == 0 ? 0.0 : p.w[m], false);
    double Tb = qrotate(mk, L, q, Tw, false);
    if (__all_sync(mk, wb == 0.0 && Tb == 0.0)) {  // nothing turns
        q_out[lane] = q;
        if (lane > 0) w_out[m] = p.w[m];
        return;
    }
    const double hh = 0.5 * h, qh2 = 0.25 * h * h;
    // per-lane constants (lane 0 holds the quaternion's scalar part only)
    const double cIhh = lane == 0 ? 0.0 : hh * p.cI[m];
    const double iIhh = lane == 0 ? 0.0 : hh * p.iI[m];
    // c = 1 - a2/2 + a2^2/24 (lane 0), sc = hh (1 - a2/6 + a2^2/120)
    // (lanes 1..3), a2 = qh2 s2: as polynomials in s2
    const double k2 = lane == 0 ? qh2 * qh2 * (1.0 / 24.0) : hh * qh2 * qh2 * (1.0 / 120.0);
    const double k1 = lane == 0 ? -0.5 * qh2 : -hh * qh2 * (1.0 / 6.0);
    const double k0 = lane == 0 ? 1.0 : hh;
    // s2 bound for the short series: a2 <= 1e-5
    const long long s2_short = __double_as_longlong(1e-5 / qh2);
    const bool neg1 = L.s1 < 0.0, neg2 = L.s2 < 0.0, neg3 = L.s3 < 0.0;
    double hT = iIhh * Tb;
    for (int sub = 0; sub < n_sub; sub++) {
        // first half-kick
        const double w1 = qget(mk, wb, L.l1), w2 = qget(mk, wb, L.l2);
        const double wh = fma(cIhh * w1, w2, wb + hT);
        // exp(h wh / 2)
        // (lane 0's vector slots carry qrotate's x component: left out)
        double sq = lane == 0 ? 0.0 : wh * wh;
        double s2 = sq + __shfl_xor_sync(mk, sq, 1, 4);
        s2 += __shfl_xor_sync(mk, s2, 2, 4);
        double d;
        if (__all_sync(mk, __double_as_longlong(s2) <= s2_short)) {
            const double poly = fma(s2, fma(s2, k2, k1), k0);
            d = poly * (lane == 0 ? 1.0 : wh);
        } else {
            const double a2 = qh2 * s2;
            double sc, c;
            if (a2 <= 1.0 / 256.0) {
                sc = hh * (1.0 + a2 * (-1.0 / 6.0 + a2 * (1.0 / 120.0 + a2 * (-1.0 / 5040.0 + a2 * (1.0 / 362880.0 + a2 * (-1.0 / 39916800.0))))));
                c = 1.0 + a2 * (-0.5 + a2 * (1.0 / 24.0 + a2 * (-1.0 / 720.0 + a2 * (1.0 / 40320.0 + a2 * (-1.0 / 3628800.0)))));
            } else {
                const double wn = sqrt(s2);
                double sn;
                sincos(hh * wn, &sn, &c);
                sc = sn / wn;
            }
            d = lane == 0 ? c : sc * wh;
        }
        // body-frame torque of the new orientation: Tb + 2 (s x (s x Tb)) - 2 c (s x Tb)
        const double s1 = qget(mk, d, L.l1), s2v = qget(mk, d, L.l2);
        const double T1 = qget(mk, Tb, L.l1), T2 = qget(mk, Tb, L.l2);
        const double X = fma(s1, T2, -(s2v * T1));
        const double X1 = qget(mk, X, L.l1), X2 = qget(mk, X, L.l2);
        const double Y = fma(s1, X2, -(s2v * X1));
        const double cc = qget(mk, d, 0);
        Tb = fma(-2.0 * cc, X, fma(2.0, Y, Tb));
        hT = iIhh * Tb;
        // closing half-kick, two fixed-point sweeps
        const double t1 = wh + hT;
        const double v1 = fma(cIhh * qget(mk, wh, L.l1), qget(mk, wh, L.l2), t1);
        wb = fma(cIhh * qget(mk, v1, L.l1), qget(mk, v1, L.l2), t1);
        // q <- q (x) d
        const double q0 = qget(mk, q, 0), q1 = qget(mk, q, 1), q2 = qget(mk, q, 2), q3 = qget(mk, q, 3);
        const double dp1 = qget(mk, d, L.p1), dp2 = qget(mk, d, L.p2), dp3 = qget(mk, d, L.p3);
        q = fma(dneg_if(q3, neg3), dp3, fma(dneg_if(q2, neg2), dp2, fma(dneg_if(q1, neg1), dp1, q0 * d)));
    }
    // renormalise once per LBM step, back to world frame
    double n2 = q * q;
    n2 += __shfl_xor_sync(mk, n2, 1, 4);
    n2 += __shfl_xor_sync(mk, n2, 2, 4);
    q *= rsqrt(n2);
    const double ww = qrotate(mk, L, q, wb, true);
    q_out[lane] = q;
    if (lane > 0) w_out[m] = ww;
}

// ---------------------------------------------------------------------------
// FP64 rigid-body integration on lattices stored below FP64 (the default):
// k_dem64_free moves every particle as if it could touch nothing during the
// step, into the records' step results, while k_dem64_plan splits the
// particles on the other stream and k_dem64t / k_dem64c (k_dem32.cu) move the
// ones that can touch something; k_dem64_commit then gives the others their
// step results.
// ---------------------------------------------------------------------------

// One CTA.  The hydrodynamic load as FP64 totals (from the sweep's
// fixed-point sums), then the split: a particle is active when its bounding
// sphere can reach a wall, or another particle's, during the step (gap <=
// reach_i + reach_j, dem_reach).  Active particles that can reach each other
// form a contact group (connected components of that relation); groups are
// independent during the step, so each gets its own CTA.  Every list keeps
// index order (dem_free() and below).  A pair or wall with contact history
// at the end of the last step (in contact, or a warm Newton start) had its
// bounding spheres overlapping, or the wall within the bounding sphere, so
// it is active again: the contact history of inactive particles is empty.
constexpr int kPlanEdges = 4096;
static_assert(kDem32MaxParticles <= kFastMaxParticles, "one plan thread per particle");
static_assert(kFastMaxParticles < 4096, "the plan's block scan packs 12-bit counts");
__global__ void __launch_bounds__(256) k_dem64_plan(Params P) {
    // one thread per particle below (np <= kFastMaxParticles = blockDim.x)
    __shared__ float xs[kFastMaxParticles][3], reach[kFastMaxParticles], br[kFastMaxParticles];
    __shared__ int act[kFastMaxParticles], parent[kFastMaxParticles], gsz[kFastMaxParticles];
    __shared__ int root[kFastMaxParticles];
    __shared__ unsigned long long wsum[kFastMaxParticles / 32];
    __shared__ unsigned edge[kPlanEdges];
    __shared__ int nedge;
    const int np = P.np;
    if (threadIdx.x == 0) nedge = 0;
    for (int i = threadIdx.x; i < np * 6; i += blockDim.x) {
        const double v = (double)(long long)P.Ffix[i] * (1.0 / (double)(1ull << kForceFixBits));
        const int k = i / 6, c = i % 6;
        if (c < 3) P.Fh[3 * k + c] = v;
        else P.Th[3 * k + c - 3] = v;
    }
    __syncthreads();  // dem_reach below reads the load that other threads converted
    const int k = threadIdx.x;
    if (k < np) {
        const DevParticle &p = P.parts[k];
        const float r = dem_reach(P, p, k);
        for (int a = 0; a < 3; a++) xs[k][a] = (float)p.x[a];
        reach[k] = r;
        br[k] = (float)p.brad;
        int on = 0;
        for (int wall = 0; wall < NWALL; wall++) {
            const int ax = wall / 2, side = wall % 2;
            if (P.per[ax]) continue;
            const float plane = side ? (float)dim_of(P, ax) - 0.5f : -0.5f;
            if (fabsf(plane - xs[k][ax]) - br[k] <= r + 1e-2f) on = 1;
        }
        act[k] = on;
        parent[k] = k;
        gsz[k] = 0;
    }
    __syncthreads();
    // candidate pairs: warp w takes rows w, w + 8, ..., its lanes the
    // columns j > i (consecutive j: conflict-free shared loads)
    float L[3], invL[3];
    for (int a = 0; a < 3; a++) {
        L[a] = P.per[a] ? (float)dim_of(P, a) : 0.f;
        invL[a] = P.per[a] ? 1.f / L[a] : 0.f;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int i = warp; i < np; i += nwarp) {
        const float xi0 = xs[i][0], xi1 = xs[i][1], xi2 = xs[i][2], ri = br[i] + reach[i] + 1e-2f;
        for (int j = i + 1 + lane; j < np; j += 32) {
            float d0 = xs[j][0] - xi0, d1 = xs[j][1] - xi1, d2 = xs[j][2] - xi2;
            d0 -= L[0] * rintf(d0 * invL[0]);
            d1 -= L[1] * rintf(d1 * invL[1]);
            d2 -= L[2] * rintf(d2 * invL[2]);
            const float lim = ri + br[j] + reach[j];
            if (d0 * d0 + d1 * d1 + d2 * d2 <= lim * lim) {
                act[i] = 1;
                act[j] = 1;
                const int e = atomicAdd(&nedge, 1);
                if (e < kPlanEdges) edge[e] = ((unsigned)i << 16) | (unsigned)j;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // connected components of the edges (union by the smaller root, so a
        // root is its group's smallest index: the partition and its roots do
        // not depend on the order of the edges); beyond the edge table,
        // every active particle is one group
        auto find = [&](int a) {
            while (parent[a] != a) {
                parent[a] = parent[parent[a]];
                a = parent[a];
            }
            return a;
        };
        const int ne = nedge;
        if (ne > kPlanEdges) {
            int r = -1;
            for (int m = 0; m < np; m++)
                if (act[m]) {
                    if (r < 0) r = m;
                    parent[m] = r;
                }
        } else {
            for (int e = 0; e < ne; e++) {
                const int a = find((int)(edge[e] >> 16)), b = find((int)(edge[e] & 0xFFFFu));
                if (a != b) {
                    if (a < b) parent[b] = a;
                    else parent[a] = b;
                }
            }
        }
    }
    __syncthreads();
    const bool on = k < np && act[k];
    int rk = -1;
    if (on) {
        rk = k;
        while (parent[rk] != rk) rk = parent[rk];
        root[k] = rk;
        atomicAdd(&gsz[rk], 1);
    }
    __syncthreads();
    // exclusive block scan of five 12-bit counters (np <= 256): free
    // particles, group members, and groups of each class (groups in the
    // order of their smallest member, the free list and each group in
    // ascending index)
    const int g = on && rk == k ? gsz[k] : 0;
    const int cls = g > kSmallContactGroup ? DEM_GROUP_LARGE : (g > kTinyContactGroup ? DEM_GROUP_SMALL : DEM_GROUP_TINY);
    const unsigned long long mine = (unsigned long long)(k < np && !on) |
                                    (unsigned long long)g << 12 |
                                    (unsigned long long)(g > 0) << (24 + 12 * cls);
    unsigned long long inc = mine;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    unsigned long long ex = inc - mine, tot = 0;
    for (int w = 0; w < nwarp; w++) {
        if (w < warp) ex += wsum[w];
        tot += wsum[w];
    }
    const int exf = (int)(ex & 0xFFF), exg = (int)(ex >> 12 & 0xFFF);
    if (k < np && !on) dem_free(P)[exf] = k;
    if (g > 0) {
        const int slot = (int)(ex >> (24 + 12 * cls) & 0xFFF);
        int *gl = dem_groups(P, cls);
        gl[2 * slot] = exg;
        gl[2 * slot + 1] = g;
        gsz[k] = exg;   // the group's first slot in the active list
    }
    __syncthreads();
    if (on) {
        int rank = 0;
        for (int m = rk; m < k; m++) rank += act[m] && root[m] == rk;
        dem_active(P)[gsz[rk] + rank] = k;
    }
    if (threadIdx.x == 0) {
        for (int f = 0; f < 5; f++) P.dem_list[f] = (int)(tot >> (12 * f) & 0xFFF);
    }
}

// Four lanes per particle, 32 particles per CTA, every particle (the plan
// runs beside it): the step of a particle that touches nothing, into its
// record's step results (nx, nv, nq, nw).  Translation in closed form over
// the unit step (x += v + a/2, v += a: what the n_s kick-drift-kick
// sub-steps give under the constant force), rotation sub-stepped by
// rotate_free_quad, all FP64.  The hydrodynamic load comes from the sweep's
// fixed-point totals by the plan's conversion (the same bits as its Fh, Th).
__global__ void __launch_bounds__(128) k_dem64_free(Params P) {
    const int np = P.np;
    const int slot = blockIdx.x * 32 + (int)(threadIdx.x >> 2);
    if (blockIdx.x * 32 + (int)((threadIdx.x & ~31u) >> 2) >= np) return;  // the whole warp is idle
    const bool has = slot < np;
    const int k = has ? slot : 0;
    const int lane = threadIdx.x & 3, m = lane == 0 ? 0 : lane - 1;
    constexpr double kFix = 1.0 / (double)(1ull << kForceFixBits);
    DevParticle &p = P.parts[k];
    const bool moving = has && !p.fixed;
    if (moving && lane > 0) {
        const double acc = p.buoy * P.g[m] + ((double)(long long)P.Ffix[6 * k + m] * kFix) * p.inv_mass;
        p.nx[m] = p.x[m] + (p.v[m] + 0.5 * acc);
        p.nv[m] = p.v[m] + acc;
    }
    const unsigned mk = __ballot_sync(0xffffffffu, moving);
    if (moving)
        rotate_free_quad(mk, p, (double)(long long)P.Ffix[6 * k + 3 + m] * kFix, 1.0 / P.n_sub, P.n_sub, p.nq, p.nw);
}

// The plan's inactive particles take k_dem64_free's step results; their
// contact load is zero.  One thread per inactive particle.
__global__ void __launch_bounds__(128) k_dem64_commit(Params P) {
    const int s = blockIdx.x * blockDim.x + (int)threadIdx.x;
    if (s >= P.dem_list[0]) return;
    const int k = dem_free(P)[s];
    DevParticle &p = P.parts[k];
    if (!p.fixed) {
        for (int a = 0; a < 3; a++) {
            p.x[a] = p.nx[a];
            p.v[a] = p.nv[a];
            p.w[a] = p.nw[a];
        }
        for (int a = 0; a < 4; a++) p.q[a] = p.nq[a];
    }
    for (int a = 0; a < 3; a++) {
        P.Fc[3 * k + a] = 0.0;
        P.Tc[3 * k + a] = 0.0;
    }
}

// One CTA.  Kick-drift-kick velocity Verlet with the hydrodynamic load frozen
// over the n_s sub-steps (§2.3.4); rotation by Euler's equations in the body
// frame.  When no contact can occur during the step, the translation of the
// n_s sub-steps under the constant force is taken in closed form (x += v +
// a/2, v += a over the unit step: what the sub-steps compute in exact
// arithmetic) and the rotation is sub-stepped by four FP64 lanes per
// particle.  (Lattices stored below FP64 use k_dem32 instead.)
__global__ void __launch_bounds__(256) k_dem(Params P) {
    const double h = 1.0 / P.n_sub;
    if (P.force_fixed) {
        // an FP32 lattice left the hydrodynamic load as fixed-point totals
        for (int i = threadIdx.x; i < P.np * 6; i += blockDim.x) {
            const double v = (double)(long long)P.Ffix[i] * (1.0 / (double)(1ull << kForceFixBits));
            const int k = i / 6, c = i % 6;
            if (c < 3) P.Fh[3 * k + c] = v;
            else P.Th[3 * k + c - 3] = v;
        }
        __syncthreads();
    }
    if (!contact_possible(P)) {
        for (int k = threadIdx.x; k < P.np; k += blockDim.x) {
            DevParticle &p = P.parts[k];
            if (p.fixed) continue;
            for (int a = 0; a < 3; a++) {
                const double acc = p.buoy * P.g[a] + P.Fh[3 * k + a] * p.inv_mass;
                p.x[a] += p.v[a] + 0.5 * acc;
                p.v[a] += acc;
            }
            for (int a = 0; a < 3; a++) { P.Fc[3 * k + a] = 0.0; P.Tc[3 * k + a] = 0.0; }
        }
        // rotation, one quad of lanes per moving particle; the shuffles name
        // exactly the quads that take part
        const int per_pass = blockDim.x / 4;
        for (int base = 0; base < P.np; base += per_pass) {
            const int k = base + (int)(threadIdx.x >> 2);
            const bool moving = k < P.np && !P.parts[k].fixed;
            const unsigned mk = __ballot_sync(0xffffffffu, moving);
            const int ql = threadIdx.x & 3;
            if (moving)
                rotate_free_quad(mk, P.parts[k], ql == 0 ? 0.0 : P.Th[3 * k + ql - 1], h, P.n_sub, P.parts[k].q,
                                 P.parts[k].w);
        }
        return;
    }
    // the load at the start: left by the previous step's DEM (same state),
    // unless the particles were set since
    if (!P.fc_valid) contacts(P, 0.0);
    for (int sub = 0; sub < P.n_sub; sub++) {
        for (int k = threadIdx.x; k < P.np; k += blockDim.x) {
            DevParticle &p = P.parts[k];
            if (p.fixed) continue;
            for (int a = 0; a < 3; a++) {
                const double acc = p.buoy * P.g[a] + (P.Fh[3 * k + a] + P.Fc[3 * k + a]) * p.inv_mass;
                p.v[a] += 0.5 * h * acc;
            }
            for (int a = 0; a < 3; a++) p.x[a] += h * p.v[a];
            // first rotational half-kick and the rotation (the closing
            // half-kick follows the new contact torque)
            double q[4] = {p.q[0], p.q[1], p.q[2], p.q[3]};
            double Tw[3], wb[3], Tb[3], dw[3];
            for (int a = 0; a < 3; a++) Tw[a] = P.Th[3 * k + a] + P.Tc[3 * k + a];
            rot_body(q, p.w, wb);
            rot_body(q, Tw, Tb);
            euler_rate(p, wb, Tb, dw);
            for (int a = 0; a < 3; a++) wb[a] += 0.5 * h * dw[a];
            quat_step(q, wb, h);
            quat_normalize(q);
            for (int a = 0; a < 4; a++) p.q[a] = q[a];
            rot_world(q, wb, p.w);
        }
        __syncthreads();
        refresh_cpw(P);
        contacts(P, h);
        for (int k = threadIdx.x; k < P.np; k += blockDim.x) {
            DevParticle &p = P.parts[k];
            if (p.fixed) continue;
            for (int a = 0; a < 3; a++) {
                const double acc = p.buoy * P.g[a] + (P.Fh[3 * k + a] + P.Fc[3 * k + a]) * p.inv_mass;
                p.v[a] += 0.5 * h * acc;
            }
            double Tw[3], wb[3], Tb[3], dw[3];
            for (int a = 0; a < 3; a++) Tw[a] = P.Th[3 * k + a] + P.Tc[3 * k + a];
            rot_body(p.q, p.w, wb);
            rot_body(p.q, Tw, Tb);
            double w1[3] = {wb[0], wb[1], wb[2]};
            for (int it = 0; it < ROT_ITERS; it++) {
                euler_rate(p, w1, Tb, dw);
                for (int a = 0; a < 3; a++) w1[a] = wb[a] + 0.5 * h * dw[a];
            }
            rot_world(p.q, w1, p.w);
        }
        __syncthreads();
    }
    // contact load of the end state (springs not advanced): reported by
    // lbm_get_contact_forces and the start load of the next step
    contacts(P, 0.0);
}

void launch_bin(const Params &P, cudaStream_t st) {
    // runs every step, with no particle too (it keeps the count ring); one
    // more CTA clears the next step's per-step region
    k_bin<<<(P.np > 0 ? P.np : 1) + (P.bin_next ? 1 : 0), 256, 0, st>>>(P);
}
void launch_force_reduce(const Params &P, cudaStream_t st) {
    if (P.np > 0) k_force_reduce<<<P.np, 256, 0, st>>>(P);
}
void launch_dem(const Params &P, cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_split, cudaEvent_t ev_free) {
    if (P.np <= 0 || P.n_sub <= 0) return;
    if (P.dem_mode == DEM_FP32) {
        launch_dem32(P, st);
    } else if (P.dem_mode == DEM_FP64_INTEGRATOR) {
        // every particle's free step on st2 beside the plan and the contact
        // groups on st; then the plan's inactive particles take theirs
        cudaEventRecord(ev_split, st);
        cudaStreamWaitEvent(st2, ev_split, 0);
        k_dem64_free<<<(P.np + 31) / 32, 128, 0, st2>>>(P);
        cudaEventRecord(ev_free, st2);
        k_dem64_plan<<<1, 256, 0, st>>>(P);
        launch_dem64c(P, st);
        cudaStreamWaitEvent(st, ev_free, 0);
        k_dem64_commit<<<(P.np + 127) / 128, 128, 0, st>>>(P);
    } else {
        k_dem<<<1, 256, 0, st>>>(P);
    }
}

}  // namespace lbmmb
