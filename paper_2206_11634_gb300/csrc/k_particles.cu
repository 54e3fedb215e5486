// Particle-side kernels, all FP64:
//   k_bin          world control points, search boxes, scatter into bricks;
//   k_force_reduce per-particle totals of the sweep's brick partials;
//   k_dem          n_sub DEM sub-steps (§2.3.4) with the hydrodynamic load
//                  frozen: metaball-metaball and metaball-wall contacts
//                  (§2.1.3-2.1.4), contact law (§2.1.1), velocity Verlet and
//                  Euler's equations in the body frame (Eq. (1)).
#include "k_flags.cuh"

namespace lbmmb {

// ---------------------------------------------------------------------------
// k_bin: one CTA per particle.  The search box AABB(x_i) -+ sqrt(sum K / c0)
// holds every node with M >= c0 (M >= c0 forces min |x - x_i|^2 <= sum K /
// c0); grown by one node it also holds every fluid node with a link into
// the particle.  The particle is appended to the list of each brick the grown
// box meets (k_flags sorts the lists).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bin(Params P) {
    const int j = blockIdx.x;
    DevParticle &p = P.parts[j];
    const int t = threadIdx.x;
    if (t < p.ncp) {
        double r[3];
        quat_rot(p.q, p.cpb[t], r);
        for (int a = 0; a < 3; a++) p.cpw[t][a] = p.x[a] + r[a];
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
    }
}

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
__device__ __forceinline__ double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
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
// start or the midpoint of the closest control-point pair; valid when
// c_tol < M < 1 for both; closest points by the first-order Taylor step of
// Eqs. (7)-(8); contact point in the middle of the overlap.
__device__ bool pair_geometry(const Params &P, const DevParticle &pi, const DevParticle &pj, bool warm,
                              double xm[3], double &delta, double nv[3], double xcp[3]) {
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
    for (int it = 0; it < 50; it++) {
        double M0, g0[3], H0[9], M1, g1[3], H1[9];
        mb_dd(P, pi, x, M0, g0, H0);
        mb_dd(P, pj, x, M1, g1, H1);
        double g[3], H[9], dx[3];
        for (int a = 0; a < 3; a++) g[a] = -(g0[a] + g1[a]);
        for (int a = 0; a < 9; a++) H[a] = H0[a] + H1[a];
        if (!solve_sym3(H, g, dx)) break;
        for (int a = 0; a < 3; a++) x[a] += dx[a];
        if (sqrt(dot3(dx, dx)) < 1e-12) break;
    }
    for (int a = 0; a < 3; a++) xm[a] = x[a];
    double M0, g0[3], H0[9], M1, g1[3], H1[9];
    mb_dd(P, pi, x, M0, g0, H0);
    mb_dd(P, pj, x, M1, g1, H1);
    if (!(M0 > P.c_tol && M0 < 1.0 && M1 > P.c_tol && M1 < 1.0)) return false;
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
__device__ bool wall_geometry(const Params &P, const DevParticle &p, int wall, bool warm, double xcw[3],
                              double &delta, double nv[3], double xcp[3]) {
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
        if (sqrt(d0 * d0 + d1 * d1) < 1e-12) break;
    }
    for (int a = 0; a < 3; a++) xcw[a] = x[a];
    double M, g[3], H[9];
    mb_dd(P, p, x, M, g, H);
    if (!(g[ax] * m_ax < 0.0)) return false;
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
        const bool warm = P.pair_on[idx] != 0;
        for (int a = 0; a < 3; a++) xm[a] = P.pair_xm[3 * idx + a];
        if (!pair_geometry(P, pi, pj, warm, xm, delta, nv, xcp)) {
            P.pair_on[idx] = 0;
            continue;
        }
        double xi[3];
        for (int a = 0; a < 3; a++) xi[a] = warm ? P.pair_xi[3 * idx + a] : 0.0;
        P.pair_on[idx] = 1;
        for (int a = 0; a < 3; a++) P.pair_xm[3 * idx + a] = xm[a];
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
            const bool warm = P.wall_on[wj] != 0;
            for (int a = 0; a < 3; a++) xcw[a] = P.wall_xcw[3 * wj + a];
            if (!wall_geometry(P, p, wall, warm, xcw, delta, nv, xcp)) { P.wall_on[wj] = 0; continue; }
            double xi[3];
            for (int a = 0; a < 3; a++) xi[a] = warm ? P.wall_xi[3 * wj + a] : 0.0;
            P.wall_on[wj] = 1;
            for (int a = 0; a < 3; a++) P.wall_xcw[3 * wj + a] = xcw[a];
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

__device__ void euler_rate(const DevParticle &p, const double wb[3], const double Tb[3], double out[3]) {
    double Iw[3], wIw[3], rhs[3];
    mv(p.I, wb, Iw);
    cross3(wb, Iw, wIw);
    for (int a = 0; a < 3; a++) rhs[a] = Tb[a] - wIw[a];
    mv(p.Iinv, rhs, out);
}

__device__ void quat_step(double q[4], const double wb[3], double h) {
    const double wn = sqrt(dot3(wb, wb));
    const double th = wn * h;
    double dq[4];
    if (th > 0.0) {
        const double sn = sin(0.5 * th) / wn;
        dq[0] = cos(0.5 * th); dq[1] = sn * wb[0]; dq[2] = sn * wb[1]; dq[3] = sn * wb[2];
    } else {
        dq[0] = 1.0; dq[1] = dq[2] = dq[3] = 0.0;
    }
    double r[4];
    r[0] = q[0] * dq[0] - q[1] * dq[1] - q[2] * dq[2] - q[3] * dq[3];
    r[1] = q[0] * dq[1] + q[1] * dq[0] + q[2] * dq[3] - q[3] * dq[2];
    r[2] = q[0] * dq[2] - q[1] * dq[3] + q[2] * dq[0] + q[3] * dq[1];
    r[3] = q[0] * dq[3] + q[1] * dq[2] - q[2] * dq[1] + q[3] * dq[0];
    const double nq = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    for (int a = 0; a < 4; a++) q[a] = r[a] / nq;
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

// One CTA; kick-drift-kick velocity Verlet, the rotation advanced with the
// half-step body angular velocity and closed by an implicit half-kick
// (ROT_ITERS fixed-point sweeps of Euler's equations).
__global__ void __launch_bounds__(256) k_dem(Params P) {
    const double h = 1.0 / P.n_sub;
    contacts(P, 0.0);
    for (int sub = 0; sub < P.n_sub; sub++) {
        for (int k = threadIdx.x; k < P.np; k += blockDim.x) {
            DevParticle &p = P.parts[k];
            if (p.fixed) continue;
            const double gr = 1.0 - P.rho0 / p.density;
            for (int a = 0; a < 3; a++) {
                const double Ft = p.mass * gr * P.g[a] + P.Fh[3 * k + a] + P.Fc[3 * k + a];
                p.v[a] += 0.5 * h * Ft / p.mass;
            }
            for (int a = 0; a < 3; a++) p.x[a] += h * p.v[a];
            double R[9], wb[3], Tw[3], Tb[3], dw[3];
            rotm(p.q, R);
            mtv(R, p.w, wb);
            for (int a = 0; a < 3; a++) Tw[a] = P.Th[3 * k + a] + P.Tc[3 * k + a];
            mtv(R, Tw, Tb);
            euler_rate(p, wb, Tb, dw);
            for (int a = 0; a < 3; a++) wb[a] += 0.5 * h * dw[a];
            quat_step(p.q, wb, h);
            rotm(p.q, R);
            mv(R, wb, p.w);
        }
        __syncthreads();
        refresh_cpw(P);
        contacts(P, h);
        for (int k = threadIdx.x; k < P.np; k += blockDim.x) {
            DevParticle &p = P.parts[k];
            if (p.fixed) continue;
            const double gr = 1.0 - P.rho0 / p.density;
            for (int a = 0; a < 3; a++) {
                const double Ft = p.mass * gr * P.g[a] + P.Fh[3 * k + a] + P.Fc[3 * k + a];
                p.v[a] += 0.5 * h * Ft / p.mass;
            }
            double R[9], wb[3], Tw[3], Tb[3], dw[3];
            rotm(p.q, R);
            mtv(R, p.w, wb);
            for (int a = 0; a < 3; a++) Tw[a] = P.Th[3 * k + a] + P.Tc[3 * k + a];
            mtv(R, Tw, Tb);
            double w1[3] = {wb[0], wb[1], wb[2]};
            for (int it = 0; it < ROT_ITERS; it++) {
                euler_rate(p, w1, Tb, dw);
                for (int a = 0; a < 3; a++) w1[a] = wb[a] + 0.5 * h * dw[a];
            }
            mv(R, w1, p.w);
        }
        __syncthreads();
    }
}

void launch_bin(const Params &P, cudaStream_t st) {
    if (P.np > 0) k_bin<<<P.np, 256, 0, st>>>(P);
}
void launch_force_reduce(const Params &P, cudaStream_t st) {
    if (P.np > 0) k_force_reduce<<<P.np, 256, 0, st>>>(P);
}
void launch_dem(const Params &P, cudaStream_t st) {
    if (P.np > 0 && P.n_sub > 0) k_dem<<<1, 256, 0, st>>>(P);
}

}  // namespace lbmmb
