// FP64 rigid-body helpers shared by the DEM kernels (§2.1.1, Eq. (1)):
// small vector algebra, Euler's equations in the principal frame, rotation of
// vectors by a unit quaternion and the quaternion update q <- q (x) exp(h w/2).
#pragma once
#include "lbm_internal.cuh"

namespace lbmmb {

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
// Euler's equations in the principal frame (Eq. (1), rotational part):
// dw_l/dt = T_l / I_l + (I_{l+1} - I_{l+2}) / I_l w_{l+1} w_{l+2}.
__device__ __forceinline__ void euler_rate(const DevParticle &p, const double wb[3], const double Tb[3], double out[3]) {
    out[0] = fma(p.cI[0] * wb[1], wb[2], p.iI[0] * Tb[0]);
    out[1] = fma(p.cI[1] * wb[2], wb[0], p.iI[1] * Tb[1]);
    out[2] = fma(p.cI[2] * wb[0], wb[1], p.iI[2] * Tb[2]);
}

// R(q) v and R(q)^T v for a unit quaternion (w, u): with c = u x v,
// R v = v + 2 w c + 2 u x c and R^T v = v - 2 w c + 2 u x c.
__device__ __forceinline__ void rot_world(const double q[4], const double v[3], double r[3]) {
    const double u[3] = {q[1], q[2], q[3]};
    double c[3], uc[3];
    cross3(u, v, c);
    cross3(u, c, uc);
    for (int a = 0; a < 3; a++) r[a] = v[a] + 2.0 * (q[0] * c[a] + uc[a]);
}
__device__ __forceinline__ void rot_body(const double q[4], const double v[3], double r[3]) {
    const double u[3] = {q[1], q[2], q[3]};
    double c[3], uc[3];
    cross3(u, v, c);
    cross3(u, c, uc);
    for (int a = 0; a < 3; a++) r[a] = v[a] + 2.0 * (uc[a] - q[0] * c[a]);
}

// q <- q (x) exp(h w_b / 2), the rotation by the body-frame angular velocity
// w_b over h.  For |w_b| h / 2 <= 1/16 the sine and cosine come from their
// Taylor series (truncation below 1e-19), which needs no square root.
__device__ __forceinline__ void quat_step(double q[4], const double wb[3], double h) {
    const double w2 = dot3(wb, wb);
    const double a2 = 0.25 * h * h * w2;  // (theta/2)^2
    double s, c;  // s = sin(theta/2) / |w_b|, c = cos(theta/2)
    if (a2 <= 1.0 / 256.0) {
        s = 0.5 * h * (1.0 + a2 * (-1.0 / 6.0 + a2 * (1.0 / 120.0 + a2 * (-1.0 / 5040.0 + a2 * (1.0 / 362880.0 + a2 * (-1.0 / 39916800.0))))));
        c = 1.0 + a2 * (-0.5 + a2 * (1.0 / 24.0 + a2 * (-1.0 / 720.0 + a2 * (1.0 / 40320.0 + a2 * (-1.0 / 3628800.0)))));
    } else {
        const double wn = sqrt(w2);
        double sn;
        sincos(0.5 * h * wn, &sn, &c);
        s = sn / wn;
    }
    const double d[4] = {c, s * wb[0], s * wb[1], s * wb[2]};
    const double r0 = q[0] * d[0] - q[1] * d[1] - q[2] * d[2] - q[3] * d[3];
    const double r1 = q[0] * d[1] + q[1] * d[0] + q[2] * d[3] - q[3] * d[2];
    const double r2 = q[0] * d[2] - q[1] * d[3] + q[2] * d[0] + q[3] * d[1];
    const double r3 = q[0] * d[3] + q[1] * d[2] - q[2] * d[1] + q[3] * d[0];
    q[0] = r0; q[1] = r1; q[2] = r2; q[3] = r3;
}

__device__ __forceinline__ void quat_normalize(double q[4]) {
    const double in = rsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; a++) q[a] *= in;
}

// Largest distance a free particle can move during one LBM step (its
// bounding sphere's centre): |v| + |a| with a the frozen acceleration of
// gravity and the hydrodynamic load (the unit step moves it by v + a/2),
// plus kDemReachMargin for the velocity contacts may add during the step;
// fixed particles do not move.  Evaluated in FP32 (rounded up by 1e-3
// relative) by both the planning and the contact kernel, so both see the
// same value.
constexpr float kDemReachMargin = 0.25f;
__device__ __forceinline__ float dem_reach(const Params &P, const DevParticle &p, int k) {
    if (p.fixed) return 0.f;
    float a2 = 0.f, v2 = 0.f;
    for (int a = 0; a < 3; a++) {
        const float acc = (float)(p.buoy * P.g[a] + P.Fh[3 * k + a] * p.inv_mass);
        a2 += acc * acc;
        v2 += (float)p.v[a] * (float)p.v[a];
    }
    return (sqrtf(v2) + sqrtf(a2)) * 1.001f + 1e-4f + kDemReachMargin;
}

}  // namespace lbmmb
