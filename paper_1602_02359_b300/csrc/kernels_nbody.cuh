// Planetary integrator (Sec. 3.7, orbital integrator for planets): one
// fixed step of the fifth-order Cash-Karp Runge-Kutta method (Tab. rk) for
// N point masses orbiting the central star, in the star's frame, FP64.
//
//   d2r_i/dt2 = -(M + m_i) r_i/|r_i|^3
//               + sum_{j != i} m_j [(r_j - r_i)/|r_j - r_i|^3 - r_j/|r_j|^3]
// (G = 1; the bracket's second term and the m_i beside M are the indirect
// acceleration of the star's frame, dropped when `indirect` is 0).  Before
// the stages the gas force kicks the velocities: v_i += h (kick_i - kick_*),
// kick_* the gas acceleration of the star (the frame's share), when given.
//
// One warp; lane i holds planet i's state and its six stage derivatives in
// registers, and the stage positions meet in shared memory.  The planetary
// system is a few dozen numbers: the kernel exists so that the force, the
// kick and the drift stay on the device, queued behind the hydrodynamical
// step, with no synchronisation with the host.
#pragma once
#include "fargo_internal.cuh"

namespace fk {

constexpr int kNbMax = 32;   // planets per call (one lane each)

struct NbArgs {
    double *y;                 // [n][6]: x, y, z, vx, vy, vz; updated in place
    const double *mass;        // [n]
    const double *kick;        // [n][kick_stride] gas accelerations (first 3 used), or null
    const double *kick_star;   // [3] the star's gas acceleration, subtracted from each kick, or null
    const double *h_dev;       // the step length on the device, or null (then h)
    double mstar, h;
    int n, kick_stride, indirect;
};

// Tab. rk: nodes (c_i are implied by the rows of a), stage matrix, weights.
__device__ __forceinline__ double ck_a(int s, int j)
{
    switch (s * 8 + j) {
    case 8: return 1.0 / 5.0;
    case 16: return 3.0 / 40.0;
    case 17: return 9.0 / 40.0;
    case 24: return 3.0 / 10.0;
    case 25: return -9.0 / 10.0;
    case 26: return 6.0 / 5.0;
    case 32: return -11.0 / 54.0;
    case 33: return 5.0 / 2.0;
    case 34: return -70.0 / 27.0;
    case 35: return 35.0 / 27.0;
    case 40: return 1631.0 / 55296.0;
    case 41: return 175.0 / 512.0;
    case 42: return 575.0 / 13824.0;
    case 43: return 44275.0 / 110592.0;
    case 44: return 253.0 / 4096.0;
    default: return 0.0;
    }
}
__device__ __forceinline__ double ck_b(int s)
{
    switch (s) {
    case 0: return 37.0 / 378.0;
    case 2: return 250.0 / 621.0;
    case 3: return 125.0 / 594.0;
    case 5: return 512.0 / 1771.0;
    default: return 0.0;
    }
}

__device__ __forceinline__ double norm3(double x, double y, double z) { return sqrt(x * x + y * y + z * z); }

static __global__ void __launch_bounds__(32) k_nbody_rk5(NbArgs a)
{
    __shared__ double sp[kNbMax][3];
    const int i = threadIdx.x;
    const bool on = i < a.n;
    const double h = a.h_dev ? *a.h_dev : a.h;
    double y0[6] = {0, 0, 0, 0, 0, 0}, k[6][6];
    if (on) {
#pragma unroll
        for (int q = 0; q < 6; q++) y0[q] = a.y[6 * i + q];
        if (a.kick) {
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const double g = a.kick[(size_t)a.kick_stride * i + q] - (a.kick_star ? a.kick_star[q] : 0.0);
                y0[3 + q] += h * g;
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 6; s++) {
        double ys[6];
#pragma unroll
        for (int q = 0; q < 6; q++) {
            double v = y0[q];
#pragma unroll
            for (int j = 0; j < s; j++) v += (h * ck_a(s, j)) * k[j][q];
            ys[q] = v;
        }
        if (on) {
            sp[i][0] = ys[0];
            sp[i][1] = ys[1];
            sp[i][2] = ys[2];
        }
        __syncwarp();
        double ax = 0.0, ay = 0.0, az = 0.0;
        if (on) {
            const double d = norm3(ys[0], ys[1], ys[2]);
            const double gm = a.mstar + (a.indirect ? a.mass[i] : 0.0);
            const double f = gm / (d * d * d);
            ax = -f * ys[0];
            ay = -f * ys[1];
            az = -f * ys[2];
            for (int j = 0; j < a.n; j++) {
                if (j == i) continue;
                const double mj = a.mass[j];
                const double dx = sp[j][0] - ys[0], dy = sp[j][1] - ys[1], dz = sp[j][2] - ys[2];
                const double dij = norm3(dx, dy, dz);
                const double fij = mj / (dij * dij * dij);
                ax += fij * dx;
                ay += fij * dy;
                az += fij * dz;
                if (a.indirect) {
                    const double dj = norm3(sp[j][0], sp[j][1], sp[j][2]);
                    const double fj = mj / (dj * dj * dj);
                    ax -= fj * sp[j][0];
                    ay -= fj * sp[j][1];
                    az -= fj * sp[j][2];
                }
            }
        }
        k[s][0] = ys[3];
        k[s][1] = ys[4];
        k[s][2] = ys[5];
        k[s][3] = ax;
        k[s][4] = ay;
        k[s][5] = az;
        __syncwarp();   // the next stage overwrites sp
    }
    if (on) {
#pragma unroll
        for (int q = 0; q < 6; q++) {
            double v = y0[q];
#pragma unroll
            for (int s = 0; s < 6; s++) v += (h * ck_b(s)) * k[s][q];
            a.y[6 * i + q] = v;
        }
    }
}

}  // namespace fk
