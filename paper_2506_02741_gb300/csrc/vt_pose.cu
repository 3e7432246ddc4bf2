// Optimiser steps of tracking and mapping.
//  - Tracking (Sec. 3.3: the pose of the latest frame is optimised with Adam,
//    learning rates lr_rot / lr_trans of the supplementary): one thread
//    updates the Adam moments from the twist gradient, forms the step and
//    retracts the pose by right-multiplication with the SE(3) exponential.
//    FP64 throughout; one launch replaces a few dozen tensor ops.
//  - Mapping (Sec. 3.4 learns colour, opacity and radius; supplementary
//    learning rates): one thread per Gaussian, Adam on (c, logit o, log r)
//    in FP32, storage written back in the section's precision.
#include "vt_common.cuh"

namespace vt {

// One warp: lanes 0..5 update the moments of one twist component each, lane
// 0 then forms the exponential and the retraction.  state: m[6], v[6], t,
// b1^t, b2^t (running products instead of pow, which is slow in FP64).
// lr: rho then phi.
__global__ void k_pose_adam(double *pose, double *d_twist, double *state, PoseAdamParams prm) {
    const int lane = threadIdx.x;
    const double t_old = state[12];
    const double p1 = (t_old == 0.0 ? 1.0 : state[13]) * prm.beta1;   // b1^t
    const double p2 = (t_old == 0.0 ? 1.0 : state[14]) * prm.beta2;   // b2^t
    double x = 0.0;
    if (lane < 6) {
        const double g = d_twist[lane];
        const double m = prm.beta1 * state[lane] + (1.0 - prm.beta1) * g;
        const double v = prm.beta2 * state[6 + lane] + (1.0 - prm.beta2) * g * g;
        state[lane] = m;
        state[6 + lane] = v;
        x = -prm.lr[lane] * (m / (1.0 - p1)) / (sqrt(v / (1.0 - p2)) + prm.eps);
        d_twist[lane] = 0.0;   // ready for the next backward's accumulation
    }
    double xi[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) xi[k] = __shfl_sync(0xffffffffu, x, k);
    if (lane != 0) return;
    state[12] = t_old + 1.0;
    state[13] = p1;
    state[14] = p2;
    // Exp of the twist (rho, phi): R = I + a K + b K^2, t = (I + b K + c K^2) rho
    const double *rho = xi, *phi = xi + 3;
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    double a, b, c;
    if (th2 < 1e-16) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        const double th = sqrt(th2);
        double s, co;
        sincos(th, &s, &co);
        a = s / th;
        b = (1.0 - co) / th2;
        c = (th - s) / (th2 * th);
    }
    const double K[9] = {0.0, -phi[2], phi[1], phi[2], 0.0, -phi[0], -phi[1], phi[0], 0.0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
    double Rd[9], J[9];
    for (int k = 0; k < 9; ++k) {
        const double e = (k % 4 == 0) ? 1.0 : 0.0;
        Rd[k] = e + a * K[k] + b * K2[k];
        J[k] = e + b * K[k] + c * K2[k];
    }
    double td[3];
    for (int i = 0; i < 3; ++i) td[i] = J[3 * i] * rho[0] + J[3 * i + 1] * rho[1] + J[3 * i + 2] * rho[2];
    // P <- P [Rd | td]
    double Rn[9], tn[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            Rn[3 * i + j] = pose[3 * i] * Rd[j] + pose[3 * i + 1] * Rd[3 + j] + pose[3 * i + 2] * Rd[6 + j];
        tn[i] = pose[3 * i] * td[0] + pose[3 * i + 1] * td[1] + pose[3 * i + 2] * td[2] + pose[9 + i];
    }
    for (int k = 0; k < 9; ++k) pose[k] = Rn[k];
    for (int i = 0; i < 3; ++i) pose[9 + i] = tn[i];
}

// Step counter of the attribute optimiser: step[0] = t (incremented),
// step[1] = 1 / (1 - b1^t), step[2] = 1 / sqrt(1 - b2^t).
__global__ void k_adam_step_count(double *step, double beta1, double beta2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double t = step[0] + 1.0;
    step[0] = t;
    step[1] = 1.0 / (1.0 - pow(beta1, t));
    step[2] = 1.0 / sqrt(1.0 - pow(beta2, t));
}

__device__ __forceinline__ void st_any(void *p, int prec, int64_t i, float x) {
    if (prec == VT_F16)
        static_cast<__half *>(p)[i] = __float2half_rn(x);
    else
        static_cast<float *>(p)[i] = x;
}

// One thread per Gaussian: chain rule to (c, logit o, log r), Adam on the
// five FP32 parameters (planes of theta / m / v), activated values written to
// the section's storage, gradients zeroed.  HBM-bound (~180 B per Gaussian):
// every input is loaded before the first store so that the loads overlap.
__global__ void __launch_bounds__(256) k_attr_adam(int64_t n, float *__restrict__ theta,
                                                   float *__restrict__ m, float *__restrict__ v,
                                                   const double *__restrict__ step,
                                                   float *__restrict__ d_colour,
                                                   float *__restrict__ d_opacity,
                                                   float *__restrict__ d_radius, int prec,
                                                   void *__restrict__ colour,
                                                   void *__restrict__ opacity,
                                                   void *__restrict__ radius, AttrAdamParams prm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float th[5], g[5], mk[5], vk[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        th[k] = theta[k * n + i];
        mk[k] = m[k * n + i];
        vk[k] = v[k * n + i];
    }
    g[0] = d_colour[3 * i];
    g[1] = d_colour[3 * i + 1];
    g[2] = d_colour[3 * i + 2];
    g[3] = d_opacity[i];
    g[4] = d_radius[i];
    const float s1 = (float)step[1], s2 = (float)step[2];
    const float o = 1.f / (1.f + expf(-th[3]));
    g[3] *= o * (1.f - o);
    g[4] *= expf(th[4]);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        mk[k] = prm.beta1 * mk[k] + (1.f - prm.beta1) * g[k];
        vk[k] = prm.beta2 * vk[k] + (1.f - prm.beta2) * g[k] * g[k];
        th[k] -= prm.lr[k] * s1 * mk[k] / (sqrtf(vk[k]) * s2 + prm.eps);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        theta[k * n + i] = th[k];
        m[k * n + i] = mk[k];
        v[k * n + i] = vk[k];
    }
    d_colour[3 * i] = 0.f;
    d_colour[3 * i + 1] = 0.f;
    d_colour[3 * i + 2] = 0.f;
    d_opacity[i] = 0.f;
    d_radius[i] = 0.f;
    st_any(colour, prec, 3 * i, th[0]);
    st_any(colour, prec, 3 * i + 1, th[1]);
    st_any(colour, prec, 3 * i + 2, th[2]);
    st_any(opacity, prec, i, 1.f / (1.f + expf(-th[3])));
    st_any(radius, prec, i, expf(th[4]));
}

// Ellipsoid shape (anisotropic variant), one thread per Gaussian: Adam on
// (log s0..2, q0..3) with the chain rule dL/dlog s = dL/ds s; the scale
// exp(log s) and the quaternion as stored are written back in the
// section's precision and the gradients zeroed.  Loads first, as above.
__global__ void __launch_bounds__(256) k_shape_adam(int64_t n, float *__restrict__ theta,
                                                    float *__restrict__ m, float *__restrict__ v,
                                                    const double *__restrict__ step,
                                                    float *__restrict__ d_scale,
                                                    float *__restrict__ d_rot, int prec,
                                                    void *__restrict__ scale,
                                                    void *__restrict__ rot, ShapeAdamParams prm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float th[7], g[7], mk[7], vk[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        th[k] = theta[k * n + i];
        mk[k] = m[k * n + i];
        vk[k] = v[k * n + i];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = d_scale[3 * i + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) g[3 + k] = d_rot[4 * i + k];
    const float s1 = (float)step[1], s2 = (float)step[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] *= expf(th[k]);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const float lr = k < 3 ? prm.lr_scale : prm.lr_rot;
        mk[k] = prm.beta1 * mk[k] + (1.f - prm.beta1) * g[k];
        vk[k] = prm.beta2 * vk[k] + (1.f - prm.beta2) * g[k] * g[k];
        th[k] -= lr * s1 * mk[k] / (sqrtf(vk[k]) * s2 + prm.eps);
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        theta[k * n + i] = th[k];
        m[k * n + i] = mk[k];
        v[k * n + i] = vk[k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d_scale[3 * i + k] = 0.f;
        st_any(scale, prec, 3 * i + k, expf(th[k]));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        d_rot[4 * i + k] = 0.f;
        st_any(rot, prec, 4 * i + k, th[3 + k]);
    }
}

// Optimiser state of the mapping step from the section's storage, one
// thread per Gaussian: theta = (c0, c1, c2, logit o, log r) with o clamped
// to [1e-4, 1 - 1e-4] (so that the logit is finite), moments zero.  With
// scale != NULL the ellipsoid shape state instead: theta = (log s0, log s1,
// log s2, q0, q1, q2, q3).
__global__ void __launch_bounds__(256) k_adam_init(int64_t n, int prec, const void *colour,
                                                   const void *opacity, const void *radius,
                                                   const void *scale, const void *rot,
                                                   float *theta, float *m, float *v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int planes = scale ? 7 : 5;
    float th[7];
    if (scale) {
        for (int k = 0; k < 3; ++k) th[k] = logf(ld_attr(scale, prec, 3 * i + k));
        for (int k = 0; k < 4; ++k) th[3 + k] = ld_attr(rot, prec, 4 * i + k);
    } else {
        for (int k = 0; k < 3; ++k) th[k] = ld_attr(colour, prec, 3 * i + k);
        const float o = fminf(fmaxf(ld_attr(opacity, prec, i), 1e-4f), 1.f - 1e-4f);
        th[3] = logf(o / (1.f - o));
        th[4] = logf(ld_attr(radius, prec, i));
    }
    for (int k = 0; k < planes; ++k) {
        theta[k * n + i] = th[k];
        m[k * n + i] = 0.f;
        v[k * n + i] = 0.f;
    }
}

}  // namespace vt
