// Tracking optimiser step (Sec. 3.3: the pose of the latest frame is
// optimised with Adam, learning rates lr_rot / lr_trans of the
// supplementary): one thread updates the Adam moments from the twist
// gradient, forms the step and retracts the pose by right-multiplication
// with the SE(3) exponential.  FP64 throughout; a single launch replaces the
// few dozen element-wise ops this takes in a tensor library.
#include "vt_common.cuh"

namespace vt {

// state: m[6], v[6], t.  lr: rho then phi.
__global__ void k_pose_adam(double *pose, double *d_twist, double *state, PoseAdamParams prm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double t = state[12] + 1.0;
    state[12] = t;
    const double c1 = 1.0 - pow(prm.beta1, t), c2 = 1.0 - pow(prm.beta2, t);
    double xi[6];
    for (int i = 0; i < 6; ++i) {
        const double g = d_twist[i];
        const double m = prm.beta1 * state[i] + (1.0 - prm.beta1) * g;
        const double v = prm.beta2 * state[6 + i] + (1.0 - prm.beta2) * g * g;
        state[i] = m;
        state[6 + i] = v;
        xi[i] = -prm.lr[i] * (m / c1) / (sqrt(v / c2) + prm.eps);
        d_twist[i] = 0.0;   // ready for the next backward's accumulation
    }
    // Exp of the twist (rho, phi): R = I + a K + b K^2, t = (I + b K + c K^2) rho
    const double *rho = xi, *phi = xi + 3;
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    double a, b, c;
    if (th2 < 1e-16) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        const double th = sqrt(th2), s = sin(th), co = cos(th);
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

}  // namespace vt
