// Boundary rules of the bounded (elliptic plate) domain, as affine maps of a boundary
// node's own post-collision populations (sm_103a, FP64, setup-time only).
//
// The paper realises its Dirichlet/Neumann conditions by boundary collisions that it
// does not spell out (Section 3.2 defers them to other work); the rules here are
// first-order, linear and local, with the wall halfway along each missing link:
//   Dirichlet (Eq. disp_Dirichlet):  f_S,k(x) =  f_C,kbar(x) + 2 f^eq_k(d_D),
//     f^eq = M^-1 N d (Eq. moments_eq) so 2 f^eq_k = w_k c_k . d_D with
//     w = 1 - theta on axis links and theta / 2 on diagonal links;
//   Neumann (Eq. disp_Neumann):      f_S,k(x) = -f_C,kbar(x) + 2 p_k,
//     p = M^-1 mbar_w, the even populations of the wall's bared moments, built from a
//     wall stress sigma_w whose traction sigma_w n is T and whose tangential part is
//     the node's own bared stress (Eq. stress_from_moments, recovered from its
//     post-collision moments as mbar = m^C (2 - omega) / (2 (1 - omega))), with
//     mbar_22 = -theta dx tr(sigma_w) / (4K) (pre-collision m22 streamed from
//     m12^C = theta d, m21^C = theta d_y).
// Each rule is evaluated on the unit vectors to give Q (8x8) and s (8) once per
// material; the sweep kernels then apply f_S,k = sum_j Q_kj f_C,j(x) + s_k.
#pragma once
#include "lbm_device.cuh"

namespace lbm {

struct BoundaryNode {
  uint8_t code[8];  // LBM_LINK_* per incoming direction
  double wd[2];     // Dirichlet displacement
  double T[2];      // traction
  double nrm[2];    // outward unit normal
};

struct Material {
  double w11, ws, wd, K;
};

__device__ inline void neumann_2p(const double (&fc)[8], double Tx, double Ty, double nx_,
                                  double ny_, const Material &m, double dx, double (&p2)[8]) {
  // post-collision even moments of the node
  const double mc11 = fc[4] - fc[5] + fc[6] - fc[7];
  const double mcs = fc[0] + fc[1] + fc[2] + fc[3] + 2.0 * (fc[4] + fc[5] + fc[6] + fc[7]);
  const double mcd = fc[0] - fc[1] + fc[2] - fc[3];
  const double b11 = mc11 * (2.0 - m.w11) / (2.0 * (1.0 - m.w11));
  const double bs = mcs * (2.0 - m.ws) / (2.0 * (1.0 - m.ws));
  const double bd = mcd * (2.0 - m.wd) / (2.0 * (1.0 - m.wd));
  const double s11 = -0.5 * (bs + bd) / dx, s22 = -0.5 * (bs - bd) / dx, s12 = -b11 / dx;
  const double rx = Tx - (s11 * nx_ + s12 * ny_);
  const double ry = Ty - (s12 * nx_ + s22 * ny_);
  const double rn = rx * nx_ + ry * ny_;
  const double w11 = s11 + 2.0 * rx * nx_ - rn * nx_ * nx_;
  const double w22 = s22 + 2.0 * ry * ny_ - rn * ny_ * ny_;
  const double w12 = s12 + rx * ny_ + ry * nx_ - rn * nx_ * ny_;
  const double m11 = -dx * w12, ms = -dx * (w11 + w22), md = -dx * (w11 - w22);
  const double m22 = kTheta * ms / (4.0 * m.K);
  // 2 p = 2 M^-1 (0, 0, m11, ms, md, 0, 0, m22)
  p2[0] = p2[2] = 0.5 * (ms + md) - m22;
  p2[1] = p2[3] = 0.5 * (ms - md) - m22;
  p2[4] = p2[6] = 0.5 * (m22 + m11);
  p2[5] = p2[7] = 0.5 * (m22 - m11);
}

__device__ inline double boundary_rule(const BoundaryNode &bn, int k, const double (&fc)[8],
                                       bool with_data, const Material &m, double dx) {
  const int cx[8] = {1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
  const int kb = (k < 4) ? ((k + 2) & 3) : (((k - 4 + 2) & 3) + 4);
  if (bn.code[k] == 1) {
    const double w = k < 4 ? (1.0 - kTheta) : 0.5 * kTheta;
    const double src = with_data ? w * (cx[k] * bn.wd[0] + cy[k] * bn.wd[1]) : 0.0;
    return fc[kb] + src;
  }
  double p2[8];
  neumann_2p(fc, with_data ? bn.T[0] : 0.0, with_data ? bn.T[1] : 0.0, bn.nrm[0], bn.nrm[1], m,
             dx, p2);
  return -fc[kb] + p2[k];
}

// One thread per boundary record: Q (row-major [k*8+j]) and s.
__global__ void k_boundary_setup(const BoundaryNode *__restrict__ nodes, long nb, Material m,
                                 double dx, double *__restrict__ Q, double *__restrict__ s) {
  const long b = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const BoundaryNode bn = nodes[b];
  double zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < 8; ++k) {
    if (bn.code[k] == 0) {
      s[b * 8 + k] = 0.0;
      for (int j = 0; j < 8; ++j) Q[b * 64 + k * 8 + j] = 0.0;
      continue;
    }
    s[b * 8 + k] = boundary_rule(bn, k, zero, true, m, dx);
    for (int j = 0; j < 8; ++j) {
      double e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      e[j] = 1.0;
      Q[b * 64 + k * 8 + j] = boundary_rule(bn, k, e, false, m, dx);
    }
  }
}

}  // namespace lbm
