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
// material (used by the tangent and gradient kernels), and in its compact form for the
// sweeps: a rule depends on the node's own post-collision populations only through the
// opposite population and the three relaxed moments (m11^C, m_s^C, m_d^C), so
//   f_S,k = sigma_k f_C,kbar(x) + r_k0 m11^C + r_k1 m_s^C + r_k2 m_d^C + s_k,
// sigma_k = +1 (Dirichlet) or -1 (Neumann), r_k = 0 for Dirichlet links.
#pragma once
#include "lbm_device.cuh"

namespace lbm {

struct BoundaryNode {
  uint8_t code[8];  // LBM_LINK_* per incoming direction
  double wd[2];     // Dirichlet displacement
  double T[2];      // traction
  double nrm[2];    // outward unit normal
};

// Forward-mode dual number: the setup kernel evaluates each rule with the modulus
// seeded (dE = 1) to get dQ/dE and ds/dE for the Young's-modulus gradient.
struct Dual {
  double v, d;
  __device__ Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
__device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}

// Material seen by the boundary rules: omega of m11, m_s, m_d and K, with their
// derivatives with respect to E (d = 0 when no derivative is wanted).
struct Material {
  double w11, ws, wd, K;
  double dw11, dws, dwd, dK;
};

// 2 p of the Neumann rule from the node's relaxed post-collision moments.
template <class T>
__device__ inline void neumann_2p_m(T mc11, T mcs, T mcd, T Tx, T Ty, double nx_, double ny_,
                                    const T (&w)[3], T K, double dx, T (&p2)[8]) {
  const T one(1.0), two(2.0), half(0.5);
  const T b11 = mc11 * (two - w[0]) / (two * (one - w[0]));
  const T bs = mcs * (two - w[1]) / (two * (one - w[1]));
  const T bd = mcd * (two - w[2]) / (two * (one - w[2]));
  const T idx(1.0 / dx), nX(nx_), nY(ny_);
  const T s11 = -(half * (bs + bd)) * idx, s22 = -(half * (bs - bd)) * idx, s12 = -b11 * idx;
  const T rx = Tx - (s11 * nX + s12 * nY);
  const T ry = Ty - (s12 * nX + s22 * nY);
  const T rn = rx * nX + ry * nY;
  const T w11 = s11 + two * rx * nX - rn * nX * nX;
  const T w22 = s22 + two * ry * nY - rn * nY * nY;
  const T w12 = s12 + rx * nY + ry * nX - rn * nX * nY;
  const T mdx(-dx);
  const T m11 = mdx * w12, ms = mdx * (w11 + w22), md = mdx * (w11 - w22);
  const T m22 = T(kTheta) * ms / (T(4.0) * K);
  // 2 p = 2 M^-1 (0, 0, m11, ms, md, 0, 0, m22)
  p2[0] = p2[2] = half * (ms + md) - m22;
  p2[1] = p2[3] = half * (ms - md) - m22;
  p2[4] = p2[6] = half * (m22 + m11);
  p2[5] = p2[7] = half * (m22 - m11);
}

template <class T>
__device__ inline void neumann_2p(const T (&fc)[8], T Tx, T Ty, double nx_, double ny_,
                                  const T (&w)[3], T K, double dx, T (&p2)[8]) {
  // post-collision even moments of the node
  const T mc11 = fc[4] - fc[5] + fc[6] - fc[7];
  const T mcs = fc[0] + fc[1] + fc[2] + fc[3] + T(2.0) * (fc[4] + fc[5] + fc[6] + fc[7]);
  const T mcd = fc[0] - fc[1] + fc[2] - fc[3];
  neumann_2p_m(mc11, mcs, mcd, Tx, Ty, nx_, ny_, w, K, dx, p2);
}

template <class T>
__device__ inline T boundary_rule(const BoundaryNode &bn, int k, const T (&fc)[8],
                                  bool with_data, const T (&w)[3], T K, double dx) {
  const int cx[8] = {1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
  const int kb = (k < 4) ? ((k + 2) & 3) : (((k - 4 + 2) & 3) + 4);
  if (bn.code[k] == 1) {
    const double wk = k < 4 ? (1.0 - kTheta) : 0.5 * kTheta;
    const double src = with_data ? wk * (cx[k] * bn.wd[0] + cy[k] * bn.wd[1]) : 0.0;
    return fc[kb] + T(src);
  }
  T p2[8];
  neumann_2p(fc, T(with_data ? bn.T[0] : 0.0), T(with_data ? bn.T[1] : 0.0), bn.nrm[0],
             bn.nrm[1], w, K, dx, p2);
  return -fc[kb] + p2[k];
}

// Material and its E-derivatives from a modulus (per-node field control).
__device__ inline Material material_of(double E, double nu) {
  const double mu = E / (2.0 * (1.0 + nu)), K = E / (2.0 * (1.0 - nu));
  const double t11 = mu / kTheta, ts = 2.0 * K / (1.0 + kTheta), td = 2.0 * mu / (1.0 - kTheta);
  const double dmu = 1.0 / (2.0 * (1.0 + nu)), dK = 1.0 / (2.0 * (1.0 - nu));
  Material m;
  m.w11 = 1.0 / (t11 + 0.5);
  m.ws = 1.0 / (ts + 0.5);
  m.wd = 1.0 / (td + 0.5);
  m.K = K;
  m.dw11 = -m.w11 * m.w11 * dmu / kTheta;
  m.dws = -m.ws * m.ws * 2.0 * dK / (1.0 + kTheta);
  m.dwd = -m.wd * m.wd * 2.0 * dmu / (1.0 - kTheta);
  m.dK = dK;
  return m;
}

// One thread per boundary record: Q (row-major [k*8+j]) and s, and their derivatives
// with respect to E (dQ, ds; skipped when dQ == nullptr; Q and s skipped when Q ==
// nullptr).  With a modulus field
// (alpha != nullptr) each record takes the material of its own node and also stores
// its boundary gamma (Eq. gamma with tau_f = 1/2).
// Compact form (R, dR: 4 doubles per link, SoA [(k*4 + i)*nb + b], i = 0..2 the
// moment coefficients, i = 3 the constant s_k; dR their E-derivatives, skipped when
// dR == nullptr).
static __global__ void k_boundary_setup(const BoundaryNode *__restrict__ nodes, long nb, Material m0,
                                 double dx, double *__restrict__ Q, double *__restrict__ s,
                                 double *__restrict__ dQ, double *__restrict__ ds,
                                 const double *__restrict__ alpha, const int *__restrict__ bnode,
                                 double nu, double *__restrict__ gam, double *__restrict__ R,
                                 double *__restrict__ dR, FixC *__restrict__ bfix,
                                 uint8_t *__restrict__ bok) {
  const long b = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const BoundaryNode bn = nodes[b];
  Material m = m0;
  if (alpha) {
    const double a = alpha[bnode[b]];
    m = material_of(a * a, nu);
    const double ts = 1.0 / m.ws - 0.5;
    const double gm = kTheta * 0.5 / ((1.0 + kTheta) * (ts - 0.5));
    gam[b] = gm;
    // the record's gamma-modified collision constants in fixed point, when below 1/2
    const double cs = 1.0 - m.ws;
    const double qs_b = cs * (0.25 + 0.5 * gm), P_b = -0.25 * gm * cs;
    const bool ok = fabs(qs_b) < 0.499 && fabs(P_b) < 0.499;
    bfix[2 * b] = ok ? fixc_of(qs_b) : FixC{0, 0};
    bfix[2 * b + 1] = ok ? fixc_of(P_b) : FixC{0, 0};
    bok[b] = ok ? 1 : 0;
  }
  const Dual w[3] = {Dual(m.w11, m.dw11), Dual(m.ws, m.dws), Dual(m.wd, m.dwd)};
  const Dual K(m.K, m.dK);
  for (int k = 0; k < 8; ++k) {
    // compact form: moment coefficients of 2 p_k (Neumann) and the constant
    Dual r[4];
    if (bn.code[k] == 2) {
      for (int i = 0; i < 3; ++i) {
        Dual p2[8];
        neumann_2p_m(Dual(i == 0 ? 1.0 : 0.0), Dual(i == 1 ? 1.0 : 0.0), Dual(i == 2 ? 1.0 : 0.0),
                     Dual(0.0), Dual(0.0), bn.nrm[0], bn.nrm[1], w, K, dx, p2);
        r[i] = p2[k];
      }
    }
    if (bn.code[k] != 0) {
      Dual zero[8];
      r[3] = boundary_rule(bn, k, zero, true, w, K, dx);
    }
    for (int i = 0; i < 4; ++i) {
      R[(long)(k * 4 + i) * nb + b] = r[i].v;
      if (dR) dR[(long)(k * 4 + i) * nb + b] = r[i].d;
    }
    if (!Q) continue;  // compact form only (batches of one geometry)
    if (bn.code[k] == 0) {
      s[b * 8 + k] = 0.0;
      if (dQ) ds[b * 8 + k] = 0.0;
      for (int j = 0; j < 8; ++j) {
        Q[b * 64 + k * 8 + j] = 0.0;
        if (dQ) dQ[b * 64 + k * 8 + j] = 0.0;
      }
      continue;
    }
    Dual zero[8];
    const Dual r0 = boundary_rule(bn, k, zero, true, w, K, dx);
    s[b * 8 + k] = r0.v;
    if (dQ) ds[b * 8 + k] = r0.d;
    for (int j = 0; j < 8; ++j) {
      Dual e[8];
      e[j] = Dual(1.0, 0.0);
      const Dual r = boundary_rule(bn, k, e, false, w, K, dx);
      Q[b * 64 + k * 8 + j] = r.v;
      if (dQ) dQ[b * 64 + k * 8 + j] = r.d;
    }
  }
}

}  // namespace lbm
