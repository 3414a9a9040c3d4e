// Device-side arithmetic of the solid LBM sweeps (sm_103a, FP64).
//
// Populations are indexed in the D2Q8 order Q of Eq. (direction_order):
//   0:(1,0) 1:(0,1) 2:(-1,0) 3:(0,-1) 4:(1,1) 5:(-1,1) 6:(-1,-1) 7:(1,-1).
// Opposite pairs (k, kbar) are (0,2), (1,3), (4,6), (5,7), so every map below works
// on the pair sums a_i and differences b_i of those pairs ("butterflies").
//
// Collision (Section 3.1, Eqs. moments .. moments_c_01, Table A.1 with
// tau_12 = tau_21 = tau_f = 1/2, i.e. omega = 1 for those three moments):
//   m10 = b1 + b3 - b4, m01 = b2 + b3 + b4, m11 = a3 - a4,
//   m_s = a1 + a2 + 2 (a3 + a4), m_d = a1 - a2,
//   mbar10 = m10 + g_x/2, mbar01 = m01 + g_y/2               (displacement d)
//   m^C: m10 + g_x, m01 + g_y, (1-w11) m11, (1-ws) m_s, (1-wd) m_d,
//        theta mbar10, theta mbar01, m_f^C = 0  => m22^C = -gamma m_s^C
// and f^C = M^-1 m^C with the inverse written out in pair form.  Only five
// pre-collision moments are needed because omega_12 = omega_21 = omega_f = 1.
//
// Adjoint collision (Eq. adjoint_collision): phi_C = A^T psi - j with A = dC/df_S
// and j_k = r . c_k, evaluated as M^T R^T M^-T psi in the same pair form.
#pragma once
#include <cstdint>

namespace lbm {

constexpr double kTheta = 1.0 / 3.0;

// Fixed-point constant C = round(c 2^62) = hi 2^31 + lo, 0 <= lo < 2^31, |c| < 1/2
// (used by the integer-pipe variant in lbm_fixed.cuh).
struct FixC {
  int hi, lo;
};

struct CoefFix {
  FixC qs, qd, q11, third;  // cs/4, cd/4, c11/4, 1/3
  FixC qs_b, P_b;           // boundary rows: cs (1/4 + gamma/2), -gamma cs / 4
  int bnd_ok;               // the boundary constants are below 1/2 in magnitude
};

// Per-material constants (host-computed, passed by value).
struct Coef {
  double c11, cs, cd;  // 1 - omega for m11, m_s, m_d
  double gam;          // gamma of Eq. (gamma) for boundary nodes (0 in the bulk)
  double dx;           // grid spacing
  double K;            // 2D bulk modulus (Eq. K)
  double w11, ws, wd;  // omega for m11, m_s, m_d
  // pre-scaled factors of the pair-form inverse (bulk and boundary rows)
  double q11, qs, qd;  // c11 / 4, cs / 4, cd / 4
  double qs_b, P_b;    // boundary: cs (1/4 + gamma/2) and -gamma cs / 4
  CoefFix fx;          // the bulk constants in fixed point
};

// Per-node material of the Young's-modulus field control: q planes hold c/4 for
// (m11, m_s, m_d) per node, gam the boundary gamma per boundary record.
struct Field {
  const double *q;      // 3N: c11/4, cs/4, cd/4
  const FixC *qfix;     // 3N: the same constants in fixed point (q11, qs, qd)
  const double *gam;    // nb
  const FixC *bfix;     // 2 nb: qs_b, P_b of each boundary record in fixed point
  const uint8_t *bok;   // nb: those are below 1/2 in magnitude
  const double *alpha;  // N: control, E_n = alpha_n^2
  double nu;
};

// c -> round(c 2^62) as hi 2^31 + lo, 0 <= lo < 2^31 (|c| < 1/2).
__device__ __forceinline__ FixC fixc_of(double c) {
  const long long C = __double2ll_rn(c * 4611686018427387904.0);
  const long long hi = C >> 31;
  return FixC{(int)hi, (int)(C - hi * 2147483648ll)};
}

// Fixed-point collision constants of a node: the handle's, or the node's own planes of a
// modulus field.
template <bool FIELD>
__device__ __forceinline__ CoefFix node_fix(const CoefFix &c, const Field &fl, long N, long n) {
  if (!FIELD) return c;
  CoefFix r = c;
  r.q11 = fl.qfix[n];
  r.qs = fl.qfix[N + n];
  r.qd = fl.qfix[2 * N + n];
  return r;
}

// The same for boundary record bi (its gamma-modified rows); false when the record's
// constants are too large for the fixed-point path.
template <bool FIELD>
__device__ __forceinline__ bool node_fix_bnd(const CoefFix &c, const Field &fl, long N, long n,
                                             long bi, CoefFix &r) {
  r = node_fix<FIELD>(c, fl, N, n);
  if (!FIELD) return c.bnd_ok != 0;
  if (!fl.bok[bi]) return false;
  r.qs_b = fl.bfix[2 * bi];
  r.P_b = fl.bfix[2 * bi + 1];
  return true;
}


// The node's collision constants: the handle's for a uniform material, or the per-node
// planes of a modulus field (boundary rows from the record's gamma).
template <bool FIELD>
__device__ __forceinline__ Coef node_coef(const Coef &c, const Field &fl, long N, long n,
                                          int bi) {
  if (!FIELD) return c;
  Coef r = c;
  r.q11 = fl.q[n];
  r.qs = fl.q[N + n];
  r.qd = fl.q[2 * N + n];
  r.c11 = 4.0 * r.q11;
  r.cs = 4.0 * r.qs;
  r.cd = 4.0 * r.qd;
  if (bi >= 0) {
    r.gam = fl.gam[bi];
    r.qs_b = r.cs * (0.25 + 0.5 * r.gam);
    r.P_b = -0.25 * r.gam * r.cs;
  }
  return r;
}

constexpr double kHalfOneMinusTheta = 0.5 * (1.0 - kTheta);
constexpr double kQuarterTheta = 0.25 * kTheta;

// Post-streaming populations -> post-collision populations; returns d = (d_x, d_y).
// q = (g_x, g_y) / 4: the lattice force is kept pre-scaled by 1/4 in memory, so that
// mbar10 = m10 + 2 q_x and the axis output o1 = (1-theta)/2 mbar10 + q_x are one FMA each.
template <bool BND>
__device__ __forceinline__ void collide(const double (&f)[8], double qx, double qy,
                                        const Coef &c, double (&o)[8], double &dx_,
                                        double &dy_) {
  const double a1 = f[0] + f[2], b1 = f[0] - f[2];
  const double a2 = f[1] + f[3], b2 = f[1] - f[3];
  const double a3 = f[4] + f[6], b3 = f[4] - f[6];
  const double a4 = f[5] + f[7], b4 = f[5] - f[7];
  const double m10 = b1 + (b3 - b4);
  const double m01 = b2 + (b3 + b4);
  const double m11 = a3 - a4;
  const double ms = fma(2.0, a3 + a4, a1 + a2);
  const double md = a1 - a2;
  const double mb10 = fma(2.0, qx, m10);  // Eq. moments_bar_1
  const double mb01 = fma(2.0, qy, m01);  // Eq. moments_bar_2
  dx_ = mb10;
  dy_ = mb01;
  const double es = (BND ? c.qs_b : c.qs) * ms;
  const double e1 = fma(c.qd, md, es);
  const double e2 = fma(-c.qd, md, es);
  const double o1 = fma(kHalfOneMinusTheta, mb10, qx);
  const double o2 = fma(kHalfOneMinusTheta, mb01, qy);
  const double u = kQuarterTheta * (mb10 + mb01);  // (m12^C + m21^C) / 4
  const double v = kQuarterTheta * (mb01 - mb10);  // (m21^C - m12^C) / 4
  const double q11 = c.q11 * m11;
  o[0] = e1 + o1;
  o[2] = e1 - o1;
  o[1] = e2 + o2;
  o[3] = e2 - o2;
  if (BND) {
    const double P = c.P_b * ms;  // m22^C / 4 = -gamma m_s^C / 4
    o[4] = (P + q11) + u;
    o[6] = (P + q11) - u;
    o[5] = (P - q11) + v;
    o[7] = (P - q11) - v;
  } else {
    o[4] = q11 + u;
    o[6] = q11 - u;
    o[5] = v - q11;
    o[7] = -q11 - v;
  }
}

// Transposed collision with the adjoint source: o = A^T psi - j, j_k = rx c_kx + ry c_ky.
// Also returns the adjoint displacement d^phi = (sum c_kx psi_k, sum c_ky psi_k).
template <bool BND>
__device__ __forceinline__ void collide_T(const double (&p)[8], double rx, double ry,
                                          const Coef &c, double (&o)[8], double &ax,
                                          double &ay) {
  const double A1 = p[0] + p[2], B1 = p[0] - p[2];
  const double A2 = p[1] + p[3], B2 = p[1] - p[3];
  const double A3 = p[4] + p[6], B3 = p[4] - p[6];
  const double A4 = p[5] + p[7], B4 = p[5] - p[7];
  const double d34 = B3 - B4, s34 = B3 + B4;
  ax = B1 + d34;
  ay = B2 + s34;
  const double n10 = fma(kHalfOneMinusTheta, B1, fma(kQuarterTheta, d34, -rx));
  const double n01 = fma(kHalfOneMinusTheta, B2, fma(kQuarterTheta, s34, -ry));
  const double n11 = c.q11 * (A3 - A4);
  const double A12 = A1 + A2;
  // d/dm_s of the outputs: cs (1/4 + gamma/2) on axis pairs, -gamma cs / 4 on diagonals
  const double ns = BND ? fma(c.qs_b, A12, c.P_b * (A3 + A4)) : c.qs * A12;
  const double nd = c.qd * (A1 - A2);
  const double S1 = ns + nd, S2 = ns - nd;
  o[0] = S1 + n10;
  o[2] = S1 - n10;
  o[1] = S2 + n01;
  o[3] = S2 - n01;
  const double T1 = fma(2.0, ns, n11), T2 = fma(2.0, ns, -n11);
  const double P1 = n10 + n01, P2 = n01 - n10;
  o[4] = T1 + P1;
  o[6] = T1 - P1;
  o[5] = T2 + P2;
  o[7] = T2 - P2;
}

// (dC/dg)^T psi for one node (the force enters m10^C with weight 1 and m12^C with
// theta/2 through mbar10; likewise for y).
__device__ __forceinline__ void force_sensitivity(const double (&p)[8], double &sx,
                                                  double &sy) {
  const double B1 = p[0] - p[2], B2 = p[1] - p[3];
  const double B3 = p[4] - p[6], B4 = p[5] - p[7];
  sx = (0.5 * (1.0 - 0.5 * kTheta)) * B1 + (0.125 * kTheta) * (B3 - B4);
  sy = (0.5 * (1.0 - 0.5 * kTheta)) * B2 + (0.125 * kTheta) * (B3 + B4);
}

// ---------------------------------------------------------------------------------
// Deterministic block reduction of NV values (warp shuffles, then one warp).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *smem /* >= 32*NV */) {
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  if (lane == 0)
    for (int i = 0; i < NV; ++i) smem[warp * NV + i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = lane < nwarps ? smem[lane * NV + i] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    }
  }
}

// max that propagates NaN (fmax drops it), so that a blown-up state reaches the monitor
__device__ __forceinline__ double nan_max(double a, double b) {
  return (a != a || b != b) ? a + b : fmax(a, b);
}

template <int NV>
__device__ __forceinline__ void block_max(double (&v)[NV], double *smem) {
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] = nan_max(v[i], __shfl_down_sync(0xffffffffu, v[i], o));
  if (lane == 0)
    for (int i = 0; i < NV; ++i) smem[warp * NV + i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = lane < nwarps ? smem[lane * NV + i] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v[i] = nan_max(v[i], __shfl_down_sync(0xffffffffu, v[i], o));
    }
  }
}

}  // namespace lbm
