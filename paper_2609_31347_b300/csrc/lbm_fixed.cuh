// Integer-pipe variant of the collision and transposed collision (sm_103a).
//
// B300 executes FP64 at 2 lanes per SM (measured 1.86 DFMA/clk/SM) but 32-bit integer
// add/logic at ~128 lanes and 32x32->64 multiply-add at ~64 lanes per SM.  The sweep
// does ~37 FP64 operations per node, so on the FP64 pipe it is ALU-bound at ~1/3 of the
// HBM roofline.  This variant keeps every population in HBM as IEEE binary64 and does
// the node's arithmetic in 64-bit fixed point on the integer pipes:
//
//   unpack  all ten inputs of a node (8 populations + 2 force or adjoint-source values)
//           share the node's largest exponent E: x -> v = trunc(x 2^(1079-E)) by moving
//           the exponent field and one cvt.rzi.s64.f64, so |v| < 2^57 (the largest
//           input has 56-57 significant bits; smaller ones keep all bits down to
//           2^-57 of the node maximum);
//   compute the same pair-form maps as lbm_device.cuh with int64 adds, arithmetic
//           shifts for the powers of two, and a truncated 64x62-bit fixed-point
//           multiply (three mul.wide.s32) for the five non-power-of-two constants;
//           intermediates stay below 2^61;
//   pack    v -> |v| 2^(E-1079) rounded to nearest binary64 (clz, shift, exponent
//           assembly, round bit added with carry into the exponent field).
//
// Every result is within a few units of 2^-56 of the node's largest input of the exact
// value (binary64 rounding of the FP64-pipe variant is 2^-53 of each operand), far
// inside the 1e-11 parity bound.  The fixed-point path is taken only when the node's
// largest biased exponent E lies in [kEmin, kEmax] (largest input between 2^-923 and
// 2^57): then every shifted input keeps a positive exponent field, zeros and
// subnormals shift to values below 1 that truncate to 0, and every nonzero result has
// a normal exponent, so no per-value range test is needed.  A node whose ten inputs are
// all zero maps to zero (both maps are linear in their inputs), exactly; other nodes
// (extreme magnitudes, subnormal-only nodes, Inf, NaN) take the FP64-pipe path.
#pragma once
#include "lbm_device.cuh"

namespace lbm {

// (v c) with v < 2^61 in magnitude: v = vh 2^31 + vl, v C = vh hi 2^62 +
// (vh lo + vl hi) 2^31 + vl lo; the last term (< 2^62, i.e. < 1 unit after >> 62) is
// dropped.
__device__ __forceinline__ long long mulfix(long long v, FixC c) {
  const int vh = (int)(v >> 31);
  const int vl = (int)(v & 0x7fffffffll);
  long long t = (long long)vh * c.lo;
  t += (long long)vl * c.hi;
  return (long long)vh * c.hi + (t >> 31);
}

constexpr int kEmin = 100, kEmax = 1079;

__device__ __forceinline__ int exp_of(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// x 2^sh truncated toward zero, sh = 1079 - E >= 0 (E in [kEmin, kEmax]): adding sh to
// the exponent field is exact for normal x; a zero or subnormal x becomes a value below
// 2^(sh-1022) <= 2^-42 < 1, which truncates to 0.
__device__ __forceinline__ long long to_fix(double x, int sh20) {
  return __double2ll_rz(__hiloint2double(__double2hiint(x) + sh20, __double2loint(x)));
}

// The same value with integer operations only: x = M 2^(e - 1075) with M the 53-bit
// significand and e the biased exponent, so the result is M shifted left by
// e - E + 4 <= 4 places (right when negative, which truncates); zero and subnormal x
// (e = 0) give 0.  Which conversion a kernel uses is a balance of its FP64 and integer
// pipes: the plate kernels convert populations with to_fix and the force values this
// way (primal sweep 0.411 -> 0.406 ms when measured on the 4096^2 lattice); boundary
// nodes (BND) convert all ten inputs this way, since their rules already load the FP64
// pipe and a boundary warp is the critical path of a small plate's sweep (2-4 % per
// sweep at N_x = 64 .. 512); the periodic sweeps convert all inputs this way and give
// the FP64 pipe the output conversions instead (from_fix_cvt).
__device__ __forceinline__ long long to_fix_alu(double x, int E) {
  const long long b = __double_as_longlong(x);
  const int e = (int)(b >> 52) & 0x7ff;
  const long long M = (b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll;
  const int s = e - E + 4;
  long long v = s >= 0 ? (M << s) : (M >> min(-s, 63));
  v = e == 0 ? 0ll : v;
  return b < 0 ? -v : v;
}

// v 2^(E-1079) rounded to nearest (ties away from zero).  With E >= kEmin every
// nonzero |v| >= 1 gives a normal result (biased exponent E + 7 - lz >= 43).
__device__ __forceinline__ double from_fix(long long v, int E) {
  const unsigned long long s = (unsigned long long)(v >> 63);
  const unsigned long long a = ((unsigned long long)v ^ s) - s;
  const int lz = __clzll((long long)a);
  const unsigned long long m = a << (lz & 63);
  unsigned long long bits =
      ((unsigned long long)(unsigned)(E + 6 - lz) << 52) + (m >> 11) + ((m >> 10) & 1ull);
  bits |= s & 0x8000000000000000ull;
  return __longlong_as_double(a == 0 ? 0ll : (long long)bits);
}

// The same value through the hardware conversion: v converted to binary64 (round to
// nearest even; exact below 2^53) and scaled by 2^(E-1079) in the exponent field, which
// stays in the normal range for |v| >= 1 and E in [kEmin, kEmax].  Three instructions
// against ~20, at the price of one conversion on the FP64 pipe per value: the periodic
// sweeps, which also convert their inputs on the integer pipes (ALU_POP), take it
// (measured at 4096^2: primal 0.410 -> 0.395 ms, adjoint 0.396 -> 0.392 ms per sweep);
// the plate kernels, on which it measured slower, keep from_fix.  Ties round to even
// instead of away from zero; the bound of a half unit in the last place is the same.
__device__ __forceinline__ double from_fix_cvt(long long v, int E) {
  const double d = __ll2double_rn(v);
  const int hi = __double2hiint(d) + ((E - 1079) << 20);
  return v == 0 ? 0.0 : __hiloint2double(hi, __double2loint(d));
}

template <bool CVT>
__device__ __forceinline__ double fix_out(long long v, int E) {
  return CVT ? from_fix_cvt(v, E) : from_fix(v, E);
}

// A node whose ten inputs are all +0 or -0 maps to zero (the collision and its transpose
// are linear): writes zeros and returns true, else returns false.  Tried only on nodes
// that the fixed-point path declined, before the FP64-pipe path.
__device__ __forceinline__ bool zero_node(const double (&f)[8], double a, double b,
                                          double (&o)[8]) {
  int m = (__double2hiint(a) & 0x7fffffff) | __double2loint(a);
  m |= (__double2hiint(b) & 0x7fffffff) | __double2loint(b);
#pragma unroll
  for (int k = 0; k < 8; ++k) m |= (__double2hiint(f[k]) & 0x7fffffff) | __double2loint(f[k]);
  if (m != 0) return false;
#pragma unroll
  for (int k = 0; k < 8; ++k) o[k] = 0.0;
  return true;
}

// Largest biased exponent of the node's ten inputs: the exponent field is monotone in
// |x|, so take the max of the high words with the sign bit cleared, then extract once.
__device__ __forceinline__ int max_exp10(const double (&f)[8], double a, double b) {
  int m = __double2hiint(a) & 0x7fffffff;
  m = max(m, __double2hiint(b) & 0x7fffffff);
#pragma unroll
  for (int k = 0; k < 8; ++k) m = max(m, __double2hiint(f[k]) & 0x7fffffff);
  return m >> 20;
}

// Collision in fixed point (same map as collide<BND>; boundary rows use qs_b, P_b).
// Returns false when the node must take the FP64-pipe path (largest exponent outside
// [kEmin, kEmax]).  ALU_POP converts the eight populations on the integer pipes as well
// (the same values: both conversions truncate the same product); CVT rounds the outputs
// back with from_fix_cvt.
template <bool MON, bool BND = false, bool ALU_POP = BND, bool CVT = false>
__device__ __forceinline__ bool collide_fix(const double (&f)[8], double qx, double qy,
                                            const CoefFix &c, double (&o)[8], double &dx_,
                                            double &dy_) {
  const int E = max_exp10(f, qx, qy);
  if (E < kEmin || E > kEmax) return false;
  const int sh20 = (1079 - E) << 20;
  long long F[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) F[k] = ALU_POP ? to_fix_alu(f[k], E) : to_fix(f[k], sh20);
  const long long QX = to_fix_alu(qx, E), QY = to_fix_alu(qy, E);
  const long long a1 = F[0] + F[2], b1 = F[0] - F[2];
  const long long a2 = F[1] + F[3], b2 = F[1] - F[3];
  const long long a3 = F[4] + F[6], b3 = F[4] - F[6];
  const long long a4 = F[5] + F[7], b4 = F[5] - F[7];
  const long long mb10 = b1 + (b3 - b4) + 2 * QX;
  const long long mb01 = b2 + (b3 + b4) + 2 * QY;
  const long long m11 = a3 - a4;
  const long long ms = a1 + a2 + 2 * (a3 + a4);
  const long long md = a1 - a2;
  const long long es = mulfix(ms, BND ? c.qs_b : c.qs);
  const long long td = mulfix(md, c.qd);
  const long long e1 = es + td, e2 = es - td;
  const long long t10 = mulfix(mb10, c.third), t01 = mulfix(mb01, c.third);
  const long long o1 = t10 + QX, o2 = t01 + QY;
  const long long u = (t10 + t01) >> 2, v = (t01 - t10) >> 2;
  const long long q11 = mulfix(m11, c.q11);
  o[0] = fix_out<CVT>(e1 + o1, E);
  o[2] = fix_out<CVT>(e1 - o1, E);
  o[1] = fix_out<CVT>(e2 + o2, E);
  o[3] = fix_out<CVT>(e2 - o2, E);
  if (BND) {
    const long long P = mulfix(ms, c.P_b);  // m22^C / 4 = -gamma m_s^C / 4
    o[4] = fix_out<CVT>((P + q11) + u, E);
    o[6] = fix_out<CVT>((P + q11) - u, E);
    o[5] = fix_out<CVT>((P - q11) + v, E);
    o[7] = fix_out<CVT>((P - q11) - v, E);
  } else {
    o[4] = fix_out<CVT>(q11 + u, E);
    o[6] = fix_out<CVT>(q11 - u, E);
    o[5] = fix_out<CVT>(v - q11, E);
    o[7] = fix_out<CVT>(-q11 - v, E);
  }
  if (MON) {
    dx_ = fix_out<CVT>(mb10, E);
    dy_ = fix_out<CVT>(mb01, E);
  }
  return true;
}

// Transposed collision in fixed point (same map as collide_T<BND>).  ALU_SRC converts the
// two source values on the integer pipes (to_fix_alu) instead of the FP64 pipe: measured
// faster for the batched adjoint (2.59 -> 2.50 ms per sweep of 97 M nodes), slower for one
// 4096^2 lattice (0.388 -> 0.392 ms), so each kernel picks.
template <bool MON, bool BND = false, bool ALU_SRC = false, bool ALU_POP = BND, bool CVT = false>
__device__ __forceinline__ bool collide_T_fix(const double (&p)[8], double rx, double ry,
                                              const CoefFix &c, double (&o)[8], double &ax,
                                              double &ay) {
  const int E = max_exp10(p, rx, ry);
  if (E < kEmin || E > kEmax) return false;
  const int sh20 = (1079 - E) << 20;
  long long P[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) P[k] = ALU_POP ? to_fix_alu(p[k], E) : to_fix(p[k], sh20);
  const long long RX = (ALU_SRC || ALU_POP) ? to_fix_alu(rx, E) : to_fix(rx, sh20);
  const long long RY = (ALU_SRC || ALU_POP) ? to_fix_alu(ry, E) : to_fix(ry, sh20);
  const long long A1 = P[0] + P[2], B1 = P[0] - P[2];
  const long long A2 = P[1] + P[3], B2 = P[1] - P[3];
  const long long A3 = P[4] + P[6], B3 = P[4] - P[6];
  const long long A4 = P[5] + P[7], B4 = P[5] - P[7];
  const long long d34 = B3 - B4, s34 = B3 + B4;
  // (1/3) B1 + (1/12) d34 - rx = (1/3) (B1 + d34/4) - rx
  const long long n10 = mulfix(B1 + (d34 >> 2), c.third) - RX;
  const long long n01 = mulfix(B2 + (s34 >> 2), c.third) - RY;
  const long long n11 = mulfix(A3 - A4, c.q11);
  // d/dm_s of the outputs: cs (1/4 + gamma/2) on axis pairs, -gamma cs / 4 on diagonals
  const long long ns = BND ? mulfix(A1 + A2, c.qs_b) + mulfix(A3 + A4, c.P_b)
                           : mulfix(A1 + A2, c.qs);
  const long long nd = mulfix(A1 - A2, c.qd);
  const long long S1 = ns + nd, S2 = ns - nd;
  o[0] = fix_out<CVT>(S1 + n10, E);
  o[2] = fix_out<CVT>(S1 - n10, E);
  o[1] = fix_out<CVT>(S2 + n01, E);
  o[3] = fix_out<CVT>(S2 - n01, E);
  const long long T1 = 2 * ns + n11, T2 = 2 * ns - n11;
  const long long P1 = n10 + n01, P2 = n01 - n10;
  o[4] = fix_out<CVT>(T1 + P1, E);
  o[6] = fix_out<CVT>(T1 - P1, E);
  o[5] = fix_out<CVT>(T2 + P2, E);
  o[7] = fix_out<CVT>(T2 - P2, E);
  if (MON) {
    ax = fix_out<CVT>(B1 + d34, E);
    ay = fix_out<CVT>(B2 + s34, E);
  }
  return true;
}

// ---------------------------------------------------------------------------------
// Pair form of the bulk collisions: two adjacent lanes (h = lane & 1) share one node, so
// that a lattice too small to give every SM sub-partition a warp of its own still uses
// them, each lane running ~60 % of the single-lane instruction chain.  Lane h holds the
// populations k = h, h + 2, h + 4, h + 6 (in[0..3]) and the force (adjoint source)
// component h; it returns the outputs k = h, h + 2, h + 4, h + 6.  The integer operations
// are those of collide_fix / collide_T_fix with ALU_POP (exact integer sums in another
// grouping), so the results are bit-identical.  Every lane of the warp must take part
// (warp shuffles); both lanes of a pair return the same flag.

__device__ __forceinline__ long long xor1(long long v) {
  return __shfl_xor_sync(0xffffffffu, v, 1);
}

// largest biased exponent of the pair's ten inputs
__device__ __forceinline__ int pair_max_exp(const double (&in)[4], double q) {
  int m = __double2hiint(q) & 0x7fffffff;
#pragma unroll
  for (int i = 0; i < 4; ++i) m = max(m, __double2hiint(in[i]) & 0x7fffffff);
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
  return m >> 20;
}

template <bool MON, bool CVT>
__device__ __forceinline__ bool collide_fix_pair(const double (&in)[4], double q, int h,
                                                 const CoefFix &c, double (&out)[4],
                                                 double &m) {
  const int E = pair_max_exp(in, q);
  if (E < kEmin || E > kEmax) return false;
  long long F[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) F[i] = to_fix_alu(in[i], E);
  const long long Q = to_fix_alu(q, E);
  const long long a = F[0] + F[1], b = F[0] - F[1];    // h = 0: a1, b1;  h = 1: a2, b2
  const long long ad = F[2] + F[3], bd = F[2] - F[3];  // h = 0: a3, b3;  h = 1: a4, b4
  const long long a_o = xor1(a), ad_o = xor1(ad), bd_o = xor1(bd);
  const long long a1 = h ? a_o : a, a2 = h ? a : a_o;
  const long long a3 = h ? ad_o : ad, a4 = h ? ad : ad_o;
  const long long b3 = h ? bd_o : bd, b4 = h ? bd : bd_o;
  const long long mb = b + (h ? (b3 + b4) : (b3 - b4)) + 2 * Q;  // mb10 / mb01
  const long long ms = a1 + a2 + 2 * (a3 + a4);
  const long long es = mulfix(ms, c.qs), td = mulfix(a1 - a2, c.qd);
  const long long e = h ? es - td : es + td;                     // e1 / e2
  const long long t = mulfix(mb, c.third);                       // t10 / t01
  const long long t_o = xor1(t);
  const long long t10 = h ? t_o : t, t01 = h ? t : t_o;
  const long long oa = t + Q;                                    // o1 / o2
  const long long u = (t10 + t01) >> 2, v = (t01 - t10) >> 2;
  const long long q11 = mulfix(a3 - a4, c.q11);
  out[0] = fix_out<CVT>(e + oa, E);
  out[1] = fix_out<CVT>(e - oa, E);
  out[2] = fix_out<CVT>(h ? v - q11 : q11 + u, E);
  out[3] = fix_out<CVT>(h ? -q11 - v : q11 - u, E);
  if (MON) m = fix_out<CVT>(mb, E);                              // d_x / d_y
  return true;
}

template <bool MON, bool CVT>
__device__ __forceinline__ bool collide_T_fix_pair(const double (&in)[4], double r, int h,
                                                   const CoefFix &c, double (&out)[4],
                                                   double &m) {
  const int E = pair_max_exp(in, r);
  if (E < kEmin || E > kEmax) return false;
  long long P[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) P[i] = to_fix_alu(in[i], E);
  const long long R = to_fix_alu(r, E);
  const long long A = P[0] + P[1], B = P[0] - P[1];    // A1, B1 / A2, B2
  const long long Ad = P[2] + P[3], Bd = P[2] - P[3];  // A3, B3 / A4, B4
  const long long A_o = xor1(A), Ad_o = xor1(Ad), Bd_o = xor1(Bd);
  const long long A1 = h ? A_o : A, A2 = h ? A : A_o;
  const long long A3 = h ? Ad_o : Ad, A4 = h ? Ad : Ad_o;
  const long long B3 = h ? Bd_o : Bd, B4 = h ? Bd : Bd_o;
  const long long dd = h ? B3 + B4 : B3 - B4;                    // d34 / s34
  const long long n = mulfix(B + (dd >> 2), c.third) - R;        // n10 / n01
  const long long n_o = xor1(n);
  const long long n10 = h ? n_o : n, n01 = h ? n : n_o;
  const long long n11 = mulfix(A3 - A4, c.q11);
  const long long ns = mulfix(A1 + A2, c.qs), nd = mulfix(A1 - A2, c.qd);
  const long long S = h ? ns - nd : ns + nd;                     // S1 / S2
  const long long T = h ? 2 * ns - n11 : 2 * ns + n11;           // T1 / T2
  const long long Pp = h ? n01 - n10 : n10 + n01;                // P1 / P2
  out[0] = fix_out<CVT>(S + n, E);
  out[1] = fix_out<CVT>(S - n, E);
  out[2] = fix_out<CVT>(T + Pp, E);
  out[3] = fix_out<CVT>(T - Pp, E);
  if (MON) m = fix_out<CVT>(B + dd, E);                          // a_x / a_y
  return true;
}

}  // namespace lbm
