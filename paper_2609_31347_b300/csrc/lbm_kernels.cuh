// Sweep, objective, gradient and reduction kernels of the solid LBM (sm_103a, FP64).
//
// Memory layout in HBM: SoA planes of N = nx*ny doubles, population k of node
// n = y*nx + x at [k*N + n] (x fastest), so a warp's 32 consecutive x of one plane
// are one coalesced 256-byte access; the pull of Eq. (local_stream) only shifts that
// window by one element in x and one row in y.
//
// Bounded grids add a uint8 node type (0 outside, 1 interior, 2 boundary) and, for
// boundary nodes only, a compact record: the incoming population of a missing link k
// is the affine map  f_S,k = sum_j Q_kj f_C,j(x) + s_k  of the node's own
// post-collision populations (bounce-back for Dirichlet, anti-bounce-back with the
// wall stress for Neumann), and a bit mask of the regular links.
#pragma once
#include "lbm_device.cuh"
#include "lbm_fixed.cuh"

namespace lbm {

// Pull sources of direction k: x - c_k.
__constant__ int kCX[8] = {1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCY[8] = {0, 1, 0, -1, 1, 1, -1, -1};

struct Grid {
  int nx, ny;
  long N;  // nodes (plane stride)
};

struct Bounded {
  const uint8_t *type;    // N
  const int *bidx;        // N: boundary record index (valid where type == 2)
  const double *Q;        // nb * 64, row-major Q[k*8+j]
  const double *s;        // nb * 8
  const uint8_t *regmask; // nb: bit k set <=> link k (incoming) is regular
  const double *dQ;       // nb * 64: dQ/dE (Young's-modulus controls only)
  const double *ds;       // nb * 8:  ds/dE
};

// Derivatives of the collision constants with respect to E (c = 1 - omega).
struct YoungDeriv {
  double dc11, dcs, dcd, dgam;
};

// Population loads.  NC = true: through the read-only (non-coherent) path, for kernels
// that never write what they read; NC = false: coherent loads, for the cluster-resident
// kernel, which rewrites its lattice between sweeps within one launch.
template <bool NC>
__device__ __forceinline__ double ldp(const double *p) {
  if (NC) return __ldg(p);
  return *p;
}

// Neighbour index with periodic wrap.
__device__ __forceinline__ long wrap_idx(int x, int y, int dx_, int dy_, const Grid &g) {
  int xs = x + dx_, ys = y + dy_;
  xs = xs < 0 ? xs + g.nx : (xs >= g.nx ? xs - g.nx : xs);
  ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
  return (long)ys * g.nx + xs;
}

// Post-streaming populations at (x, y): f_S,k(x) = f_C,k(x - c_k) (Eq. local_stream),
// with the boundary rules at boundary nodes.  Returns false for outside nodes.
template <bool BOUNDED, bool NC = true>
__device__ __forceinline__ bool pull_primal(const double *__restrict__ fin, int x, int y,
                                            const Grid &g, const Bounded &b, double (&f)[8],
                                            double &gam_sel) {
  const long n = (long)y * g.nx + x;
  gam_sel = 0.0;
  if (!BOUNDED) {
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const long rm = (long)(y == 0 ? g.ny - 1 : y - 1) * g.nx;
    const long rp = (long)(y == g.ny - 1 ? 0 : y + 1) * g.nx;
    const long r0 = (long)y * g.nx;
    f[0] = ldp<NC>(fin + 0 * g.N + r0 + xm);
    f[1] = ldp<NC>(fin + 1 * g.N + rm + x);
    f[2] = ldp<NC>(fin + 2 * g.N + r0 + xp);
    f[3] = ldp<NC>(fin + 3 * g.N + rp + x);
    f[4] = ldp<NC>(fin + 4 * g.N + rm + xm);
    f[5] = ldp<NC>(fin + 5 * g.N + rm + xp);
    f[6] = ldp<NC>(fin + 6 * g.N + rp + xp);
    f[7] = ldp<NC>(fin + 7 * g.N + rp + xm);
    return true;
  } else {
    const uint8_t t = b.type[n];
    if (t == 0) return false;
    if (t == 1) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        f[k] = ldp<NC>(fin + k * g.N + n - kCX[k] - (long)kCY[k] * g.nx);
      return true;
    }
    const int bi = b.bidx[n];
    const unsigned reg = b.regmask[bi];
    double own[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) own[j] = ldp<NC>(fin + j * g.N + n);
    const double *Q = b.Q + (long)bi * 64;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (reg & (1u << k)) {
        f[k] = ldp<NC>(fin + k * g.N + n - kCX[k] - (long)kCY[k] * g.nx);
      } else {
        double acc = b.s[(long)bi * 8 + k];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc += Q[k * 8 + j] * own[j];
        f[k] = acc;
      }
    }
    gam_sel = 1.0;
    return true;
  }
}

// Adjoint streaming phi_S = S'^T phi_C at (x, y): phi_S,j(x) = phi_C,j(x + c_j) where
// that node pulls from x, plus Q^T phi_C(x) at boundary nodes.
template <bool BOUNDED, bool NC = true>
__device__ __forceinline__ bool pull_adjoint(const double *__restrict__ pin, int x, int y,
                                             const Grid &g, const Bounded &b, double (&p)[8],
                                             double &gam_sel) {
  const long n = (long)y * g.nx + x;
  gam_sel = 0.0;
  if (!BOUNDED) {
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const long rm = (long)(y == 0 ? g.ny - 1 : y - 1) * g.nx;
    const long rp = (long)(y == g.ny - 1 ? 0 : y + 1) * g.nx;
    const long r0 = (long)y * g.nx;
    p[0] = ldp<NC>(pin + 0 * g.N + r0 + xp);
    p[1] = ldp<NC>(pin + 1 * g.N + rp + x);
    p[2] = ldp<NC>(pin + 2 * g.N + r0 + xm);
    p[3] = ldp<NC>(pin + 3 * g.N + rm + x);
    p[4] = ldp<NC>(pin + 4 * g.N + rp + xp);
    p[5] = ldp<NC>(pin + 5 * g.N + rp + xm);
    p[6] = ldp<NC>(pin + 6 * g.N + rm + xm);
    p[7] = ldp<NC>(pin + 7 * g.N + rm + xp);
    return true;
  } else {
    const uint8_t t = b.type[n];
    if (t == 0) return false;
    if (t == 1) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        p[k] = ldp<NC>(pin + k * g.N + n + kCX[k] + (long)kCY[k] * g.nx);
      return true;
    }
    const int bi = b.bidx[n];
    const unsigned reg = b.regmask[bi];
    double own[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) own[k] = ldp<NC>(pin + k * g.N + n);
    const double *Q = b.Q + (long)bi * 64;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      // downstream node x + c_j pulls f_C,j(x) iff its link j is regular, i.e. iff the
      // opposite link jbar at x is regular (its source x - c_jbar = x + c_j is active)
      const int jb = (j < 4) ? ((j + 2) & 3) : (((j - 4 + 2) & 3) + 4);
      double acc = (reg & (1u << jb)) ? ldp<NC>(pin + j * g.N + n + kCX[j] + (long)kCY[j] * g.nx)
                                      : 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) acc += Q[k * 8 + j] * own[k];  // rows of regular links are 0
      p[j] = acc;
    }
    gam_sel = 1.0;
    return true;
  }
}

// One primal sweep: f_C(t) = C[S' f_C(t-1), g]; optional monitor partial sum of |d|^2.
// ARITH 0: every operation on the FP64 pipe; ARITH 1: bulk nodes in 64-bit fixed point
// on the integer pipes (lbm_fixed.cuh), boundary nodes on the FP64 pipe.
template <bool BOUNDED, bool MONITOR, int ARITH, bool FIELD>
__global__ void __launch_bounds__(256) k_primal(const double *__restrict__ fin,
                                                double *__restrict__ fout,
                                                const double *__restrict__ g2, Grid g,
                                                Bounded b, Coef c0, Field fl,
                                                double *__restrict__ partial) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  double mon[1] = {0.0};
  if (x < g.nx && y < g.ny) {
    const long n = (long)y * g.nx + x;
    double f[8], gsel;
    if (pull_primal<BOUNDED>(fin, x, y, g, b, f, gsel)) {
      double o[8], dxn = 0.0, dyn = 0.0;
      const double qx = __ldg(g2 + n), qy = __ldg(g2 + g.N + n);
      const Coef c = node_coef<FIELD>(c0, fl, g.N, n,
                                      (BOUNDED && FIELD && gsel != 0.0) ? b.bidx[n] : -1);
      if (BOUNDED && gsel != 0.0)
        collide<true>(f, qx, qy, c, o, dxn, dyn);
      else if (ARITH == 0 ||
               !collide_fix<MONITOR, false, !BOUNDED, !BOUNDED>(f, qx, qy, node_fix<FIELD>(c0.fx, fl, g.N, n), o, dxn, dyn))
        collide<false>(f, qx, qy, c, o, dxn, dyn);
#pragma unroll
      for (int k = 0; k < 8; ++k) fout[k * g.N + n] = o[k];
      if (MONITOR) mon[0] = dxn * dxn + dyn * dyn;
    }
  }
  if (MONITOR) {
    __shared__ double sm[32];
    block_sum<1>(mon, sm);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = mon[0];
  }
}

// Collision only (first sweep from an explicit f_S state): fout = C[fin, g], with the
// same arithmetic as k_primal so that a restart from a checkpoint reproduces the
// uninterrupted run bit for bit.
template <bool BOUNDED, int ARITH, bool FIELD>
__global__ void __launch_bounds__(256) k_collide_only(const double *__restrict__ fin,
                                                      double *__restrict__ fout,
                                                      const double *__restrict__ g2, Grid g,
                                                      Bounded b, Coef c0, Field fl) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long n = (long)y * g.nx + x;
  bool bnd = false;
  if (BOUNDED) {
    const uint8_t t = b.type[n];
    if (t == 0) return;
    bnd = t == 2;
  }
  const Coef c = node_coef<FIELD>(c0, fl, g.N, n, (FIELD && bnd) ? b.bidx[n] : -1);
  double f[8], o[8], dxn, dyn;
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] = fin[k * g.N + n];
  const double qx = g2[n], qy = g2[g.N + n];
  if (bnd)
    collide<true>(f, qx, qy, c, o, dxn, dyn);
  else if (ARITH == 0 || !collide_fix<false, false, !BOUNDED, !BOUNDED>(f, qx, qy, node_fix<FIELD>(c0.fx, fl, g.N, n), o,
                                             dxn, dyn))
    collide<false>(f, qx, qy, c, o, dxn, dyn);
#pragma unroll
  for (int k = 0; k < 8; ++k) fout[k * g.N + n] = o[k];
}

// f_S = S' f_C (no collision): checkpoint read-out of the primal state.
template <bool BOUNDED>
__global__ void k_pull_primal(const double *__restrict__ fin, double *__restrict__ fs, Grid g,
                              Bounded b) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long n = (long)y * g.nx + x;
  double f[8], gsel;
  if (!pull_primal<BOUNDED>(fin, x, y, g, b, f, gsel))
    for (int k = 0; k < 8; ++k) f[k] = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) fs[k * g.N + n] = f[k];
}

// phi_S = S'^T phi_C (no collision).
template <bool BOUNDED>
__global__ void k_pull_adjoint(const double *__restrict__ pin, double *__restrict__ ps, Grid g,
                               Bounded b) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long n = (long)y * g.nx + x;
  double p[8], gsel;
  if (!pull_adjoint<BOUNDED>(pin, x, y, g, b, p, gsel))
    for (int k = 0; k < 8; ++k) p[k] = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) ps[k * g.N + n] = p[k];
}

// Displacement of the primal state (source = explicit f_S or f_C(t-1) via pull).
template <bool BOUNDED, bool FROM_FC>
__global__ void k_displacement(const double *__restrict__ src, const double *__restrict__ g2,
                               double *__restrict__ d, Grid g, Bounded b) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long n = (long)y * g.nx + x;
  double f[8], gsel;
  bool act;
  if (FROM_FC) {
    act = pull_primal<BOUNDED>(src, x, y, g, b, f, gsel);
  } else {
    act = !BOUNDED || b.type[n] != 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = src[k * g.N + n];
  }
  double dxn = 0.0, dyn = 0.0;
  if (act) {
    dxn = (f[0] - f[2]) + (f[4] - f[6]) - (f[5] - f[7]) + 2.0 * g2[n];
    dyn = (f[1] - f[3]) + (f[4] - f[6]) + (f[5] - f[7]) + 2.0 * g2[g.N + n];
  }
  d[n] = dxn;
  d[g.N + n] = dyn;
}

// Objective partials and adjoint source: e = d - d*, J_n = 0.5 obs |e|^2 (times
// dx^2 / Cbar outside), r = (dx^2 / Cbar) obs e  (Eqs. node_J, discrete_J;
// (dJ/df_S)_k = r . c_k).
template <bool BOUNDED, bool FROM_FC>
__global__ void __launch_bounds__(256) k_objective(const double *__restrict__ src,
                                                   const double *__restrict__ g2,
                                                   const double *__restrict__ dstar,
                                                   const double *__restrict__ obs,
                                                   double *__restrict__ r, double scale, Grid g,
                                                   Bounded b, double *__restrict__ partial) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  double acc[1] = {0.0};
  if (x < g.nx && y < g.ny) {
    const long n = (long)y * g.nx + x;
    double f[8], gsel;
    bool act;
    if (FROM_FC) {
      act = pull_primal<BOUNDED>(src, x, y, g, b, f, gsel);
    } else {
      act = !BOUNDED || b.type[n] != 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = src[k * g.N + n];
    }
    double rx = 0.0, ry = 0.0;
    if (act) {
      const double w = obs ? obs[n] : 1.0;
      const double ex = (f[0] - f[2]) + (f[4] - f[6]) - (f[5] - f[7]) + 2.0 * g2[n] - dstar[n];
      const double ey = (f[1] - f[3]) + (f[4] - f[6]) + (f[5] - f[7]) + 2.0 * g2[g.N + n] -
                        dstar[g.N + n];
      acc[0] = w * (ex * ex + ey * ey);
      rx = scale * w * ex;
      ry = scale * w * ey;
    }
    r[n] = rx;
    r[g.N + n] = ry;
  }
  __shared__ double sm[32];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = acc[0];
}

// One adjoint sweep: phi_C(k+1) = A^T S'^T phi_C(k) - j; optional monitor of |d^phi|^2.
template <bool BOUNDED, bool MONITOR, int ARITH, bool FIELD>
__global__ void __launch_bounds__(256) k_adjoint(const double *__restrict__ pin,
                                                 double *__restrict__ pout,
                                                 const double *__restrict__ r, Grid g,
                                                 Bounded b, Coef c0, Field fl,
                                                 double *__restrict__ partial) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  double mon[1] = {0.0};
  if (x < g.nx && y < g.ny) {
    const long n = (long)y * g.nx + x;
    double p[8], gsel;
    if (pull_adjoint<BOUNDED>(pin, x, y, g, b, p, gsel)) {
      double o[8], ax = 0.0, ay = 0.0;
      const double rx = __ldg(r + n), ry = __ldg(r + g.N + n);
      const Coef c = node_coef<FIELD>(c0, fl, g.N, n,
                                      (BOUNDED && FIELD && gsel != 0.0) ? b.bidx[n] : -1);
      if (BOUNDED && gsel != 0.0)
        collide_T<true>(p, rx, ry, c, o, ax, ay);
      else if (ARITH == 0 ||
               !collide_T_fix<MONITOR, false, false, !BOUNDED, !BOUNDED>(p, rx, ry, node_fix<FIELD>(c0.fx, fl, g.N, n), o, ax, ay))
        collide_T<false>(p, rx, ry, c, o, ax, ay);
#pragma unroll
      for (int k = 0; k < 8; ++k) pout[k * g.N + n] = o[k];
      if (MONITOR) mon[0] = ax * ax + ay * ay;
    }
  }
  if (MONITOR) {
    __shared__ double sm[32];
    block_sum<1>(mon, sm);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = mon[0];
  }
}

// Force gradient (Eq. optimality): dJ/dF_n = dx^2 (r_n / 2 - (dC/dg)^T phi_S,n).
// MODE 0: write the 2N field (and its component sums for the zero-mean projection);
// MODE 1: reduce against the two basis fields: dJ/dalpha_i = sum_n Phi_i . dJ/dF_n.
template <bool BOUNDED, int MODE>
__global__ void __launch_bounds__(256) k_grad_force(const double *__restrict__ pin,
                                                    const double *__restrict__ r,
                                                    const double *__restrict__ basis,
                                                    double *__restrict__ grad, double dx2, Grid g,
                                                    Bounded b, double *__restrict__ partial) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  double acc[2] = {0.0, 0.0};
  if (x < g.nx && y < g.ny) {
    const long n = (long)y * g.nx + x;
    double p[8], gsel;
    double gx = 0.0, gy = 0.0;
    if (pull_adjoint<BOUNDED>(pin, x, y, g, b, p, gsel)) {
      double sx, sy;
      force_sensitivity(p, sx, sy);
      gx = dx2 * (0.5 * r[n] - sx);
      gy = dx2 * (0.5 * r[g.N + n] - sy);
    }
    if (MODE == 0) {
      grad[n] = gx;
      grad[g.N + n] = gy;
      acc[0] = gx;
      acc[1] = gy;
    } else {
      acc[0] = basis[n] * gx + basis[g.N + n] * gy;
      acc[1] = basis[2 * g.N + n] * gx + basis[3 * g.N + n] * gy;
    }
  }
  __shared__ double sm[64];
  block_sum<2>(acc, sm);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const long bl = blockIdx.y * gridDim.x + blockIdx.x;
    partial[bl * 2 + 0] = acc[0];
    partial[bl * 2 + 1] = acc[1];
  }
}

// ---------------------------------------------------------------------------------
// The objective pass and the force gradient of a periodic lattice with the node's
// arithmetic on the integer pipes.  Both kernels move ~100 B per node and did ~20 FP64
// instructions per node, which held them at ~2 TB/s on B300's FP64 pipe; here the
// differences of populations, force and target are formed in 64-bit fixed point at the
// largest exponent of the node's inputs (exact sums of the truncated inputs, one rounding
// back to binary64, within a few 2^-56 of the node's largest input, like the sweeps), and
// only the products and the sums of the reduction stay in FP64.  Nodes whose inputs fall
// outside [kEmin, kEmax] use the FP64 formula.  Grid-stride over the nodes (a fixed grid,
// so the partials and their reduction order are fixed).

// largest biased exponent of n values
template <int NV>
__device__ __forceinline__ int max_exp_n(const double (&v)[NV]) {
  int m = 0;
#pragma unroll
  for (int i = 0; i < NV; ++i) m = max(m, __double2hiint(v[i]) & 0x7fffffff);
  return m >> 20;
}

// e = d - d* (Eq. node_J) of one node from its pulled populations, force and target.
__device__ __forceinline__ void residual_e(const double (&f)[8], double gx, double gy,
                                           double sx, double sy, double &ex, double &ey) {
  const double v[12] = {f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], gx, gy, sx, sy};
  const int E = max_exp_n<12>(v);
  if (E >= kEmin && E <= kEmax) {
    long long F[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) F[k] = to_fix_alu(f[k], E);
    const long long b3 = F[4] - F[6], b4 = F[5] - F[7];
    const long long EX = (F[0] - F[2]) + (b3 - b4) + 2 * to_fix_alu(gx, E) - to_fix_alu(sx, E);
    const long long EY = (F[1] - F[3]) + (b3 + b4) + 2 * to_fix_alu(gy, E) - to_fix_alu(sy, E);
    ex = from_fix(EX, E);
    ey = from_fix(EY, E);
  } else {
    ex = (f[0] - f[2]) + (f[4] - f[6]) - (f[5] - f[7]) + 2.0 * gx - sx;
    ey = (f[1] - f[3]) + (f[4] - f[6]) + (f[5] - f[7]) + 2.0 * gy - sy;
  }
}

template <bool OBS>
__global__ void __launch_bounds__(256) k_objective_fix(const double *__restrict__ src,
                                                       const double *__restrict__ g2,
                                                       const double *__restrict__ dstar,
                                                       const double *__restrict__ obs,
                                                       double *__restrict__ r, double scale,
                                                       Grid g, double *__restrict__ partial) {
  double acc[1] = {0.0};
  const Bounded none{};
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < g.N;
       n += (long)gridDim.x * blockDim.x) {
    const int y = (int)(n / g.nx), x = (int)(n - (long)y * g.nx);
    double f[8], gsel, ex, ey;
    pull_primal<false>(src, x, y, g, none, f, gsel);
    residual_e(f, __ldg(g2 + n), __ldg(g2 + g.N + n), __ldg(dstar + n), __ldg(dstar + g.N + n),
               ex, ey);
    const double w = OBS ? __ldg(obs + n) : 1.0;
    const double e2 = fma(ex, ex, ey * ey);
    acc[0] += OBS ? w * e2 : e2;
    const double sw = OBS ? scale * w : scale;
    r[n] = sw * ex;
    r[g.N + n] = sw * ey;
  }
  __shared__ double sm[32];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc[0];
}

// Eq. optimality as k_grad_force: dJ/dF_n = dx^2 (r_n / 2 - (dC/dg)^T phi_S,n); MODE 0
// the field (and its component sums), MODE 1 the two basis projections.
template <int MODE>
__global__ void __launch_bounds__(256) k_grad_force_fix(const double *__restrict__ pin,
                                                        const double *__restrict__ r,
                                                        const double *__restrict__ basis,
                                                        double *__restrict__ grad, double dx2,
                                                        Grid g, double *__restrict__ partial) {
  double acc[2] = {0.0, 0.0};
  const Bounded none{};
  const FixC cA = fixc_of(0.5 * (1.0 - 0.5 * kTheta)), cB = fixc_of(0.125 * kTheta);
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < g.N;
       n += (long)gridDim.x * blockDim.x) {
    const int y = (int)(n / g.nx), x = (int)(n - (long)y * g.nx);
    double p[8], gsel;
    pull_adjoint<false>(pin, x, y, g, none, p, gsel);
    const double rx = __ldg(r + n), ry = __ldg(r + g.N + n);
    const double v[10] = {p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], rx, ry};
    const int E = max_exp_n<10>(v);
    double gx, gy;
    if (E >= kEmin && E <= kEmax) {
      long long P[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) P[k] = to_fix_alu(p[k], E);
      const long long B1 = P[0] - P[2], B2 = P[1] - P[3], B3 = P[4] - P[6], B4 = P[5] - P[7];
      const long long SX = mulfix(B1, cA) + mulfix(B3 - B4, cB);
      const long long SY = mulfix(B2, cA) + mulfix(B3 + B4, cB);
      gx = dx2 * from_fix((to_fix_alu(rx, E) >> 1) - SX, E);
      gy = dx2 * from_fix((to_fix_alu(ry, E) >> 1) - SY, E);
    } else {
      double sx, sy;
      force_sensitivity(p, sx, sy);
      gx = dx2 * (0.5 * rx - sx);
      gy = dx2 * (0.5 * ry - sy);
    }
    if (MODE == 0) {
      grad[n] = gx;
      grad[g.N + n] = gy;
      acc[0] += gx;
      acc[1] += gy;
    } else {
      acc[0] += __ldg(basis + n) * gx + __ldg(basis + g.N + n) * gy;
      acc[1] += __ldg(basis + 2 * g.N + n) * gx + __ldg(basis + 3 * g.N + n) * gy;
    }
  }
  __shared__ double sm[64];
  block_sum<2>(acc, sm);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 2 + 0] = acc[0];
    partial[blockIdx.x * 2 + 1] = acc[1];
  }
}

// Young's-modulus gradient (Eq. optimality with E entering omega_beta(E) and, at
// boundary nodes, gamma(E) and the Neumann rule):
//   dJ/dE = - sum_n phi_S,n^T dC_n/dE - sum_n phi_C,n^T (dS'/dE f_C)_n,
// with J free of E (the loads are held fixed) and dC_n/dE read off the pair form:
// c11 scales m11/4 on the diagonals (+,-,+,-), cs scales m_s on the axis pairs
// (1/4 + gamma/2) and on the diagonals (-gamma/4), cd scales m_d/4 on the axis pairs
// (+,-,+,-), gamma scales cs m_s (1/2 on axis, -1/4 on diagonals).
template <bool BOUNDED, bool FIELD>
__global__ void __launch_bounds__(256) k_grad_young(const double *__restrict__ fin,
                                                    const double *__restrict__ pin, Grid g,
                                                    Bounded b, Coef c0, YoungDeriv yd0, Field fl,
                                                    double *__restrict__ grad,
                                                    double *__restrict__ partial) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  double acc[1] = {0.0};
  if (x < g.nx && y < g.ny) {
    const long n = (long)y * g.nx + x;
    double f[8], p[8], gsel, gsel2;
    double gn = 0.0;
    if (pull_primal<BOUNDED>(fin, x, y, g, b, f, gsel) &&
        pull_adjoint<BOUNDED>(pin, x, y, g, b, p, gsel2)) {
      const bool bnd = BOUNDED && gsel != 0.0;
      const int bi = bnd ? b.bidx[n] : -1;
      const Coef c = node_coef<FIELD>(c0, fl, g.N, n, bi);
      YoungDeriv yd = yd0;
      if (FIELD) {
        // d(1 - omega)/dE = omega^2 dtau/dE with the node's omega = 1 - c
        const double w11 = 1.0 - c.c11, ws = 1.0 - c.cs, wd = 1.0 - c.cd;
        const double dt11 = 1.0 / (2.0 * (1.0 + fl.nu) * kTheta);
        const double dts = 1.0 / ((1.0 - fl.nu) * (1.0 + kTheta));
        const double dtd = 1.0 / ((1.0 + fl.nu) * (1.0 - kTheta));
        yd.dc11 = w11 * w11 * dt11;
        yd.dcs = ws * ws * dts;
        yd.dcd = wd * wd * dtd;
        const double ts = 1.0 / ws - 0.5;
        yd.dgam = BOUNDED ? -kTheta * 0.5 * dts / ((1.0 + kTheta) * (ts - 0.5) * (ts - 0.5)) : 0.0;
      }
      const double m11 = (f[4] + f[6]) - (f[5] + f[7]);
      const double ms = (f[0] + f[1] + f[2] + f[3]) + 2.0 * (f[4] + f[5] + f[6] + f[7]);
      const double md = (f[0] + f[2]) - (f[1] + f[3]);
      const double pax = p[0] + p[1] + p[2] + p[3], pdg = p[4] + p[5] + p[6] + p[7];
      const double gam = bnd ? c.gam : 0.0;
      double t = yd.dc11 * 0.25 * m11 * ((p[4] + p[6]) - (p[5] + p[7]));
      t += yd.dcd * 0.25 * md * ((p[0] + p[2]) - (p[1] + p[3]));
      t += yd.dcs * ms * ((0.25 + 0.5 * gam) * pax - 0.25 * gam * pdg);
      if (bnd) {
        t += yd.dgam * c.cs * ms * (0.5 * pax - 0.25 * pdg);
        const unsigned reg = b.regmask[bi];
        double own[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) own[j] = __ldg(fin + j * g.N + n);
        for (int k = 0; k < 8; ++k) {
          if (reg & (1u << k)) continue;
          double ds_ = b.ds[(long)bi * 8 + k];
#pragma unroll
          for (int j = 0; j < 8; ++j) ds_ += b.dQ[(long)bi * 64 + k * 8 + j] * own[j];
          t += __ldg(pin + k * g.N + n) * ds_;
        }
      }
      gn = -t;
    }
    if (FIELD)
      grad[n] = 2.0 * fl.alpha[n] * gn;  // E_n = alpha_n^2
    else
      acc[0] = gn;
  }
  if (!FIELD) {
    __shared__ double sm[32];
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = acc[0];
  }
}

// Per-node collision constants of a modulus field: E_n = alpha_n^2 (Eq. E_substitution),
// plane-stress moduli (Eqs. mu, K), relaxation (Table A.1, Eq. relaxation).
static __global__ void k_set_young_field(const double *__restrict__ alpha, double nu, long N,
                                  double *__restrict__ q, FixC *__restrict__ qfix) {
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N;
       n += (long)gridDim.x * blockDim.x) {
    const double E = alpha[n] * alpha[n];
    const double mu = E / (2.0 * (1.0 + nu)), K = E / (2.0 * (1.0 - nu));
    const double w11 = 1.0 / (mu / kTheta + 0.5);
    const double ws = 1.0 / (2.0 * K / (1.0 + kTheta) + 0.5);
    const double wd = 1.0 / (2.0 * mu / (1.0 - kTheta) + 0.5);
    q[n] = 0.25 * (1.0 - w11);
    q[N + n] = 0.25 * (1.0 - ws);
    q[2 * N + n] = 0.25 * (1.0 - wd);
    // round(c 2^62) as hi 2^31 + lo, 0 <= lo < 2^31 (|c| < 1/2, so |C| < 2^61)
    for (int i = 0; i < 3; ++i) {
      const long long C = __double2ll_rn(q[i * N + n] * 4611686018427387904.0);
      const long long hi = C >> 31;
      qfix[i * N + n] = FixC{(int)hi, (int)(C - hi * 2147483648ll)};
    }
  }
}

// Tangent of the streaming step at (x, y): tf_S = S' tf_C + Edot (dS'/dE f_C + ds/dE),
// i.e. the boundary rules without their constant part, plus their E-derivative applied
// to the primal post-collision state fprim.  Returns false for outside nodes; bnd tells
// whether the node is a boundary node.
template <bool BOUNDED, bool YOUNG>
__device__ __forceinline__ bool pull_tangent(const double *__restrict__ tin,
                                             const double *__restrict__ fprim, int x, int y,
                                             const Grid &g, const Bounded &b, double Edot,
                                             double (&t)[8], bool &bnd) {
  const long n = (long)y * g.nx + x;
  double gsel;
  bnd = false;
  if (!BOUNDED) return pull_primal<false>(tin, x, y, g, b, t, gsel);
  const uint8_t ty = b.type[n];
  if (ty == 0) return false;
  if (ty == 1) return pull_primal<true>(tin, x, y, g, b, t, gsel);
  bnd = true;
  const int bi = b.bidx[n];
  const unsigned reg = b.regmask[bi];
  double own[8], ownf[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    own[j] = tin[j * g.N + n];
    ownf[j] = YOUNG ? fprim[j * g.N + n] : 0.0;
  }
  for (int k = 0; k < 8; ++k) {
    if (reg & (1u << k)) {
      t[k] = tin[k * g.N + n - kCX[k] - (long)kCY[k] * g.nx];
    } else {
      double acc = 0.0, dacc = YOUNG ? b.ds[(long)bi * 8 + k] : 0.0;
      for (int j = 0; j < 8; ++j) {
        acc += b.Q[(long)bi * 64 + k * 8 + j] * own[j];
        if (YOUNG) dacc += b.dQ[(long)bi * 64 + k * 8 + j] * ownf[j];
      }
      t[k] = acc + (YOUNG ? Edot * dacc : 0.0);
    }
  }
  return true;
}

// Forward-mode (f-AD, Eq. fAD) tangent sweep at a converged primal state (held in fprim
// as f_C, so that f_S = S' f_C + s): the tangent obeys the differentiated step
//   tf_S = S' tf_C + Edot (dS'/dE f_C + ds/dE),
//   tf_C = A tf_S + B tg + Edot (dC/dE) f_S,
// with tg = dx^2 dF (the force direction, kept as q-dot = tg / 4) and Edot the modulus
// direction.  dC/dE uses the same pair-form derivatives as k_grad_young.
template <bool BOUNDED, bool YOUNG>
__global__ void __launch_bounds__(256) k_tangent(const double *__restrict__ fprim,
                                                 const double *__restrict__ tin,
                                                 double *__restrict__ tout,
                                                 const double *__restrict__ qdot, Grid g,
                                                 Bounded b, Coef c, YoungDeriv yd, double Edot) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long n = (long)y * g.nx + x;
  double t[8];
  bool bnd;
  if (!pull_tangent<BOUNDED, YOUNG>(tin, fprim, x, y, g, b, Edot, t, bnd)) return;
  double o[8], dd, de;
  const double qx = qdot ? qdot[n] : 0.0, qy = qdot ? qdot[g.N + n] : 0.0;
  if (bnd)
    collide<true>(t, qx, qy, c, o, dd, de);
  else
    collide<false>(t, qx, qy, c, o, dd, de);
  if (YOUNG) {
    double f[8], gs2;
    pull_primal<BOUNDED>(fprim, x, y, g, b, f, gs2);
    const double m11 = (f[4] + f[6]) - (f[5] + f[7]);
    const double ms = (f[0] + f[1] + f[2] + f[3]) + 2.0 * (f[4] + f[5] + f[6] + f[7]);
    const double md = (f[0] + f[2]) - (f[1] + f[3]);
    const double gam = bnd ? c.gam : 0.0;
    const double d11 = Edot * yd.dc11 * 0.25 * m11;
    const double dd_ = Edot * yd.dcd * 0.25 * md;
    double dax = Edot * yd.dcs * ms * (0.25 + 0.5 * gam);
    double ddg = -Edot * yd.dcs * ms * 0.25 * gam;
    if (bnd) {
      dax += Edot * yd.dgam * c.cs * ms * 0.5;
      ddg -= Edot * yd.dgam * c.cs * ms * 0.25;
    }
    o[0] += dax + dd_;
    o[2] += dax + dd_;
    o[1] += dax - dd_;
    o[3] += dax - dd_;
    o[4] += ddg + d11;
    o[6] += ddg + d11;
    o[5] += ddg - d11;
    o[7] += ddg - d11;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) tout[k * g.N + n] = o[k];
}

// dJ along the tangent: sum_n obs (d - d*) . d-dot, with d from the primal state and
// d-dot = m10(tf_S) + 2 q-dot (times dx^2 / Cbar outside).
template <bool BOUNDED, bool YOUNG>
__global__ void __launch_bounds__(256) k_tangent_objective(
    const double *__restrict__ fprim, const double *__restrict__ tcur,
    const double *__restrict__ g2, const double *__restrict__ qdot,
    const double *__restrict__ dstar, const double *__restrict__ obs, Grid g, Bounded b,
    double Edot, double *__restrict__ partial) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  double acc[1] = {0.0};
  if (x < g.nx && y < g.ny) {
    const long n = (long)y * g.nx + x;
    double f[8], t[8], gs;
    bool bnd;
    if (pull_primal<BOUNDED>(fprim, x, y, g, b, f, gs) &&
        pull_tangent<BOUNDED, YOUNG>(tcur, fprim, x, y, g, b, Edot, t, bnd)) {
      const double w = obs ? obs[n] : 1.0;
      const double ex = (f[0] - f[2]) + (f[4] - f[6]) - (f[5] - f[7]) + 2.0 * g2[n] - dstar[n];
      const double ey = (f[1] - f[3]) + (f[4] - f[6]) + (f[5] - f[7]) + 2.0 * g2[g.N + n] -
                        dstar[g.N + n];
      const double tx = (t[0] - t[2]) + (t[4] - t[6]) - (t[5] - t[7]) + (qdot ? 2.0 * qdot[n] : 0.0);
      const double ty = (t[1] - t[3]) + (t[4] - t[6]) + (t[5] - t[7]) +
                        (qdot ? 2.0 * qdot[g.N + n] : 0.0);
      acc[0] = w * (ex * tx + ey * ty);
    }
  }
  __shared__ double sm[32];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = acc[0];
}

// Subtract per-component means over active nodes (Eq. zero_mean_projection).
template <bool BOUNDED>
__global__ void k_subtract_mean(double *__restrict__ v, const double *__restrict__ mean, Grid g,
                                Bounded b) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long n = (long)y * g.nx + x;
  if (BOUNDED && b.type[n] == 0) return;
  v[n] -= mean[0];
  v[g.N + n] -= mean[1];
}

// ---------------------------------------------------------------------------------
// Compact launch of a bounded grid.  The box is mostly outside the domain, and a warp
// that holds one boundary node runs that node's rule and gamma-modified collision on
// the FP64 pipe for all its lanes.  So the sweep launches only active nodes: first
// `bblocks` blocks of boundary nodes packed one per thread (they take longest, so
// they start first), then the interior nodes as warp-sized chunks of up to 32
// consecutive nodes of one row (every pull of such a warp is a contiguous, coalesced
// access).  Interior nodes have all eight links regular.  A block holds blockDim.x
// boundary records or blockDim.x / 32 chunks; every kernel of one compact layout is
// launched with the same block size (a multiple of 32, at most kCompactThreads).
constexpr int kCompactThreads = 128;

struct Compact {
  const int2 *chunk;      // nchunk: (first node, count <= 32) of interior nodes of a row
  const int *bnode;       // nb: node of boundary record b
  const double *R;        // nb * 32: compact rules [(k*4 + i)*nb + b] (lbm_boundary.cuh)
  const uint8_t *negmask; // nb: bit k set <=> missing link k is Neumann (sigma_k = -1)
  long nchunk, nb;
  int bblocks;            // blocks of boundary nodes (first in the grid)
};

// Missing-link populations of boundary record bi at node n from its own post-collision
// populations own[] (compact rule form); regular links pulled as usual.  HOIST issues
// every load of the record (own and pulled populations, the rule coefficients of all
// missing links) before the first arithmetic: one L2 round trip instead of one per
// missing link (a rule's coefficients are otherwise loaded inside its branch and used
// at once), for more registers; the host takes it where the sweep is latency-bound.
// The HOIST kernels also convert interior nodes' populations on the integer pipes
// (measured at N_x = 512: primal 5.31 -> 5.04 us, adjoint 5.91 -> 5.26 us per sweep; on
// the 128-thread launch of N_x = 1024 it cost 12 %, so the other kernels keep to_fix).
template <bool NC = true, bool HOIST = false>
__device__ __forceinline__ void pull_boundary_c(const double *__restrict__ fin, long n,
                                                const Grid &g, const Bounded &b,
                                                const Compact &c, long bi,
                                                double (&f)[8]) {
  const unsigned reg = b.regmask[bi];
  const unsigned neg = c.negmask[bi];
  double own[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) own[j] = ldp<NC>(fin + j * g.N + n);
  if (HOIST) {
    double rk[8][4];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (reg & (1u << k)) {
        f[k] = ldp<NC>(fin + k * g.N + n - kCX[k] - (long)kCY[k] * g.nx);
        rk[k][0] = rk[k][1] = rk[k][2] = rk[k][3] = 0.0;
      } else {
        const double *r = c.R + (long)(k * 4) * c.nb + bi;
        rk[k][0] = __ldg(r);
        rk[k][1] = __ldg(r + c.nb);
        rk[k][2] = __ldg(r + 2 * c.nb);
        rk[k][3] = __ldg(r + 3 * c.nb);
      }
    }
    const double mc11 = (own[4] - own[5]) + (own[6] - own[7]);
    const double mcs = ((own[0] + own[1]) + (own[2] + own[3])) +
                       2.0 * ((own[4] + own[5]) + (own[6] + own[7]));
    const double mcd = (own[0] - own[1]) + (own[2] - own[3]);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (!(reg & (1u << k))) {
        const int kb = (k < 4) ? ((k + 2) & 3) : (((k - 4 + 2) & 3) + 4);
        const double ob = (neg & (1u << k)) ? -own[kb] : own[kb];
        f[k] = fma(rk[k][0], mc11, fma(rk[k][1], mcs, fma(rk[k][2], mcd, ob + rk[k][3])));
      }
    }
    return;
  }
  const double mc11 = (own[4] - own[5]) + (own[6] - own[7]);
  const double mcs = ((own[0] + own[1]) + (own[2] + own[3])) +
                     2.0 * ((own[4] + own[5]) + (own[6] + own[7]));
  const double mcd = (own[0] - own[1]) + (own[2] - own[3]);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (reg & (1u << k)) {
      f[k] = ldp<NC>(fin + k * g.N + n - kCX[k] - (long)kCY[k] * g.nx);
    } else {
      const int kb = (k < 4) ? ((k + 2) & 3) : (((k - 4 + 2) & 3) + 4);
      const double *r = c.R + (long)(k * 4) * c.nb + bi;
      const double ob = (neg & (1u << k)) ? -own[kb] : own[kb];
      f[k] = fma(__ldg(r), mc11, fma(__ldg(r + c.nb), mcs,
                 fma(__ldg(r + 2 * c.nb), mcd, ob + __ldg(r + 3 * c.nb))));
    }
  }
}

// Transposed pull of boundary record bi: phi_S,j(x) = [link jbar regular] phi_C,j(x + c_j)
// + sigma_jbar [link jbar missing] phi_C,jbar(x) + sum_i t_i dm_i/df_j, with
// t_i = sum over missing links k of r_ki phi_C,k(x) (the transpose of pull_boundary_c).
template <bool NC = true, bool HOIST = false>
__device__ __forceinline__ void pull_boundary_adj_c(const double *__restrict__ pin, long n,
                                                    const Grid &g, const Bounded &b,
                                                    const Compact &c, long bi,
                                                    double (&p)[8]) {
  const unsigned reg = b.regmask[bi];
  const unsigned neg = c.negmask[bi];
  double own[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) own[k] = ldp<NC>(pin + k * g.N + n);
  double t11 = 0.0, ts = 0.0, td = 0.0;
  double pv[8];  // HOIST: the regular links' pulled values, loaded up front
  if (HOIST) {  // all loads first (see pull_boundary_c)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int jb = (j < 4) ? ((j + 2) & 3) : (((j - 4 + 2) & 3) + 4);
      pv[j] = (reg & (1u << jb)) ? ldp<NC>(pin + j * g.N + n + kCX[j] + (long)kCY[j] * g.nx)
                                 : 0.0;
    }
    double rk[8][3];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double *r = c.R + (long)(k * 4) * c.nb + bi;
      const bool miss = !(reg & (1u << k));
      rk[k][0] = miss ? __ldg(r) : 0.0;
      rk[k][1] = miss ? __ldg(r + c.nb) : 0.0;
      rk[k][2] = miss ? __ldg(r + 2 * c.nb) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (!(reg & (1u << k))) {
        t11 = fma(rk[k][0], own[k], t11);
        ts = fma(rk[k][1], own[k], ts);
        td = fma(rk[k][2], own[k], td);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (!(reg & (1u << k))) {
        const double *r = c.R + (long)(k * 4) * c.nb + bi;
        t11 = fma(__ldg(r), own[k], t11);
        ts = fma(__ldg(r + c.nb), own[k], ts);
        td = fma(__ldg(r + 2 * c.nb), own[k], td);
      }
    }
  }
  const double ax = ts + td, ay = ts - td, d1 = 2.0 * ts + t11, d2 = 2.0 * ts - t11;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int jb = (j < 4) ? ((j + 2) & 3) : (((j - 4 + 2) & 3) + 4);
    double acc;
    if (reg & (1u << jb)) {
      acc = HOIST ? pv[j] : ldp<NC>(pin + j * g.N + n + kCX[j] + (long)kCY[j] * g.nx);
    } else {
      acc = (neg & (1u << jb)) ? -own[jb] : own[jb];
    }
    // dm11/df = (0,0,0,0,1,-1,1,-1), dms/df = (1,1,1,1,2,2,2,2), dmd/df = (1,-1,1,-1,0,..)
    const double m = j < 4 ? ((j & 1) ? ay : ax) : ((j & 1) ? d2 : d1);
    p[j] = acc + m;
  }
}

// The per-thread work of a primal sweep of a bounded grid (compact launch, block
// blockIdx.x); mon receives |d|^2 of the thread's node (0 if none).
template <bool MONITOR, int ARITH, bool FIELD, bool HOIST = false>
__device__ __forceinline__ void sweep_primal_c(const double *__restrict__ fin,
                                               double *__restrict__ fout,
                                               const double *__restrict__ g2, const Grid &g,
                                               const Bounded &b, const Compact &c,
                                               const Coef &c0, const Field &fl, double &mon) {
  mon = 0.0;
  if ((int)blockIdx.x < c.bblocks) {
    const long bi = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (bi < c.nb) {
      const long n = c.bnode[bi];
      double f[8], o[8], dxn = 0.0, dyn = 0.0, qx, qy;
      CoefFix cf;
      bool fix_ok;
      if (HOIST) {  // the node's other loads before the pull's arithmetic as well
        qx = __ldg(g2 + n);
        qy = __ldg(g2 + g.N + n);
        fix_ok = ARITH != 0 && node_fix_bnd<FIELD>(c0.fx, fl, g.N, n, bi, cf);
        pull_boundary_c<true, true>(fin, n, g, b, c, bi, f);
      } else {
        pull_boundary_c<true, false>(fin, n, g, b, c, bi, f);
        qx = __ldg(g2 + n);
        qy = __ldg(g2 + g.N + n);
        fix_ok = ARITH != 0 && node_fix_bnd<FIELD>(c0.fx, fl, g.N, n, bi, cf);
      }
      if (!fix_ok || !collide_fix<MONITOR, true>(f, qx, qy, cf, o, dxn, dyn))
        collide<true>(f, qx, qy, node_coef<FIELD>(c0, fl, g.N, n, (int)bi), o, dxn, dyn);
#pragma unroll
      for (int k = 0; k < 8; ++k) fout[k * g.N + n] = o[k];
      if (MONITOR) mon = dxn * dxn + dyn * dyn;
    }
  } else {
    const long w = ((long)(blockIdx.x - c.bblocks) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w < c.nchunk) {
      const int2 ch = c.chunk[w];
      if (lane < ch.y) {
        const long n = (long)ch.x + lane;
        double f[8], o[8], dxn = 0.0, dyn = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          f[k] = __ldg(fin + k * g.N + n - kCX[k] - (long)kCY[k] * g.nx);
        const double qx = __ldg(g2 + n), qy = __ldg(g2 + g.N + n);
        // (interior nodes are still all zero in the first sweeps of a traction-driven
        // solve from rest: they map to zero without the FP64 pipe)
        if (ARITH == 0 ||
            !collide_fix<MONITOR, false, HOIST>(f, qx, qy, node_fix<FIELD>(c0.fx, fl, g.N, n), o, dxn, dyn))
          if (ARITH == 0 || !zero_node(f, qx, qy, o))
            collide<false>(f, qx, qy, node_coef<FIELD>(c0, fl, g.N, n, -1), o, dxn, dyn);
#pragma unroll
        for (int k = 0; k < 8; ++k) fout[k * g.N + n] = o[k];
        if (MONITOR) mon = dxn * dxn + dyn * dyn;
      }
    }
  }
}

// One primal sweep of a bounded grid (compact launch); monitor partial per block.
template <bool MONITOR, int ARITH, bool FIELD, bool HOIST>
__global__ void __launch_bounds__(kCompactThreads) k_primal_c(const double *__restrict__ fin,
                                                              double *__restrict__ fout,
                                                              const double *__restrict__ g2,
                                                              Grid g, Bounded b, Compact c,
                                                              Coef c0, Field fl,
                                                              double *__restrict__ partial) {
  double mon[1];
  sweep_primal_c<MONITOR, ARITH, FIELD, HOIST>(fin, fout, g2, g, b, c, c0, fl, mon[0]);
  if (MONITOR) {
    __shared__ double sm[32];
    block_sum<1>(mon, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = mon[0];
  }
}

// Batches of one bounded geometry: instance blockIdx.y has its own populations
// ([8 N i, 8 N (i + 1))) and its own per-node material (modulus field planes and
// boundary records); the geometry lists and the force are shared.
__device__ __forceinline__ void offset_instance(long i, const Grid &g, Field &fl, Compact &c) {
  fl.q += 3 * g.N * i;
  fl.qfix += 3 * g.N * i;
  fl.gam += c.nb * i;
  fl.bfix += 2 * c.nb * i;
  fl.bok += c.nb * i;
  fl.alpha += g.N * i;
  c.R += 32 * c.nb * i;
}

template <int ARITH>
__global__ void __launch_bounds__(kCompactThreads) k_primal_cb(const double *__restrict__ fin,
                                                               double *__restrict__ fout,
                                                               const double *__restrict__ g2,
                                                               Grid g, Bounded b, Compact c,
                                                               Coef c0, Field fl) {
  const long i = blockIdx.y;
  offset_instance(i, g, fl, c);
  double mon;
  sweep_primal_c<false, ARITH, true>(fin + 8 * g.N * i, fout + 8 * g.N * i, g2, g, b, c, c0,
                                     fl, mon);
}

// First sweep of a batch from explicit states f_S (collision only), compact launch.
template <int ARITH>
__global__ void __launch_bounds__(kCompactThreads) k_collide_cb(const double *__restrict__ fin,
                                                                double *__restrict__ fout,
                                                                const double *__restrict__ g2,
                                                                Grid g, Compact c, Coef c0,
                                                                Field fl) {
  const long i = blockIdx.y;
  offset_instance(i, g, fl, c);
  fin += 8 * g.N * i;
  fout += 8 * g.N * i;
  long n = -1, bi = -1;
  if ((int)blockIdx.x < c.bblocks) {
    bi = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (bi < c.nb) n = c.bnode[bi];
  } else {
    const long w = ((long)(blockIdx.x - c.bblocks) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w < c.nchunk) {
      const int2 ch = c.chunk[w];
      if (lane < ch.y) n = (long)ch.x + lane;
    }
  }
  if (n < 0) return;
  double f[8], o[8], dxn, dyn;
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] = fin[k * g.N + n];
  const double qx = g2[n], qy = g2[g.N + n];
  if (bi >= 0 && bi < c.nb) {
    CoefFix cf;
    if (ARITH == 0 || !node_fix_bnd<true>(c0.fx, fl, g.N, n, bi, cf) ||
        !collide_fix<false, true>(f, qx, qy, cf, o, dxn, dyn))
      collide<true>(f, qx, qy, node_coef<true>(c0, fl, g.N, n, (int)bi), o, dxn, dyn);
  } else if (ARITH == 0 ||
             !collide_fix<false>(f, qx, qy, node_fix<true>(c0.fx, fl, g.N, n), o, dxn, dyn)) {
    if (ARITH == 0 || !zero_node(f, qx, qy, o))
      collide<false>(f, qx, qy, node_coef<true>(c0, fl, g.N, n, -1), o, dxn, dyn);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) fout[k * g.N + n] = o[k];
}

// f_S = S' f_C of every instance of a batch (compact launch; inactive nodes untouched).
static __global__ void __launch_bounds__(kCompactThreads) k_pull_cb(
    const double *__restrict__ fin, double *__restrict__ fs, Grid g, Bounded b, Compact c) {
  const long i = blockIdx.y;
  Field unused{};
  offset_instance(i, g, unused, c);
  fin += 8 * g.N * i;
  fs += 8 * g.N * i;
  double f[8];
  if ((int)blockIdx.x < c.bblocks) {
    const long bi = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (bi >= c.nb) return;
    const long n = c.bnode[bi];
    pull_boundary_c(fin, n, g, b, c, bi, f);
#pragma unroll
    for (int k = 0; k < 8; ++k) fs[k * g.N + n] = f[k];
  } else {
    const long w = ((long)(blockIdx.x - c.bblocks) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= c.nchunk) return;
    const int2 ch = c.chunk[w];
    if (lane >= ch.y) return;
    const long n = (long)ch.x + lane;
#pragma unroll
    for (int k = 0; k < 8; ++k) fs[k * g.N + n] = fin[k * g.N + n - kCX[k] - (long)kCY[k] * g.nx];
  }
}

// One adjoint sweep of a bounded grid (compact launch).
template <bool MONITOR, int ARITH, bool FIELD, bool HOIST>
__global__ void __launch_bounds__(kCompactThreads) k_adjoint_c(const double *__restrict__ pin,
                                                               double *__restrict__ pout,
                                                               const double *__restrict__ r,
                                                               Grid g, Bounded b, Compact c,
                                                               Coef c0, Field fl,
                                                               double *__restrict__ partial) {
  double mon[1] = {0.0};
  if ((int)blockIdx.x < c.bblocks) {
    const long bi = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (bi < c.nb) {
      const long n = c.bnode[bi];
      double p[8], o[8], ax = 0.0, ay = 0.0, rx, ry;
      CoefFix cf;
      bool fix_ok;
      if (HOIST) {
        rx = __ldg(r + n);
        ry = __ldg(r + g.N + n);
        fix_ok = ARITH != 0 && node_fix_bnd<FIELD>(c0.fx, fl, g.N, n, bi, cf);
        pull_boundary_adj_c<true, true>(pin, n, g, b, c, bi, p);
      } else {
        pull_boundary_adj_c<true, false>(pin, n, g, b, c, bi, p);
        rx = __ldg(r + n);
        ry = __ldg(r + g.N + n);
        fix_ok = ARITH != 0 && node_fix_bnd<FIELD>(c0.fx, fl, g.N, n, bi, cf);
      }
      if (!fix_ok || !collide_T_fix<MONITOR, true>(p, rx, ry, cf, o, ax, ay))
        collide_T<true>(p, rx, ry, node_coef<FIELD>(c0, fl, g.N, n, (int)bi), o, ax, ay);
#pragma unroll
      for (int k = 0; k < 8; ++k) pout[k * g.N + n] = o[k];
      if (MONITOR) mon[0] = ax * ax + ay * ay;
    }
  } else {
    const long w = ((long)(blockIdx.x - c.bblocks) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w < c.nchunk) {
      const int2 ch = c.chunk[w];
      if (lane < ch.y) {
        const long n = (long)ch.x + lane;
        double p[8], o[8], ax = 0.0, ay = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          p[k] = __ldg(pin + k * g.N + n + kCX[k] + (long)kCY[k] * g.nx);
        const double rx = __ldg(r + n), ry = __ldg(r + g.N + n);
        if (ARITH == 0 ||
            !collide_T_fix<MONITOR, false, false, HOIST>(p, rx, ry, node_fix<FIELD>(c0.fx, fl, g.N, n), o, ax, ay))
          if (ARITH == 0 || !zero_node(p, rx, ry, o))
            collide_T<false>(p, rx, ry, node_coef<FIELD>(c0, fl, g.N, n, -1), o, ax, ay);
#pragma unroll
        for (int k = 0; k < 8; ++k) pout[k * g.N + n] = o[k];
        if (MONITOR) mon[0] = ax * ax + ay * ay;
      }
    }
  }
  if (MONITOR) {
    __shared__ double sm[32];
    block_sum<1>(mon, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = mon[0];
  }
}

// Residual partials of a bounded grid over its active nodes only (compact launch):
// max |a - b| and max |a| over the eight planes.
static __global__ void __launch_bounds__(kCompactThreads) k_residual_c(
    const double *__restrict__ a, const double *__restrict__ bb, Grid g, Compact c,
    double *__restrict__ partial) {
  double v[2] = {0.0, 0.0};
  long n = -1;
  if ((int)blockIdx.x < c.bblocks) {
    const long bi = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (bi < c.nb) n = c.bnode[bi];
  } else {
    const long w = ((long)(blockIdx.x - c.bblocks) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w < c.nchunk) {
      const int2 ch = c.chunk[w];
      if (lane < ch.y) n = (long)ch.x + lane;
    }
  }
  if (n >= 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double ai = a[k * g.N + n];
      v[0] = nan_max(v[0], fabs(ai - bb[k * g.N + n]));
      v[1] = nan_max(v[1], fabs(ai));
    }
  }
  __shared__ double sm[64];
  block_max<2>(v, sm);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 2 + 0] = v[0];
    partial[blockIdx.x * 2 + 1] = v[1];
  }
}

// First adjoint sweep from rest: phi_C(1) = A^T S'^T 0 - j = -j (Eq. adjoint_iteration
// with phi_C(0) = 0), written without reading the zero state: the values are those of
// the transposed collision (lbm_device.cuh) with psi = 0, j_k = r . c_k.  Bounded grids
// write their active nodes only (the others keep the zeros they were created with).
template <bool BOUNDED>
__global__ void __launch_bounds__(256) k_adjoint_rest(const double *__restrict__ r,
                                                      double *__restrict__ pout, Grid g,
                                                      Bounded b) {
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < g.N;
       n += (long)gridDim.x * blockDim.x) {
    if (BOUNDED && b.type[n] == 0) continue;
    const double rx = r[n], ry = r[g.N + n];
    const double P1 = -rx - ry, P2 = rx - ry;
    pout[0 * g.N + n] = -rx;
    pout[1 * g.N + n] = -ry;
    pout[2 * g.N + n] = rx;
    pout[3 * g.N + n] = ry;
    pout[4 * g.N + n] = P1;
    pout[5 * g.N + n] = P2;
    pout[6 * g.N + n] = -P1;
    pout[7 * g.N + n] = -P2;
  }
}

// ---------------------------------------------------------------------------------
// Cluster-resident sweeps for small lattices.  A lattice of a few thousand nodes is
// latency-bound: each sweep launch costs more than its work.  One launch of a thread
// block cluster (up to 16 CTAs, one GPC) runs a whole chunk of sweeps (the host uses it
// for periodic lattices of up to 2048 nodes, where it measured faster); the sweeps are
// ordered by the hardware cluster barrier with release / acquire semantics at cluster
// scope, which makes every thread's writes of sweep s visible to every thread of the
// cluster before sweep s + 1 reads them.  Populations are read with coherent loads
// (they change within the launch); constants through the read-only path.
//
// Work items: periodic lattices, item = node; bounded grids, items [0, nb) are the
// boundary records and [nb, nb + ninner) the interior nodes of `inner`.
struct ClusterWork {
  const int *inner;  // bounded: interior nodes
  long nitems;
};

__device__ __forceinline__ void cluster_sync_release_acquire() {
  asm volatile("barrier.cluster.arrive.release;\n\t"
               "barrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// State of a solve loop that runs on the device (a cluster kernel that loops over chunks
// itself, or a CUDA graph whose conditional WHILE node repeats chunk -> residual ->
// decision): the tolerance and the chunk limit in, the chunks run and the last residual
// out.
struct LoopState {
  double tol;
  long long max_iters, iters;
  double metric;
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ double ld_cluster(unsigned local_addr, unsigned rank) {
  unsigned remote;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_addr), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
  return v;
}

// The residual rule's decision at the end of a chunk, taken identically by every CTA of
// a cluster: (v0, v1) are the thread's max |f(t) - f(t-1)| and max |f(t)|; the cluster
// maxima (NaN propagating, so order-free) give r = v0 / v1, as the host loop computes it;
// stop when r is below tol or not finite, or when chunk `it` is the last allowed.
// `red` (2 doubles) and `flag` are the CTA's shared slots, `sm` block_max scratch.
__device__ __forceinline__ bool cluster_residual_stop(double v0, double v1, double tol,
                                                      long long it, long long max_iters,
                                                      double *red, double *sm, double *flag) {
  double v[2] = {v0, v1};
  block_max<2>(v, sm);
  if (threadIdx.x == 0) {
    red[0] = v[0];
    red[1] = v[1];
  }
  cluster_sync_release_acquire();
  if (threadIdx.x < 32) {  // lane q reads CTA q's maxima (a cluster has at most 16 CTAs)
    const unsigned C = cluster_size(), q = threadIdx.x;
    double a = 0.0, b = 0.0;
    if (q < C) {
      a = ld_cluster(smem_addr(red), q);
      b = ld_cluster(smem_addr(red + 1), q);
    }
    for (int o = 16; o > 0; o >>= 1) {
      a = nan_max(a, __shfl_down_sync(0xffffffffu, a, o));
      b = nan_max(b, __shfl_down_sync(0xffffffffu, b, o));
    }
    if (q == 0) {
      double r = b > 0.0 ? a / b : (a > 0.0 ? INFINITY : 0.0);
      if (!isfinite(a) || !isfinite(b)) r = NAN;
      flag[0] = (!(r >= tol) || it + 1 >= max_iters) ? 1.0 : 0.0;
      flag[1] = r;
    }
  }
  __syncthreads();
  return flag[0] != 0.0;
}

// One item of a primal sweep (coherent population loads); mon += |d|^2 if MON.
template <bool BOUNDED, int ARITH, bool FIELD, bool MON>
__device__ __forceinline__ void primal_item(const double *fin, double *fout,
                                            const double *__restrict__ g2, const Grid &g,
                                            const Bounded &b, const Compact &c,
                                            const Coef &c0, const Field &fl,
                                            const ClusterWork &w, long it, double &mon) {
  double f[8], o[8], dxn = 0.0, dyn = 0.0;
  long n;
  if (BOUNDED && it < c.nb) {
    n = c.bnode[it];
    pull_boundary_c<false>(fin, n, g, b, c, it, f);
    const double qx = __ldg(g2 + n), qy = __ldg(g2 + g.N + n);
    CoefFix cf;
    if (ARITH == 0 || !node_fix_bnd<FIELD>(c0.fx, fl, g.N, n, it, cf) ||
        !collide_fix<MON, true>(f, qx, qy, cf, o, dxn, dyn))
      collide<true>(f, qx, qy, node_coef<FIELD>(c0, fl, g.N, n, (int)it), o, dxn, dyn);
  } else {
    if (BOUNDED) {
      n = w.inner[it - c.nb];
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = fin[k * g.N + n - kCX[k] - (long)kCY[k] * g.nx];
    } else {
      n = it;
      double gs;
      pull_primal<false, false>(fin, (int)(n % g.nx), (int)(n / g.nx), g, b, f, gs);
    }
    const double qx = __ldg(g2 + n), qy = __ldg(g2 + g.N + n);
    if (ARITH == 0 ||
        !collide_fix<MON, false, !BOUNDED, !BOUNDED>(f, qx, qy, node_fix<FIELD>(c0.fx, fl, g.N, n), o, dxn, dyn))
      if (ARITH == 0 || !zero_node(f, qx, qy, o))
        collide<false>(f, qx, qy, node_coef<FIELD>(c0, fl, g.N, n, -1), o, dxn, dyn);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) fout[k * g.N + n] = o[k];
  if (MON) mon += dxn * dxn + dyn * dyn;
}

// One item of an adjoint sweep (coherent loads); mon += |d^phi|^2 if MON.
template <bool BOUNDED, int ARITH, bool FIELD, bool MON>
__device__ __forceinline__ void adjoint_item(const double *pin, double *pout,
                                             const double *__restrict__ r, const Grid &g,
                                             const Bounded &b, const Compact &c,
                                             const Coef &c0, const Field &fl,
                                             const ClusterWork &w, long it, double &mon) {
  double p[8], o[8], ax = 0.0, ay = 0.0;
  long n;
  if (BOUNDED && it < c.nb) {
    n = c.bnode[it];
    pull_boundary_adj_c<false>(pin, n, g, b, c, it, p);
    const double rx = __ldg(r + n), ry = __ldg(r + g.N + n);
    CoefFix cf;
    if (ARITH == 0 || !node_fix_bnd<FIELD>(c0.fx, fl, g.N, n, it, cf) ||
        !collide_T_fix<MON, true>(p, rx, ry, cf, o, ax, ay))
      collide_T<true>(p, rx, ry, node_coef<FIELD>(c0, fl, g.N, n, (int)it), o, ax, ay);
  } else {
    if (BOUNDED) {
      n = w.inner[it - c.nb];
#pragma unroll
      for (int k = 0; k < 8; ++k) p[k] = pin[k * g.N + n + kCX[k] + (long)kCY[k] * g.nx];
    } else {
      n = it;
      double gs;
      pull_adjoint<false, false>(pin, (int)(n % g.nx), (int)(n / g.nx), g, b, p, gs);
    }
    const double rx = __ldg(r + n), ry = __ldg(r + g.N + n);
    if (ARITH == 0 ||
        !collide_T_fix<MON, false, false, !BOUNDED, !BOUNDED>(p, rx, ry, node_fix<FIELD>(c0.fx, fl, g.N, n), o, ax, ay))
      if (ARITH == 0 || !zero_node(p, rx, ry, o))
        collide_T<false>(p, rx, ry, node_coef<FIELD>(c0, fl, g.N, n, -1), o, ax, ay);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) pout[k * g.N + n] = o[k];
  if (MON) mon += ax * ax + ay * ay;
}

// One node of a periodic sweep shared by the lane pair (2j, 2j + 1) of a warp (pair form,
// lbm_fixed.cuh): lane h pulls the populations k = h, h + 2, h + 4, h + 6 and the force
// (adjoint source) component h, and writes its four outputs.  it2 counts half-nodes
// (node it2 / 2); every lane of the warp must call it (inactive lanes, it2 >= nitems2,
// work on node 0 and store nothing).  Nodes outside the fixed-point range take the FP64
// pipe with the pair's ten inputs gathered by shuffles (all-zero nodes map to zero).
template <int KIND, bool FIELD, bool MON>
__device__ __forceinline__ void pair_item(const double *fin, double *fout,
                                          const double *__restrict__ src2, const Grid &g,
                                          const Coef &c0, const Field &fl, long it2,
                                          long nitems2, double &mon) {
  const int h = threadIdx.x & 1;
  const bool act = it2 < nitems2;
  const long n = act ? (it2 >> 1) : 0;
  const int x = (int)(n % g.nx), y = (int)(n / g.nx);
  double in[4], out[4], m = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = h + 2 * j;
    const int dx = KIND == 0 ? -kCX[k] : kCX[k], dy = KIND == 0 ? -kCY[k] : kCY[k];
    in[j] = fin[k * g.N + wrap_idx(x, y, dx, dy, g)];
  }
  const double q = __ldg(src2 + h * g.N + n);
  const CoefFix cf = node_fix<FIELD>(c0.fx, fl, g.N, n);
  const bool ok = KIND == 0 ? collide_fix_pair<MON, true>(in, q, h, cf, out, m)
                            : collide_T_fix_pair<MON, true>(in, q, h, cf, out, m);
  if (__any_sync(0xffffffffu, !ok)) {
    double oth[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) oth[j] = __shfl_xor_sync(0xffffffffu, in[j], 1);
    const double q_o = __shfl_xor_sync(0xffffffffu, q, 1);
    if (!ok) {
      double f[8], o[8], d1 = 0.0, d2 = 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // (selects keep the arrays in registers)
        f[2 * j] = h ? oth[j] : in[j];
        f[2 * j + 1] = h ? in[j] : oth[j];
      }
      const double qx = h ? q_o : q, qy = h ? q : q_o;
      if (!zero_node(f, qx, qy, o)) {
        const Coef cc = node_coef<FIELD>(c0, fl, g.N, n, -1);
        if (KIND == 0)
          collide<false>(f, qx, qy, cc, o, d1, d2);
        else
          collide_T<false>(f, qx, qy, cc, o, d1, d2);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = h ? o[2 * j + 1] : o[2 * j];
      if (MON) m = h ? d2 : d1;
    }
  }
  if (act) {
#pragma unroll
    for (int j = 0; j < 4; ++j) fout[(h + 2 * j) * g.N + n] = out[j];
    if (MON) mon += m * m;
  }
}

// One sweep of the cluster's items (k_sweeps_cl): one node per thread, or (PAIR) one
// node per lane pair over a warp-uniform loop.
template <int KIND, bool BOUNDED, int ARITH, bool FIELD, bool MON, bool PAIR>
__device__ __forceinline__ void cluster_sweep(const double *in, double *out,
                                              const double *__restrict__ src2, const Grid &g,
                                              const Bounded &b, const Compact &c,
                                              const Coef &c0, const Field &fl,
                                              const ClusterWork &w, long t0, long T,
                                              double &mon) {
  if (PAIR) {
    const long n2 = 2 * w.nitems, lane = threadIdx.x & 31;
    for (long b0 = t0 - lane; b0 < n2; b0 += T)
      pair_item<KIND, FIELD, MON>(in, out, src2, g, c0, fl, b0 + lane, n2, mon);
    return;
  }
  for (long i = t0; i < w.nitems; i += T) {
    if (KIND == 0)
      primal_item<BOUNDED, ARITH, FIELD, MON>(in, out, src2, g, b, c, c0, fl, w, i, mon);
    else
      adjoint_item<BOUNDED, ARITH, FIELD, MON>(in, out, src2, g, b, c, c0, fl, w, i, mon);
  }
}

// `nsweeps` sweeps (KIND 0 primal, 1 adjoint) from buffer a (the state) to a or b
// (b after an odd count).  With monitor, the last sweep's partial sums of |d|^2 go to
// partial[rank] and partial[ncta .. npartial) are zeroed, so the usual finishing pass
// over npartial entries gives the monitor.  Launched as ONE cluster of gridDim.x CTAs.
// With chunk > 0 the kernel is the whole residual-rule solve loop instead: a first chunk
// of `first` sweeps, then chunks of `chunk`, each followed by the residual of its last
// two states and the cluster-wide decision (cluster_residual_stop), at most max_iters
// chunks; ls receives the chunks run and the last residual (the state ends in b after
// an odd total of sweeps, as for nsweeps).  PAIR: one node per lane pair (periodic,
// fixed point; the host launches twice the threads).
template <int KIND, bool BOUNDED, int ARITH, bool FIELD, bool PAIR>
__global__ void __launch_bounds__(256) k_sweeps_cl(double *a, double *b2,
                                                    const double *__restrict__ src2, Grid g,
                                                    Bounded b, Compact c, Coef c0, Field fl,
                                                    ClusterWork w, int nsweeps, int monitor,
                                                    double *__restrict__ partial,
                                                    long npartial, int chunk, int first,
                                                    long long max_iters, double tol,
                                                    LoopState *ls) {
  const unsigned rank = cluster_rank(), ncta = cluster_size();
  const long T = (long)ncta * blockDim.x;
  const long t0 = (long)rank * blockDim.x + threadIdx.x;
  double mon[1] = {0.0};
  if (chunk > 0) {
    __shared__ double red[2], flag[2], smx[64];
    int par = 0;  // sweeps run so far, mod 2: the latest state is in b2 when odd
    for (long long it = 0;; ++it) {
      const int len = it == 0 ? first : chunk;
      for (int s = 0; s < len; ++s) {
        const double *in = par ? b2 : a;
        double *out = par ? a : b2;
        cluster_sweep<KIND, BOUNDED, ARITH, FIELD, false, PAIR>(in, out, src2, g, b, c, c0, fl,
                                                                 w, t0, T, mon[0]);
        cluster_sync_release_acquire();
        par ^= 1;
      }
      const double *cur = par ? b2 : a, *prv = par ? a : b2;
      double v0 = 0.0, v1 = 0.0;
      for (long i = t0; i < w.nitems; i += T) {
        const long n = !BOUNDED ? i : (i < c.nb ? (long)c.bnode[i] : (long)w.inner[i - c.nb]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const double ai = cur[k * g.N + n];
          v0 = nan_max(v0, fabs(ai - prv[k * g.N + n]));
          v1 = nan_max(v1, fabs(ai));
        }
      }
      if (cluster_residual_stop(v0, v1, tol, it, max_iters, red, smx, flag)) {
        if (rank == 0 && threadIdx.x == 0) {
          ls->iters = it + 1;
          ls->metric = flag[1];
        }
        break;
      }
    }
    cluster_sync_release_acquire();  // no CTA leaves while another may read its `red`
    return;
  }
  for (int s = 0; s < nsweeps; ++s) {
    const double *in = (s & 1) ? b2 : a;
    double *out = (s & 1) ? a : b2;
    if (monitor && s == nsweeps - 1)
      cluster_sweep<KIND, BOUNDED, ARITH, FIELD, true, PAIR>(in, out, src2, g, b, c, c0, fl, w,
                                                              t0, T, mon[0]);
    else
      cluster_sweep<KIND, BOUNDED, ARITH, FIELD, false, PAIR>(in, out, src2, g, b, c, c0, fl, w,
                                                               t0, T, mon[0]);
    cluster_sync_release_acquire();
  }
  if (monitor) {
    __shared__ double sm[32];
    block_sum<1>(mon, sm);
    if (threadIdx.x == 0) partial[rank] = mon[0];
    if (rank == 0)
      for (long i = (long)ncta + threadIdx.x; i < npartial; i += blockDim.x) partial[i] = 0.0;
  }
}

// ---------------------------------------------------------------------------------
// Lattice resident in distributed shared memory (periodic lattices, uniform material).
// One cluster of C CTAs holds the whole lattice: CTA q owns rows [q h, (q + 1) h) (h =
// ny / C) in its shared memory, two population buffers (8 planes of h nx values each,
// SoA) and the node's force or adjoint source (2 planes).  A sweep reads the pulled
// populations of its own rows from its shared memory and those of the rows just above
// and below its band from the neighbouring CTA's (mapa + ld.shared::cluster), writes the
// other buffer, and ends at the cluster barrier (release / acquire), so no sweep touches
// L2.  The state is read from global memory once at the start and written back at the
// end: the final state to `a` (even count) or `b2` (odd), the one before it to the other,
// as the graph-replayed sweeps leave them.  Populations are converted on the integer
// pipes (a CTA holds few warps, and a lone warp's FP64 instruction costs 64 cycles).

// Dynamic shared memory of k_sweeps_dsm: 18 doubles per node of the band.
constexpr int kDsmDoublesPerNode = 18;

// With chunk > 0: the residual-rule solve loop as in k_sweeps_cl (a first chunk of
// `first` sweeps, then chunks of `chunk`), the residual read from the two shared-memory
// buffers.
template <int KIND, int ARITH>
__global__ void __launch_bounds__(512) k_sweeps_dsm(double *a, double *b2,
                                                     const double *__restrict__ src2, Grid g,
                                                     Coef c0, int h, int nsweeps, int monitor,
                                                     double *__restrict__ partial,
                                                     long npartial, int chunk, int first,
                                                     long long max_iters, double tol,
                                                     LoopState *ls) {
  extern __shared__ __align__(16) double dsm[];
  const unsigned rank = cluster_rank(), C = cluster_size();
  const int nx = g.nx;
  const long L = (long)h * nx;
  const long base = (long)rank * L;  // first node of the band (rows are contiguous)
  double *B0 = dsm, *B1 = dsm + 8 * L, *Q = dsm + 16 * L;
  for (long l = threadIdx.x; l < L; l += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 8; ++k) B0[k * L + l] = a[k * g.N + base + l];
    Q[l] = src2[base + l];
    Q[L + l] = src2[g.N + base + l];
  }
  const unsigned up = (rank + 1) % C, down = (rank + C - 1) % C;
  double mon[1] = {0.0};
  __shared__ double red[2], flag[2], smx[64];
  cluster_sync_release_acquire();
  long long it = 0;
  long total = 0;  // sweeps run; the latest state is in B1 when odd
  int len = chunk > 0 ? first : nsweeps;
  for (int s = 0;; ++s) {
    if (s == len) {  // end of a chunk (loop mode) or of the run
      if (chunk <= 0) break;
      const double *cur = (total & 1) ? B1 : B0, *prv = (total & 1) ? B0 : B1;
      double v0 = 0.0, v1 = 0.0;
      for (long l = threadIdx.x; l < L; l += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const double ai = cur[k * L + l];
          v0 = nan_max(v0, fabs(ai - prv[k * L + l]));
          v1 = nan_max(v1, fabs(ai));
        }
      }
      if (cluster_residual_stop(v0, v1, tol, it, max_iters, red, smx, flag)) {
        if (rank == 0 && threadIdx.x == 0) {
          ls->iters = it + 1;
          ls->metric = flag[1];
        }
        break;
      }
      ++it;
      s = 0;
      len = chunk;
    }
    const double *S = (total & 1) ? B1 : B0;
    double *D = (total & 1) ? B0 : B1;
    const unsigned Sa = smem_addr(S);
    const bool last_mon = chunk <= 0 && monitor && s == nsweeps - 1;
    for (long l = threadIdx.x; l < L; l += blockDim.x) {
      const int x = (int)(l % nx), yl = (int)(l / nx);
      // source of link k: primal pulls from x - c_k, the adjoint from x + c_k; rows
      // outside the band belong to the neighbouring CTA (|c_y| <= 1)
      const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
      double f[8], o[8], m1 = 0.0, m2 = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int dx = KIND == 0 ? -kCX[k] : kCX[k], dy = KIND == 0 ? -kCY[k] : kCY[k];
        const int sx = dx < 0 ? xm : (dx > 0 ? xp : x);
        const int sy = yl + dy;
        if (sy >= 0 && sy < h) {
          f[k] = S[k * L + (long)sy * nx + sx];
        } else {
          const long off = k * L + (long)(sy < 0 ? h - 1 : 0) * nx + sx;
          f[k] = ld_cluster(Sa + (unsigned)(off * 8), sy < 0 ? down : up);
        }
      }
      const double qx = Q[l], qy = Q[L + l];
      if (KIND == 0) {
        if (last_mon) {
          if (ARITH == 0 || !collide_fix<true, false, true, true>(f, qx, qy, c0.fx, o, m1, m2))
            collide<false>(f, qx, qy, c0, o, m1, m2);
        } else if (ARITH == 0 || !collide_fix<false, false, true, true>(f, qx, qy, c0.fx, o, m1, m2)) {
          collide<false>(f, qx, qy, c0, o, m1, m2);
        }
      } else {
        if (last_mon) {
          if (ARITH == 0 || !collide_T_fix<true, false, false, true, true>(f, qx, qy, c0.fx, o, m1, m2))
            collide_T<false>(f, qx, qy, c0, o, m1, m2);
        } else if (ARITH == 0 ||
                   !collide_T_fix<false, false, false, true, true>(f, qx, qy, c0.fx, o, m1, m2)) {
          collide_T<false>(f, qx, qy, c0, o, m1, m2);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) D[k * L + l] = o[k];
      if (last_mon) mon[0] += m1 * m1 + m2 * m2;
    }
    cluster_sync_release_acquire();
    ++total;
  }
  if (total > 0) {
    const bool odd = total & 1;
    const double *fin = odd ? B1 : B0, *prev = odd ? B0 : B1;
    double *gfin = odd ? b2 : a, *gprev = odd ? a : b2;
    for (long l = threadIdx.x; l < L; l += blockDim.x) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        gfin[k * g.N + base + l] = fin[k * L + l];
        gprev[k * g.N + base + l] = prev[k * L + l];
      }
    }
  }
  if (chunk > 0) cluster_sync_release_acquire();  // no CTA leaves while another reads `red`
  if (monitor) {
    __shared__ double sm[32];
    block_sum<1>(mon, sm);
    if (threadIdx.x == 0) partial[rank] = mon[0];
    if (rank == 0)
      for (long i = (long)C + threadIdx.x; i < npartial; i += blockDim.x) partial[i] = 0.0;
  }
}

// The decision at the end of a chunk, from the reduced residual partials (max |a - b|,
// max |a|): the same relative residual as the host loop computes, stop (condition 0)
// when it is below tol, not finite, or the chunk limit is reached.
static __global__ void k_loop_decide(const double *__restrict__ dres, LoopState *ls,
                                     cudaGraphConditionalHandle hnd) {
  const double a = dres[0], b = dres[1];
  double r = b > 0.0 ? a / b : (a > 0.0 ? INFINITY : 0.0);
  if (!isfinite(a) || !isfinite(b)) r = NAN;
  const long long it = ls->iters + 1;
  ls->iters = it;
  ls->metric = r;
  const bool stop = !(r >= ls->tol) || it >= ls->max_iters;
  cudaGraphSetConditional(hnd, stop ? 0u : 1u);
}

// Residual partials: max |a - b| and max |a| over all planes.
static __global__ void __launch_bounds__(256) k_residual(const double *__restrict__ a,
                                                  const double *__restrict__ bb, long total,
                                                  double *__restrict__ partial) {
  double v[2] = {0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const double ai = a[i];
    v[0] = nan_max(v[0], fabs(ai - bb[i]));
    v[1] = nan_max(v[1], fabs(ai));
  }
  __shared__ double sm[64];
  block_max<2>(v, sm);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 2 + 0] = v[0];
    partial[blockIdx.x * 2 + 1] = v[1];
  }
}

// Second pass: out[v] = reduce over nb partials (fixed order, one block).  op 0 sum, 1 max.
static __global__ void __launch_bounds__(256) k_finish(const double *__restrict__ partial, long nb,
                                                int nv, int op, double scale,
                                                double *__restrict__ out) {
  __shared__ double sm[32 * 4];
  for (int v = 0; v < nv; ++v) {
    double acc[1] = {0.0};
    for (long i = threadIdx.x; i < nb; i += blockDim.x) {
      const double t = partial[i * nv + v];
      acc[0] = op == 0 ? acc[0] + t : nan_max(acc[0], t);
    }
    if (op == 0)
      block_sum<1>(acc, sm);
    else
      block_max<1>(acc, sm);
    if (threadIdx.x == 0) out[v] = acc[0] * scale;
    __syncthreads();
  }
}

// Quarter lattice force q = g / 4 = dx^2 (a1 Phi_1 + a2 Phi_2) / 4 from the two basis
// fields, or q = dx^2 F / 4 from a nodal force (alpha == nullptr).
static __global__ void k_set_force(double *__restrict__ g2, const double *__restrict__ src,
                            const double *__restrict__ basis, const double *__restrict__ alpha2,
                            double dx2, long N, const uint8_t *__restrict__ type) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 2 * N;
       i += (long)gridDim.x * blockDim.x) {
    double v;
    if (alpha2)
      v = alpha2[0] * basis[i] + alpha2[1] * basis[2 * N + i];
    else
      v = src ? src[i] : 0.0;
    const long n = i < N ? i : i - N;
    if (type && type[n] == 0) v = 0.0;
    g2[i] = dx2 * v;
  }
}

// Cbar partial sums: sum_n obs |d*_n|^2 (times dx^2 outside).
template <bool BOUNDED>
__global__ void __launch_bounds__(256) k_cbar(const double *__restrict__ dstar,
                                              const double *__restrict__ obs, Grid g, Bounded b,
                                              double *__restrict__ partial) {
  double acc[1] = {0.0};
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < g.N;
       n += (long)gridDim.x * blockDim.x) {
    if (BOUNDED && b.type[n] == 0) continue;
    const double w = obs ? obs[n] : 1.0;
    acc[0] += w * (dstar[n] * dstar[n] + dstar[g.N + n] * dstar[g.N + n]);
  }
  __shared__ double sm[32];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc[0];
}

}  // namespace lbm
