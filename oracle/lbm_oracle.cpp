// CPU reference ("oracle") for the solid LBM of arXiv 2609.31347 -- TEST
// INFRASTRUCTURE ONLY (see lbm_oracle.h).  Plain FP64, step by step in the order
// of the paper; nothing here is blocked, fused or reordered for speed.
//
// Threads: loops whose iterations each write their own node (collision, gather
// streaming, per-node setup) carry one OpenMP "parallel for"; every iteration does the
// same arithmetic as in a serial run, so results do not depend on the thread count.
// Sums (objective, Cbar, monitor) and the scatter of the transposed streaming on
// bounded grids stay serial.
#include "lbm_oracle.h"

#include <omp.h>

#include <cmath>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual number for f-AD (Section 3.3.1, Eq. fAD).
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual &operator+=(Dual &a, Dual b) { a = a + b; return a; }
inline double value(double a) { return a; }
inline double value(Dual a) { return a.v; }
inline double tangent(double) { return 0.0; }
inline double tangent(Dual a) { return a.d; }

// ---------------------------------------------------------------------------
// D2Q8 stencil, ordered set Q of Eq. (direction_order): no rest population.
const int CX[8] = {1, 0, -1, 0, 1, -1, -1, 1};
const int CY[8] = {0, 1, 0, -1, 1, 1, -1, -1};
const double THETA = 1.0 / 3.0;  // theta of Eq. (gamma) and Eq. (moments_eq)

int opposite(int k) {
  for (int j = 0; j < 8; ++j)
    if (CX[j] == -CX[k] && CY[j] == -CY[k]) return j;
  return -1;
}

// Moment matrix rows: m10, m01, m11, m_s = m20+m02, m_d = m20-m02, m12, m21,
// m_f = m22 + gamma m_s (Eqs. moments, moment_s, moment_d, moment_f), built from the
// raw-moment definition m_ab = sum_k i_k^a j_k^b f_k.
template <class T>
void build_M(T gamma, T M[64]) {
  for (int k = 0; k < 8; ++k) {
    const double i = CX[k], j = CY[k];
    M[0 * 8 + k] = T(i);
    M[1 * 8 + k] = T(j);
    M[2 * 8 + k] = T(i * j);
    M[3 * 8 + k] = T(i * i + j * j);
    M[4 * 8 + k] = T(i * i - j * j);
    M[5 * 8 + k] = T(i * j * j);
    M[6 * 8 + k] = T(i * i * j);
    M[7 * 8 + k] = T(i * i * j * j) + gamma * T(i * i + j * j);
  }
}

// Gauss-Jordan inverse with partial pivoting (pivot chosen on the value part).
template <class T>
bool invert8(const T A_in[64], T Ainv[64]) {
  T A[64];
  for (int i = 0; i < 64; ++i) { A[i] = A_in[i]; Ainv[i] = T(0.0); }
  for (int i = 0; i < 8; ++i) Ainv[i * 8 + i] = T(1.0);
  for (int c = 0; c < 8; ++c) {
    int p = c;
    for (int r = c + 1; r < 8; ++r)
      if (std::fabs(value(A[r * 8 + c])) > std::fabs(value(A[p * 8 + c]))) p = r;
    if (std::fabs(value(A[p * 8 + c])) < 1e-300) return false;
    if (p != c)
      for (int j = 0; j < 8; ++j) {
        T t = A[c * 8 + j]; A[c * 8 + j] = A[p * 8 + j]; A[p * 8 + j] = t;
        t = Ainv[c * 8 + j]; Ainv[c * 8 + j] = Ainv[p * 8 + j]; Ainv[p * 8 + j] = t;
      }
    T piv = A[c * 8 + c];
    for (int j = 0; j < 8; ++j) { A[c * 8 + j] = A[c * 8 + j] / piv; Ainv[c * 8 + j] = Ainv[c * 8 + j] / piv; }
    for (int r = 0; r < 8; ++r) {
      if (r == c) continue;
      T fct = A[r * 8 + c];
      for (int j = 0; j < 8; ++j) {
        A[r * 8 + j] = A[r * 8 + j] - fct * A[c * 8 + j];
        Ainv[r * 8 + j] = Ainv[r * 8 + j] - fct * Ainv[c * 8 + j];
      }
    }
  }
  return true;
}

template <class T>
void matvec8(const T A[64], const T x[8], T y[8]) {
  for (int r = 0; r < 8; ++r) {
    T s(0.0);
    for (int c = 0; c < 8; ++c) s += A[r * 8 + c] * x[c];
    y[r] = s;
  }
}

// Material map (Eqs. lambda, mu, K) and relaxation times (Table A.1, Eq. relaxation).
template <class T>
struct Material {
  T omega[6];  // beta = 11, s, d, 12, 21, f  (moment indices 2..7)
  T gamma_b;   // gamma of Eq. (gamma) with tau_f = 1/2, used at boundary nodes
  T K;         // 2D bulk modulus (Eq. K), lattice units = physical units (dt = dx^2)
};

template <class T>
bool material(T E, double nu, Material<T> &m) {
  if (!(value(E) > 0.0) || !(nu > -1.0 && nu < 1.0)) return false;
  const T mu = E / T(2.0 * (1.0 + nu));
  const T lam = E * T(nu) / T(1.0 - nu * nu);
  const T K = mu + lam;
  m.K = K;
  const T tau[6] = {mu / T(THETA), T(2.0) * K / T(1.0 + THETA), T(2.0) * mu / T(1.0 - THETA),
                    T(0.5), T(0.5), T(0.5)};
  for (int b = 0; b < 6; ++b) m.omega[b] = T(1.0) / (tau[b] + T(0.5));
  const T tau_s = tau[1], tau_f = T(0.5);
  if (std::fabs(value(tau_s) - value(tau_f)) < 1e-14) return false;
  m.gamma_b = T(THETA) * tau_f / (T(1.0 + THETA) * (tau_s - tau_f));
  return true;
}

// One local collision C_n[f_S, g] (Eq. local_collide): moments, half force,
// equilibrium, relaxation, second half force, back to populations.
template <class T>
void collide(const T fS[8], T gx, T gy, const Material<T> &mat, const T M[64],
             const T Minv[64], T fC[8]) {
  T m[8];
  matvec8(M, fS, m);
  const T b10 = m[0] + gx * T(0.5);  // Eq. moments_bar_1
  const T b01 = m[1] + gy * T(0.5);  // Eq. moments_bar_2
  // m^eq = N (b10, b01), N^T rows (1,0,0,0,0,theta,0,0), (0,1,0,0,0,0,theta,0)
  const T meq[8] = {b10, b01, T(0.0), T(0.0), T(0.0), T(THETA) * b10, T(THETA) * b01, T(0.0)};
  T mc[8];
  mc[0] = b10 + gx * T(0.5);  // Eq. moments_c_10
  mc[1] = b01 + gy * T(0.5);  // Eq. moments_c_01
  for (int b = 2; b < 8; ++b) mc[b] = m[b] + mat.omega[b - 2] * (meq[b] - m[b]);  // Eq. moments_c
  matvec8(Minv, mc, fC);
}

// ---------------------------------------------------------------------------
// Lattice bookkeeping.
struct Lat {
  int nx, ny, N;
  bool periodic;
  double dx, nu;
  std::vector<unsigned char> type;  // 0 outside, 1 interior, 2 boundary
  std::vector<unsigned char> link;  // [k*N+n]
  const double *wall_d, *wall_T, *wall_n;
  long n_active;
};

bool make_lat(const orc_grid *g, Lat &L) {
  if (!g || g->nx < 1 || g->ny < 1 || !(g->dx > 0.0)) return false;
  L.nx = g->nx; L.ny = g->ny; L.N = g->nx * g->ny;
  L.periodic = g->periodic != 0;
  L.dx = g->dx; L.nu = g->nu;
  L.type.assign(L.N, 1);
  L.link.assign(8 * (size_t)L.N, 0);
  if (g->node_type) std::memcpy(L.type.data(), g->node_type, L.N);
  if (g->link) std::memcpy(L.link.data(), g->link, 8 * (size_t)L.N);
  L.wall_d = g->wall_d; L.wall_T = g->wall_T; L.wall_n = g->wall_n;
  L.n_active = 0;
  for (int n = 0; n < L.N; ++n) L.n_active += L.type[n] != 0;
  if (L.periodic) {
    for (int n = 0; n < L.N; ++n)
      if (L.type[n] != 1) return false;
    for (size_t i = 0; i < L.link.size(); ++i)
      if (L.link[i] != 0) return false;
  } else {
    // every missing link must carry a rule, and its data must be present
    for (int n = 0; n < L.N; ++n) {
      if (!L.type[n]) continue;
      const int x = n % L.nx, y = n / L.nx;
      for (int k = 0; k < 8; ++k) {
        const int xs = x - CX[k], ys = y - CY[k];
        const bool inside = xs >= 0 && xs < L.nx && ys >= 0 && ys < L.ny && L.type[ys * L.nx + xs];
        const unsigned char lk = L.link[(size_t)k * L.N + n];
        if (inside && lk != 0) return false;
        if (!inside && lk == 0) return false;
        if (lk == 1 && !L.wall_d) return false;
        if (lk == 2 && (!L.wall_T || !L.wall_n)) return false;
      }
    }
  }
  return true;
}

// Per-node collision data: material, M and M^-1 (gamma-modified at boundary nodes,
// Appendix A.1), lattice force g = dx^2 F (forcing term with Delta t = dx^2).
template <class T>
struct NodeOps {
  std::vector<Material<T>> mat;
  std::vector<T> M, Minv;  // 64 per node
  std::vector<T> gx, gy;
};

template <class T>
bool make_ops(const Lat &L, const T *E, const T *Fx, const T *Fy, NodeOps<T> &ops) {
  ops.mat.resize(L.N);
  ops.M.assign(64 * (size_t)L.N, T(0.0));
  ops.Minv.assign(64 * (size_t)L.N, T(0.0));
  ops.gx.assign(L.N, T(0.0));
  ops.gy.assign(L.N, T(0.0));
  const double dx2 = L.dx * L.dx;
  int bad = 0;
#pragma omp parallel for reduction(| : bad)
  for (int n = 0; n < L.N; ++n) {
    if (!L.type[n]) continue;
    if (!material(E[n], L.nu, ops.mat[n])) { bad |= 1; continue; }
    const T gamma = (L.type[n] == 2) ? ops.mat[n].gamma_b : T(0.0);  // gamma = 0 in the bulk
    build_M(gamma, &ops.M[64 * (size_t)n]);
    if (!invert8(&ops.M[64 * (size_t)n], &ops.Minv[64 * (size_t)n])) { bad |= 1; continue; }
    ops.gx[n] = T(dx2) * Fx[n];
    ops.gy[n] = T(dx2) * Fy[n];
  }
  return bad == 0;
}

// ---------------------------------------------------------------------------
// Streaming S' (Eq. local_stream) with the bounded-domain rules written as a
// sparse affine map: f_S[dst] = sum_t coef_t f_C[src_t] + cst.
//  regular link        f_S,k(x) = f_C,k(x - c_k)              (periodic: index wrap)
//  Dirichlet-missing   f_S,k(x) = f_C,kbar(x) + 2 f^eq_k(d_D)   (bounce-back + source)
//  Neumann-missing     f_S,k(x) = -f_C,kbar(x) + 2 p_k           (anti-bounce-back)
// with f^eq = M0^-1 N d_D and p = M0^-1 mbar_w, mbar_w the bared even moments of the
// wall stress sigma_w: its traction sigma_w n equals T and its tangential part is
// the node's own bared stress, recovered from the node's post-collision moments
// (mbar = m^C (2 - omega) / (2 (1 - omega)) for the relaxed moments 11, s, d).
template <class T>
struct Rule {
  int nterm;
  long src[9];
  T coef[9];
  T cst;
};

// Wall-stress even populations p (8) for a Neumann node, given its post-collision
// populations fCn and traction (Tx, Ty); affine in (fCn, T).
template <class T>
void neumann_p(const T fCn[8], T Tx, T Ty, double nx_, double ny_, const Material<T> &mat,
               double dx, T p[8]) {
  T M0[64], M0inv[64];
  build_M(T(0.0), M0);
  invert8(M0, M0inv);
  T mC[8];
  matvec8(M0, fCn, mC);
  auto bared = [](T mc, T w) { return mc * (T(2.0) - w) / (T(2.0) * (T(1.0) - w)); };
  const T b11 = bared(mC[2], mat.omega[0]);
  const T bs = bared(mC[3], mat.omega[1]);
  const T bd = bared(mC[4], mat.omega[2]);
  // node stress, physical units: sigma = -mbar_2 / dx (Eq. stress_from_moments)
  const T s11 = -(bs + bd) * T(0.5 / dx);
  const T s22 = -(bs - bd) * T(0.5 / dx);
  const T s12 = -b11 * T(1.0 / dx);
  const T nxT(nx_), nyT(ny_);
  const T rx = Tx - (s11 * nxT + s12 * nyT);  // traction defect r = T - sigma n
  const T ry = Ty - (s12 * nxT + s22 * nyT);
  const T rn = rx * nxT + ry * nyT;
  // sigma_w = sigma + r n^T + n r^T - (r.n) n n^T
  const T w11 = s11 + T(2.0) * rx * nxT - rn * nxT * nxT;
  const T w22 = s22 + T(2.0) * ry * nyT - rn * nyT * nyT;
  const T w12 = s12 + rx * nyT + ry * nxT - rn * nxT * nyT;
  T mw[8];
  for (int i = 0; i < 8; ++i) mw[i] = T(0.0);
  mw[2] = -T(dx) * w12;
  mw[3] = -T(dx) * (w11 + w22);
  mw[4] = -T(dx) * (w11 - w22);
  // bared m22 of the wall state: pre-collision m22 = -theta dx div(d) to first order
  // (streaming of m12^C = theta d, m21^C = theta d_y), post-collision m22 = 0, and
  // div(d) = tr(sigma) / (2K) (trace of Eq. stress).
  mw[7] = -T(THETA * dx) * (w11 + w22) / (T(4.0) * mat.K);
  matvec8(M0inv, mw, p);
}

template <class T>
bool make_rules(const Lat &L, const NodeOps<T> &ops, std::vector<Rule<T>> &rules) {
  const int N = L.N;
  rules.assign(8 * (size_t)N, Rule<T>());
  T M0[64], M0inv[64];
  build_M(T(0.0), M0);
  invert8(M0, M0inv);
  int bad = 0;
#pragma omp parallel for reduction(| : bad)
  for (int n = 0; n < N; ++n) {
    const int x = n % L.nx, y = n / L.nx;
    for (int k = 0; k < 8; ++k) {
      Rule<T> &r = rules[(size_t)k * N + n];
      r.nterm = 0;
      r.cst = T(0.0);
      if (!L.type[n]) continue;
      const unsigned char lk = L.link[(size_t)k * N + n];
      const int kb = opposite(k);
      if (lk == 0) {
        int xs = x - CX[k], ys = y - CY[k];
        if (L.periodic) { xs = (xs + L.nx) % L.nx; ys = (ys + L.ny) % L.ny; }
        r.nterm = 1;
        r.src[0] = (long)k * N + (long)ys * L.nx + xs;
        r.coef[0] = T(1.0);
      } else if (lk == 1) {
        const T dD[8] = {T(L.wall_d[n]), T(L.wall_d[N + n]), T(0.0), T(0.0), T(0.0),
                         T(THETA) * T(L.wall_d[n]), T(THETA) * T(L.wall_d[N + n]), T(0.0)};
        T feq[8];
        matvec8(M0inv, dD, feq);
        r.nterm = 1;
        r.src[0] = (long)kb * N + n;
        r.coef[0] = T(1.0);
        r.cst = T(2.0) * feq[k];
      } else if (lk == 2) {
        const double nxv = L.wall_n[n], nyv = L.wall_n[N + n];
        // constant part: p(f_C = 0, T)
        T zero[8], p[8];
        for (int j = 0; j < 8; ++j) zero[j] = T(0.0);
        neumann_p(zero, T(L.wall_T[n]), T(L.wall_T[N + n]), nxv, nyv, ops.mat[n], L.dx, p);
        r.cst = T(2.0) * p[k];
        // linear part: -f_C,kbar(x) + 2 dp_k/df_C,j(x) f_C,j(x)
        r.nterm = 8;
        for (int j = 0; j < 8; ++j) {
          T e[8];
          for (int i = 0; i < 8; ++i) e[i] = T(i == j ? 1.0 : 0.0);
          neumann_p(e, T(0.0), T(0.0), nxv, nyv, ops.mat[n], L.dx, p);
          r.src[j] = (long)j * N + n;
          r.coef[j] = T(2.0) * p[k] + T(j == kb ? -1.0 : 0.0);
        }
      } else {
        bad |= 1;
      }
    }
  }
  return bad == 0;
}

template <class T>
void stream(const Lat &L, const std::vector<Rule<T>> &rules, const std::vector<T> &fC,
            std::vector<T> &fS, bool with_sources) {
  const long nd = (long)rules.size();
#pragma omp parallel for
  for (long d = 0; d < nd; ++d) {
    const Rule<T> &r = rules[d];
    T s = with_sources ? r.cst : T(0.0);
    for (int t = 0; t < r.nterm; ++t) s += r.coef[t] * fC[r.src[t]];
    fS[d] = s;
  }
  (void)L;
}

// Transposed streaming phi_S = S'^T phi_C (Eq. adjoint_streaming, S^-1 = S^T).  On a
// periodic lattice every rule is one term and the sources form a permutation, so the
// scatter writes each entry once and runs in parallel; the boundary rules of a bounded
// lattice add several terms into the same entries, so there it stays serial.
void stream_T(const Lat &L, const std::vector<Rule<double>> &rules,
              const std::vector<double> &phiC, std::vector<double> &phiS) {
  std::fill(phiS.begin(), phiS.end(), 0.0);
  const long nd = (long)rules.size();
  if (L.periodic) {
#pragma omp parallel for
    for (long d = 0; d < nd; ++d) {
      const Rule<double> &r = rules[d];
      for (int t = 0; t < r.nterm; ++t) phiS[r.src[t]] += r.coef[t] * phiC[d];
    }
    return;
  }
  for (long d = 0; d < nd; ++d) {
    const Rule<double> &r = rules[d];
    for (int t = 0; t < r.nterm; ++t) phiS[r.src[t]] += r.coef[t] * phiC[d];
  }
}

template <class T>
void collide_all(const Lat &L, const NodeOps<T> &ops, const std::vector<T> &fS,
                 std::vector<T> &fC, bool with_force) {
  const int N = L.N;
#pragma omp parallel for
  for (int n = 0; n < N; ++n) {
    if (!L.type[n]) {
      for (int k = 0; k < 8; ++k) fC[(size_t)k * N + n] = T(0.0);
      continue;
    }
    T f[8], c[8];
    for (int k = 0; k < 8; ++k) f[k] = fS[(size_t)k * N + n];
    collide(f, with_force ? ops.gx[n] : T(0.0), with_force ? ops.gy[n] : T(0.0), ops.mat[n],
            &ops.M[64 * (size_t)n], &ops.Minv[64 * (size_t)n], c);
    for (int k = 0; k < 8; ++k) fC[(size_t)k * N + n] = c[k];
  }
}

// c of Eq. (convergence) for a displacement field given per node by disp(n, dx_, dy_):
// the mean of |d_n|^2 over the active nodes.
template <class Disp>
double mean_sq_disp(const Lat &L, Disp disp) {
  double s = 0.0;
  for (int n = 0; n < L.N; ++n) {
    if (!L.type[n]) continue;
    double a, b;
    disp(n, a, b);
    s += a * a + b * b;
  }
  return L.n_active ? s / (double)L.n_active : 0.0;
}

template <class T>
void node_disp(const Lat &L, const std::vector<T> &fS, int n, T gx, T gy, T &dx_, T &dy_);

// trace (optional, steps + 1 values): c(t) of f_S(t) for t = 0 .. steps.
template <class T>
int run_primal(const Lat &L, const T *E, const T *Fx, const T *Fy, const double *fS0,
               long steps, std::vector<T> &fS, std::vector<T> &fC, double *trace = nullptr) {
  NodeOps<T> ops;
  if (!make_ops(L, E, Fx, Fy, ops)) return -2;
  std::vector<Rule<T>> rules;
  if (!make_rules(L, ops, rules)) return -3;
  const size_t P = 8 * (size_t)L.N;
  fS.assign(P, T(0.0));
  fC.assign(P, T(0.0));
  if (fS0)
    for (size_t i = 0; i < P; ++i) fS[i] = T(fS0[i]);
  auto c_of_state = [&]() {
    return mean_sq_disp(L, [&](int n, double &a, double &b) {
      T ta, tb;
      node_disp(L, fS, n, ops.gx[n], ops.gy[n], ta, tb);
      a = value(ta);
      b = value(tb);
    });
  };
  if (trace) trace[0] = c_of_state();
  for (long t = 0; t < steps; ++t) {
    collide_all(L, ops, fS, fC, true);  // f_C(t) = C[f_S(t), F]
    stream(L, rules, fC, fS, true);     // f_S(t+1) = S' f_C(t)
    if (trace) trace[t + 1] = c_of_state();
  }
  return 0;
}

// d of one node from f_S (Eq. disp_from_moments with Eq. moments_bar_1/2).
template <class T>
void node_disp(const Lat &L, const std::vector<T> &fS, int n, T gx, T gy, T &dx_, T &dy_) {
  T m10(0.0), m01(0.0);
  for (int k = 0; k < 8; ++k) {
    m10 += T((double)CX[k]) * fS[(size_t)k * L.N + n];
    m01 += T((double)CY[k]) * fS[(size_t)k * L.N + n];
  }
  dx_ = m10 + gx * T(0.5);
  dy_ = m01 + gy * T(0.5);
}

double cbar_of(const Lat &L, const double *dstar, const double *obs) {
  double C = 0.0;
  for (int n = 0; n < L.N; ++n) {
    if (!L.type[n]) continue;
    const double w = obs ? obs[n] : 1.0;
    C += w * (dstar[n] * dstar[n] + dstar[L.N + n] * dstar[L.N + n]) * L.dx * L.dx;
  }
  return C;
}

template <class T>
T objective_of(const Lat &L, const std::vector<T> &fS, const T *Fx, const T *Fy,
               const double *dstar, const double *obs, double Cbar) {
  T J(0.0);
  const double dx2 = L.dx * L.dx;
  for (int n = 0; n < L.N; ++n) {
    if (!L.type[n]) continue;
    const double w = obs ? obs[n] : 1.0;
    if (w == 0.0) continue;
    T dxn, dyn;
    node_disp(L, fS, n, T(dx2) * Fx[n], T(dx2) * Fy[n], dxn, dyn);
    const T ex = dxn - T(dstar[n]), ey = dyn - T(dstar[L.N + n]);
    J += T(0.5 * w * dx2 / Cbar) * (ex * ex + ey * ey);  // Eqs. node_J, discrete_J
  }
  return J;
}

// Jacobian of one node's collision w.r.t. its populations, column j = C(e_j, g=0):
// the collision is affine in f_S, so this is exact.
void collision_jacobian(const NodeOps<double> &ops, int n, double A[64]) {
  for (int j = 0; j < 8; ++j) {
    double e[8] = {0, 0, 0, 0, 0, 0, 0, 0}, c[8];
    e[j] = 1.0;
    collide(e, 0.0, 0.0, ops.mat[n], &ops.M[64 * (size_t)n], &ops.Minv[64 * (size_t)n], c);
    for (int r = 0; r < 8; ++r) A[r * 8 + j] = c[r];
  }
}

// Algorithm 1.  trace (optional, steps + 1 values): c of Eq. (convergence) for the
// adjoint displacement d^phi_n = (sum_k c_kx phi_S,k, sum_k c_ky phi_S,k) of
// phi_S(i) = S'^T phi_C(i), i = 0 .. steps.
int run_adjoint(const orc_grid *g, const double *E_node, const double *F, const double *fS,
                const double *dstar, const double *obs, long steps, double *phiC_out,
                double *phiS_out, double *trace) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !F || !fS || !dstar || !phiC_out || !phiS_out || steps < 0)
    return -1;
  const int N = L.N;
  const size_t P = 8 * (size_t)N;
  NodeOps<double> ops;
  if (!make_ops(L, E_node, F, F + N, ops)) return -2;
  std::vector<Rule<double>> rules;
  if (!make_rules(L, ops, rules)) return -3;
  const double C = cbar_of(L, dstar, obs);
  if (!(C > 0.0)) return -4;
  // constant terms of Algorithm 1: A_n = dC_n/df and j = (dJ/df_S)^T at f_S
  std::vector<double> A(64 * (size_t)N, 0.0), j(P, 0.0);
  std::vector<double> f(fS, fS + P);
  const double dx2 = L.dx * L.dx;
#pragma omp parallel for
  for (int n = 0; n < N; ++n) {
    if (!L.type[n]) continue;
    collision_jacobian(ops, n, &A[64 * (size_t)n]);
    const double w = obs ? obs[n] : 1.0;
    double dxn, dyn;
    node_disp(L, f, n, ops.gx[n], ops.gy[n], dxn, dyn);
    const double rx = w * dx2 / C * (dxn - dstar[n]);
    const double ry = w * dx2 / C * (dyn - dstar[N + n]);
    const double *M = &ops.M[64 * (size_t)n];
    for (int k = 0; k < 8; ++k) j[(size_t)k * N + n] = rx * M[0 * 8 + k] + ry * M[1 * 8 + k];
  }
  std::vector<double> phiC(P, 0.0), phiS(P, 0.0);  // Eq. adjoint_init
  auto c_of_phiS = [&]() {
    return mean_sq_disp(L, [&](int n, double &a, double &b) {
      a = b = 0.0;
      for (int k = 0; k < 8; ++k) {
        a += CX[k] * phiS[(size_t)k * N + n];
        b += CY[k] * phiS[(size_t)k * N + n];
      }
    });
  };
  for (long it = 0; it < steps; ++it) {
    stream_T(L, rules, phiC, phiS);  // Eq. adjoint_streaming
    if (trace) trace[it] = c_of_phiS();
#pragma omp parallel for
    for (int n = 0; n < N; ++n) {  // Eq. adjoint_collision
      if (!L.type[n]) continue;
      const double *An = &A[64 * (size_t)n];
      for (int c = 0; c < 8; ++c) {
        double s = 0.0;
        for (int r = 0; r < 8; ++r) s += An[r * 8 + c] * phiS[(size_t)r * N + n];
        phiC[(size_t)c * N + n] = s - j[(size_t)c * N + n];
      }
    }
  }
  stream_T(L, rules, phiC, phiS);  // phi_S^inf = S^-1 phi_C^inf
  if (trace) trace[steps] = c_of_phiS();
  std::memcpy(phiC_out, phiC.data(), sizeof(double) * P);
  std::memcpy(phiS_out, phiS.data(), sizeof(double) * P);
  return 0;
}

}  // namespace

// ===========================================================================
extern "C" {

int orc_moment_matrix(double gamma, double *M, double *Minv) {
  if (!M || !Minv) return -1;
  build_M(gamma, M);
  return invert8(M, Minv) ? 0 : -1;
}

int orc_material(double E, double nu, double *omega6, double *gamma_b) {
  Material<double> m;
  if (!material(E, nu, m)) return -1;
  if (omega6)
    for (int b = 0; b < 6; ++b) omega6[b] = m.omega[b];
  if (gamma_b) *gamma_b = m.gamma_b;
  return 0;
}

int orc_collide(double E, double nu, int boundary_node, const double *fS8, double gx,
                double gy, double *fC8) {
  Material<double> m;
  if (!fS8 || !fC8 || !material(E, nu, m)) return -1;
  double M[64], Minv[64];
  build_M(boundary_node ? m.gamma_b : 0.0, M);
  if (!invert8(M, Minv)) return -1;
  collide(fS8, gx, gy, m, M, Minv, fC8);
  return 0;
}

int orc_primal(const orc_grid *g, const double *E_node, const double *F, const double *fS0,
               long steps, double *fS_out, double *fC_out) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !F || !fS_out || steps < 0) return -1;
  std::vector<double> fS, fC;
  const int rc = run_primal<double>(L, E_node, F, F + L.N, fS0, steps, fS, fC);
  if (rc) return rc;
  std::memcpy(fS_out, fS.data(), sizeof(double) * fS.size());
  if (fC_out) std::memcpy(fC_out, fC.data(), sizeof(double) * fC.size());
  return 0;
}

int orc_primal_trace(const orc_grid *g, const double *E_node, const double *F, long steps,
                     double *c_out) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !F || !c_out || steps < 0) return -1;
  std::vector<double> fS, fC;
  return run_primal<double>(L, E_node, F, F + L.N, nullptr, steps, fS, fC, c_out);
}

long orc_cv_stop(const double *c, long n, long window, double tol, double *metric) {
  if (!c || n < 0 || window < 2) return -2;
  for (long i = window - 1; i < n; ++i) {
    // the trailing window c[i - window + 1 .. i] (Eq. convergence_crit)
    double mean = 0.0;
    for (long j = i - window + 1; j <= i; ++j) mean += c[j];
    mean /= (double)window;
    double var = 0.0;
    for (long j = i - window + 1; j <= i; ++j) var += (c[j] - mean) * (c[j] - mean);
    const double sd = std::sqrt(var / (double)window);
    const double cv = mean > 0.0 ? sd / mean : (sd == 0.0 ? 0.0 : INFINITY);
    if (metric) *metric = cv;
    if (cv < tol) return i;
  }
  return -1;
}

int orc_set_threads(int n) {
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
  return omp_get_max_threads();
}

int orc_threads(void) { return omp_get_max_threads(); }

int orc_primal_tangent(const orc_grid *g, const double *E_node, const double *Edot,
                       const double *F, const double *Fdot, long steps, double *fS_out,
                       double *fSdot_out) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !F || !fS_out || !fSdot_out || steps < 0) return -1;
  std::vector<Dual> E(L.N), Fx(L.N), Fy(L.N);
  for (int n = 0; n < L.N; ++n) {
    E[n] = Dual(E_node[n], Edot ? Edot[n] : 0.0);
    Fx[n] = Dual(F[n], Fdot ? Fdot[n] : 0.0);
    Fy[n] = Dual(F[L.N + n], Fdot ? Fdot[L.N + n] : 0.0);
  }
  std::vector<Dual> fS, fC;
  const int rc = run_primal<Dual>(L, E.data(), Fx.data(), Fy.data(), nullptr, steps, fS, fC);
  if (rc) return rc;
  for (size_t i = 0; i < fS.size(); ++i) { fS_out[i] = fS[i].v; fSdot_out[i] = fS[i].d; }
  return 0;
}

int orc_objective(const orc_grid *g, const double *fS, const double *F, const double *dstar,
                  const double *obs, double *J, double *Cbar) {
  Lat L;
  if (!make_lat(g, L) || !fS || !F || !dstar || !J) return -1;
  const double C = cbar_of(L, dstar, obs);
  if (!(C > 0.0)) return -2;
  std::vector<double> f(fS, fS + 8 * (size_t)L.N);
  *J = objective_of<double>(L, f, F, F + L.N, dstar, obs, C);
  if (Cbar) *Cbar = C;
  return 0;
}

int orc_objective_tangent(const orc_grid *g, const double *fS, const double *fSdot,
                          const double *F, const double *Fdot, const double *dstar,
                          const double *obs, double *J, double *Jdot) {
  Lat L;
  if (!make_lat(g, L) || !fS || !fSdot || !F || !dstar || !J || !Jdot) return -1;
  const double C = cbar_of(L, dstar, obs);
  if (!(C > 0.0)) return -2;
  std::vector<Dual> f(8 * (size_t)L.N), Fx(L.N), Fy(L.N);
  for (size_t i = 0; i < f.size(); ++i) f[i] = Dual(fS[i], fSdot[i]);
  for (int n = 0; n < L.N; ++n) {
    Fx[n] = Dual(F[n], Fdot ? Fdot[n] : 0.0);
    Fy[n] = Dual(F[L.N + n], Fdot ? Fdot[L.N + n] : 0.0);
  }
  const Dual r = objective_of<Dual>(L, f, Fx.data(), Fy.data(), dstar, obs, C);
  *J = r.v;
  *Jdot = r.d;
  return 0;
}

int orc_displacement(const orc_grid *g, const double *fS, const double *F, double *d_out) {
  Lat L;
  if (!make_lat(g, L) || !fS || !F || !d_out) return -1;
  std::vector<double> f(fS, fS + 8 * (size_t)L.N);
  const double dx2 = L.dx * L.dx;
  for (int n = 0; n < L.N; ++n) {
    double a = 0.0, b = 0.0;
    if (L.type[n]) node_disp(L, f, n, dx2 * F[n], dx2 * F[L.N + n], a, b);
    d_out[n] = a;
    d_out[L.N + n] = b;
  }
  return 0;
}

int orc_stress(const orc_grid *g, const double *E_node, const double *fS, const double *F,
               double *sigma_out) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !fS || !F || !sigma_out) return -1;
  NodeOps<double> ops;
  if (!make_ops(L, E_node, F, F + L.N, ops)) return -2;
  const int N = L.N;
  for (int n = 0; n < N; ++n) {
    sigma_out[n] = sigma_out[N + n] = sigma_out[2 * N + n] = 0.0;
    if (!L.type[n]) continue;
    double f[8], c[8], m[8], mc[8];
    for (int k = 0; k < 8; ++k) f[k] = fS[(size_t)k * N + n];
    const double *M = &ops.M[64 * (size_t)n];
    collide(f, ops.gx[n], ops.gy[n], ops.mat[n], M, &ops.Minv[64 * (size_t)n], c);
    matvec8(M, f, m);
    matvec8(M, c, mc);
    // bared moments (Eq. bared_moments) -> sigma = -[[mbar20, mbar11],[mbar11, mbar02]]
    const double b11 = 0.5 * (m[2] + mc[2]), bs = 0.5 * (m[3] + mc[3]), bd = 0.5 * (m[4] + mc[4]);
    sigma_out[n] = -0.5 * (bs + bd) / L.dx;
    sigma_out[N + n] = -0.5 * (bs - bd) / L.dx;
    sigma_out[2 * N + n] = -b11 / L.dx;
  }
  return 0;
}

int orc_monitor(const orc_grid *g, const double *fS, const double *F, double *c) {
  Lat L;
  if (!make_lat(g, L) || !fS || !F || !c) return -1;
  std::vector<double> f(fS, fS + 8 * (size_t)L.N);
  const double dx2 = L.dx * L.dx;
  double s = 0.0;
  for (int n = 0; n < L.N; ++n) {
    if (!L.type[n]) continue;
    double a, b;
    node_disp(L, f, n, dx2 * F[n], dx2 * F[L.N + n], a, b);
    s += a * a + b * b;
  }
  *c = L.n_active ? s / (double)L.n_active : 0.0;
  return 0;
}

int orc_apply_step(const orc_grid *g, const double *E_node, const double *x, double *y) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !x || !y) return -1;
  std::vector<double> zero(L.N, 0.0);
  NodeOps<double> ops;
  if (!make_ops(L, E_node, zero.data(), zero.data(), ops)) return -2;
  std::vector<Rule<double>> rules;
  if (!make_rules(L, ops, rules)) return -3;
  const size_t P = 8 * (size_t)L.N;
  std::vector<double> fS(x, x + P), fC(P), out(P);
  collide_all(L, ops, fS, fC, false);
  stream(L, rules, fC, out, false);
  std::memcpy(y, out.data(), sizeof(double) * P);
  return 0;
}

int orc_apply_step_transpose(const orc_grid *g, const double *E_node, const double *y,
                             double *x) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !x || !y) return -1;
  std::vector<double> zero(L.N, 0.0);
  NodeOps<double> ops;
  if (!make_ops(L, E_node, zero.data(), zero.data(), ops)) return -2;
  std::vector<Rule<double>> rules;
  if (!make_rules(L, ops, rules)) return -3;
  const size_t P = 8 * (size_t)L.N;
  std::vector<double> phiC(y, y + P), phiS(P);
  stream_T(L, rules, phiC, phiS);
  for (int n = 0; n < L.N; ++n) {
    for (int k = 0; k < 8; ++k) x[(size_t)k * L.N + n] = 0.0;
    if (!L.type[n]) continue;
    double A[64];
    collision_jacobian(ops, n, A);
    for (int j = 0; j < 8; ++j) {
      double s = 0.0;
      for (int r = 0; r < 8; ++r) s += A[r * 8 + j] * phiS[(size_t)r * L.N + n];
      x[(size_t)j * L.N + n] = s;
    }
  }
  return 0;
}

int orc_adjoint(const orc_grid *g, const double *E_node, const double *F, const double *fS,
                const double *dstar, const double *obs, long steps, double *phiC_out,
                double *phiS_out) {
  return run_adjoint(g, E_node, F, fS, dstar, obs, steps, phiC_out, phiS_out, nullptr);
}

int orc_adjoint_trace(const orc_grid *g, const double *E_node, const double *F,
                      const double *fS, const double *dstar, const double *obs, long steps,
                      double *c_out) {
  if (!c_out) return -1;
  Lat L;
  if (!make_lat(g, L)) return -1;
  std::vector<double> pc(8 * (size_t)L.N), ps(8 * (size_t)L.N);
  return run_adjoint(g, E_node, F, fS, dstar, obs, steps, pc.data(), ps.data(), c_out);
}

int orc_gradient_force(const orc_grid *g, const double *E_node, const double *F,
                       const double *fS, const double *phiS, const double *dstar,
                       const double *obs, double *grad_out) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !F || !fS || !phiS || !dstar || !grad_out) return -1;
  const int N = L.N;
  NodeOps<double> ops;
  if (!make_ops(L, E_node, F, F + N, ops)) return -2;
  const double C = cbar_of(L, dstar, obs);
  if (!(C > 0.0)) return -4;
  const double dx2 = L.dx * L.dx;
  std::vector<double> f(fS, fS + 8 * (size_t)N);
#pragma omp parallel for
  for (int n = 0; n < N; ++n) {
    grad_out[n] = grad_out[N + n] = 0.0;
    if (!L.type[n]) continue;
    const double w = obs ? obs[n] : 1.0;
    double dxn, dyn;
    node_disp(L, f, n, ops.gx[n], ops.gy[n], dxn, dyn);
    // dC_n/dg_i: the collision is affine in g, so C(0, e_i) - C(0, 0) is exact.
    double zero[8] = {0, 0, 0, 0, 0, 0, 0, 0}, c0[8], cx[8], cy[8];
    const double *M = &ops.M[64 * (size_t)n], *Mi = &ops.Minv[64 * (size_t)n];
    collide(zero, 0.0, 0.0, ops.mat[n], M, Mi, c0);
    collide(zero, 1.0, 0.0, ops.mat[n], M, Mi, cx);
    collide(zero, 0.0, 1.0, ops.mat[n], M, Mi, cy);
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < 8; ++k) {
      sx += phiS[(size_t)k * N + n] * (cx[k] - c0[k]);
      sy += phiS[(size_t)k * N + n] * (cy[k] - c0[k]);
    }
    // dJ/dF = dJ/dF (explicit, via g/2 in d) - (dC/dF)^T phi_S, with g = dx^2 F
    grad_out[n] = w * dx2 / C * (dxn - dstar[n]) * 0.5 * dx2 - dx2 * sx;
    grad_out[N + n] = w * dx2 / C * (dyn - dstar[N + n]) * 0.5 * dx2 - dx2 * sy;
  }
  return 0;
}

int orc_gradient_young(const orc_grid *g, const double *E_node, const double *F,
                       const double *fS, const double *phiS, const double *phiC,
                       double *grad_node, double *grad_total) {
  Lat L;
  if (!make_lat(g, L) || !E_node || !F || !fS || !phiS || !phiC) return -1;
  const int N = L.N;
  // Seed every node's modulus: each node's collision and streaming rules depend
  // only on its own E_n, so the tangents below are the per-node partials.
  std::vector<Dual> E(N), Fx(N), Fy(N);
  for (int n = 0; n < N; ++n) {
    E[n] = Dual(E_node[n], 1.0);
    Fx[n] = Dual(F[n], 0.0);
    Fy[n] = Dual(F[N + n], 0.0);
  }
  NodeOps<Dual> ops;
  if (!make_ops(L, E.data(), Fx.data(), Fy.data(), ops)) return -2;
  std::vector<Rule<Dual>> rules;
  if (!make_rules(L, ops, rules)) return -3;
  // f_C at the fixed point and dC/dE at fixed f_S
  std::vector<Dual> fSd(8 * (size_t)N), fCd(8 * (size_t)N);
  for (size_t i = 0; i < fSd.size(); ++i) fSd[i] = Dual(fS[i], 0.0);
  collide_all(L, ops, fSd, fCd, true);
  double total = 0.0;
  for (int n = 0; n < N; ++n) {
    double gn = 0.0;
    if (L.type[n]) {
      for (int k = 0; k < 8; ++k) gn -= phiS[(size_t)k * N + n] * fCd[(size_t)k * N + n].d;
      // streaming rules at node n (dst = (k, n)) depend on E_n through omega
      for (int k = 0; k < 8; ++k) {
        const Rule<Dual> &r = rules[(size_t)k * N + n];
        double ds = r.cst.d;
        for (int t = 0; t < r.nterm; ++t) ds += r.coef[t].d * fCd[r.src[t]].v;
        gn -= phiC[(size_t)k * N + n] * ds;
      }
    }
    if (grad_node) grad_node[n] = gn;
    total += gn;
  }
  if (grad_total) *grad_total = total;
  return 0;
}

}  // extern "C"
