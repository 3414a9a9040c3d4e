// Host side of the C ABI declared in include/lbm_solid.h: handle, validation, the
// primal / adjoint solve loops with their stopping rules, and kernel launches.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include "lbm_boundary.cuh"
#include "lbm_kernels.cuh"
#include "lbm_solid.h"

using namespace lbm;

struct lbm_solid {
  int nx = 0, ny = 0;
  long N = 0;
  double dx = 0.0;
  int periodic = 1;
  double nu = 0.0, E = 0.0;
  int control = 0, kernel = 0;
  cudaStream_t stream = nullptr;
  Grid grid{};
  Bounded bnd{};
  Coef coef{};
  Material mat{};
  long n_active = 0;
  bool has_neumann = false;
  // device buffers
  double *fA = nullptr, *fB = nullptr, *pA = nullptr, *pB = nullptr;
  double *g2 = nullptr, *r2 = nullptr, *dstar = nullptr, *obs = nullptr;
  double *basis = nullptr, *Fbase = nullptr;
  uint8_t *type = nullptr, *regmask = nullptr;
  int *bidx = nullptr;
  double *Q = nullptr, *s = nullptr, *dQ = nullptr, *ds = nullptr;
  YoungDeriv yd{};
  double alpha = 0.0;  // scalar Young control (E = alpha^2)
  // modulus field control: per-node constants, control copy, per-record gamma / node
  double *qfield = nullptr, *alphaN = nullptr, *gamf = nullptr;
  FixC *qfix = nullptr, *bfix = nullptr;
  uint8_t *bok = nullptr;
  int *bnode = nullptr;
  // compact launch of bounded grids: interior row chunks, boundary rules in compact form
  Compact cmp{};
  int2 *chunk = nullptr;
  uint8_t *negmask = nullptr;
  double *R = nullptr;
  long cblocks = 0;
  long obj_parts = 0;  // partials of the last objective pass
  int ctpb = kCompactThreads;  // threads per block of every compact launch
  bool hoist = false;          // boundary loads issued up front (latency-bound grids)
  long nmon = 0;  // blocks that write monitor partials in a sweep
  // cluster-resident sweeps of small periodic lattices (0 CTAs: not used)
  ClusterWork cw{};
  int cl_ncta = 0, cl_threads = 0;
  bool cl_pair = false;  // one node per lane pair (k_sweeps_cl PAIR)
  // lattice resident in distributed shared memory (0 CTAs: not used)
  int dsm_ncta = 0, dsm_h = 0, dsm_threads = 0;
  size_t dsm_smem = 0;
  Field fl{};
  bool field = false;
  // CUDA graphs of sweep chunks (launch overhead dominates small lattices): captured on
  // a private stream, replayed on the caller's stream, rebuilt when kernel parameters
  // passed by value change (version).
  cudaStream_t cap = nullptr;
  struct GraphEnt {
    int kind, parity, mon;
    long k, version;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEnt> graphs;
  // device-side solve loops (residual rule): graphs with a conditional WHILE node over
  // chunks of c sweeps, keyed like the sweep graphs; their state block in device and
  // pinned host memory
  std::vector<GraphEnt> loops;
  LoopState *dloop = nullptr, *hloop = nullptr;
  bool no_dloop = false;  // a loop graph could not be built: host loop only
  long version = 0;
  // forward-mode tangent (f-AD) buffers, allocated on first use
  double *tA = nullptr, *tB = nullptr, *qdot = nullptr;
  BoundaryNode *bnodes = nullptr;
  long nb = 0;
  double *partial = nullptr;
  long partial_cap = 0;
  double *dres = nullptr;
  double *hres = nullptr;  // pinned
  // state
  double *fcur = nullptr, *fnext = nullptr, *pcur = nullptr, *pnext = nullptr;
  bool fcur_is_fs = true;  // fcur holds an explicit f_S; otherwise f_C(t-1)
  bool have_target = false, adjoint_valid = false, adj_warm = false;
  // r (the adjoint source) is current while r_at == pstate; pstate changes with the
  // primal state, the force and the target
  long pstate = 0, r_at = -1;
  bool pcur_rest = false;  // the adjoint state is phi_C = 0 (not stored)
  double cbar = 0.0;
  long launches = 0;
  std::vector<double> samples;  // monitor samples c of the last criterion-0 solve
  bool broken = false;
  std::string err;
  dim3 blk, grd;
  long nblocks2d = 0;
};

namespace {

lbm_status fail(lbm_solid *h, lbm_status st, const std::string &msg) {
  if (h) {
    h->err = msg;
    if (st == LBM_ERR_CUDA) h->broken = true;
  }
  return st;
}

#define CK(h, call)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(h, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

#define LAUNCHED(h)                                                                     \
  do {                                                                                  \
    ++(h)->launches;                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess)                                                              \
      return fail(h, LBM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

constexpr double kTh = 1.0 / 3.0;

// c -> round(c 2^62) split as hi 2^31 + lo with 0 <= lo < 2^31 (|c| < 1/2).
FixC to_fixc(double c) {
  const long long C = std::llround(std::ldexp(c, 62));
  const long long hi = C >> 31;  // arithmetic shift: floor
  return FixC{(int)hi, (int)(C - hi * (1LL << 31))};
}

// Material map (Eqs. lambda, mu, K) and relaxation (Table A.1, Eq. relaxation, Eq. gamma).
bool material_coefs(double E, double nu, bool bounded, bool neumann, Coef &c, Material &m,
                    YoungDeriv &yd, std::string &why) {
  if (!(E > 0.0) || !std::isfinite(E)) { why = "Young's modulus must be > 0"; return false; }
  if (!(nu > -1.0 && nu < 1.0)) { why = "Poisson ratio must lie in (-1, 1)"; return false; }
  const double mu = E / (2.0 * (1.0 + nu));
  const double K = E / (2.0 * (1.0 - nu));
  const double t11 = mu / kTh, ts = 2.0 * K / (1.0 + kTh), td = 2.0 * mu / (1.0 - kTh);
  const double w11 = 1.0 / (t11 + 0.5), ws = 1.0 / (ts + 0.5), wd = 1.0 / (td + 0.5);
  c.c11 = 1.0 - w11; c.cs = 1.0 - ws; c.cd = 1.0 - wd;
  c.w11 = w11; c.ws = ws; c.wd = wd; c.K = K;
  c.gam = 0.0;
  if (bounded) {
    if (std::fabs(ts - 0.5) < 1e-14) { why = "tau_s = tau_f = 1/2 makes gamma singular"; return false; }
    c.gam = kTh * 0.5 / ((1.0 + kTh) * (ts - 0.5));
    if (neumann && (std::fabs(c.c11) < 1e-12 || std::fabs(c.cs) < 1e-12 || std::fabs(c.cd) < 1e-12)) {
      why = "a relaxed moment with omega = 1 leaves the Neumann wall stress undefined";
      return false;
    }
  }
  c.q11 = 0.25 * c.c11; c.qs = 0.25 * c.cs; c.qd = 0.25 * c.cd;
  c.fx = CoefFix{to_fixc(c.qs), to_fixc(c.qd), to_fixc(c.q11), to_fixc(1.0 / 3.0)};
  c.qs_b = c.cs * (0.25 + 0.5 * c.gam);
  c.P_b = -0.25 * c.gam * c.cs;
  c.fx.bnd_ok = std::fabs(c.qs_b) < 0.499 && std::fabs(c.P_b) < 0.499;
  if (c.fx.bnd_ok) {
    c.fx.qs_b = to_fixc(c.qs_b);
    c.fx.P_b = to_fixc(c.P_b);
  }
  // derivatives with respect to E: d omega = -omega^2 d tau
  const double dmu = 1.0 / (2.0 * (1.0 + nu)), dK = 1.0 / (2.0 * (1.0 - nu));
  const double dt11 = dmu / kTh, dts = 2.0 * dK / (1.0 + kTh), dtd = 2.0 * dmu / (1.0 - kTh);
  m.w11 = w11; m.ws = ws; m.wd = wd; m.K = K;
  m.dw11 = -w11 * w11 * dt11; m.dws = -ws * ws * dts; m.dwd = -wd * wd * dtd; m.dK = dK;
  yd.dc11 = -m.dw11; yd.dcs = -m.dws; yd.dcd = -m.dwd;
  yd.dgam = bounded ? -kTh * 0.5 * dts / ((1.0 + kTh) * (ts - 0.5) * (ts - 0.5)) : 0.0;
  return true;
}

lbm_status setup_boundary(lbm_solid *h) {
  if (h->periodic || h->nb == 0) return LBM_OK;
  const unsigned threads = 128;
  const unsigned blocks = (unsigned)((h->nb + threads - 1) / threads);
  k_boundary_setup<<<blocks, threads, 0, h->stream>>>(
      h->bnodes, h->nb, h->mat, h->dx, h->Q, h->s, h->dQ, h->ds, h->field ? h->alphaN : nullptr,
      h->bnode, h->nu, h->gamf, h->R, nullptr, h->bfix, h->bok);
  LAUNCHED(h);
  return LBM_OK;
}

lbm_status set_material(lbm_solid *h, double E) {
  Coef c{};
  Material m{};
  YoungDeriv yd{};
  std::string why;
  if (!material_coefs(E, h->nu, !h->periodic, h->has_neumann, c, m, yd, why))
    return fail(h, LBM_ERR_ARG, why);
  c.dx = h->dx;
  h->coef = c;
  h->mat = m;
  h->yd = yd;
  ++h->version;  // graphs bake Coef in as a kernel parameter
  h->E = E;
  return setup_boundary(h);
}

lbm_status finish(lbm_solid *h, long nb, int nv, int op, double scale, double *out) {
  k_finish<<<1, 256, 0, h->stream>>>(h->partial, nb, nv, op, scale, out);
  LAUNCHED(h);
  return LBM_OK;
}

lbm_status fetch(lbm_solid *h, int nv) {
  CK(h, cudaMemcpyAsync(h->hres, h->dres, sizeof(double) * nv, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

// Bounded grids launch their active nodes only (compact launch, lbm_kernels.cuh).
template <int A, bool F>
void launch_primal(lbm_solid *h, bool monitor) {
  if (h->periodic) {
    if (monitor)
      k_primal<false, true, A, F><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->fnext, h->g2, h->grid, h->bnd, h->coef, h->fl, h->partial);
    else
      k_primal<false, false, A, F><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->fnext, h->g2, h->grid, h->bnd, h->coef, h->fl, nullptr);
  } else {
    const unsigned nbk = (unsigned)h->cblocks;
    if (h->hoist) {
      if (monitor)
        k_primal_c<true, A, F, true><<<nbk, h->ctpb, 0, h->stream>>>(h->fcur, h->fnext, h->g2, h->grid, h->bnd, h->cmp, h->coef, h->fl, h->partial);
      else
        k_primal_c<false, A, F, true><<<nbk, h->ctpb, 0, h->stream>>>(h->fcur, h->fnext, h->g2, h->grid, h->bnd, h->cmp, h->coef, h->fl, nullptr);
    } else if (monitor) {
      k_primal_c<true, A, F, false><<<nbk, h->ctpb, 0, h->stream>>>(h->fcur, h->fnext, h->g2, h->grid, h->bnd, h->cmp, h->coef, h->fl, h->partial);
    } else {
      k_primal_c<false, A, F, false><<<nbk, h->ctpb, 0, h->stream>>>(h->fcur, h->fnext, h->g2, h->grid, h->bnd, h->cmp, h->coef, h->fl, nullptr);
    }
  }
}

template <int A, bool F>
void launch_adjoint(lbm_solid *h, bool monitor) {
  if (h->periodic) {
    if (monitor)
      k_adjoint<false, true, A, F><<<h->grd, h->blk, 0, h->stream>>>(h->pcur, h->pnext, h->r2, h->grid, h->bnd, h->coef, h->fl, h->partial);
    else
      k_adjoint<false, false, A, F><<<h->grd, h->blk, 0, h->stream>>>(h->pcur, h->pnext, h->r2, h->grid, h->bnd, h->coef, h->fl, nullptr);
  } else {
    const unsigned nbk = (unsigned)h->cblocks;
    if (h->hoist) {
      if (monitor)
        k_adjoint_c<true, A, F, true><<<nbk, h->ctpb, 0, h->stream>>>(h->pcur, h->pnext, h->r2, h->grid, h->bnd, h->cmp, h->coef, h->fl, h->partial);
      else
        k_adjoint_c<false, A, F, true><<<nbk, h->ctpb, 0, h->stream>>>(h->pcur, h->pnext, h->r2, h->grid, h->bnd, h->cmp, h->coef, h->fl, nullptr);
    } else if (monitor) {
      k_adjoint_c<true, A, F, false><<<nbk, h->ctpb, 0, h->stream>>>(h->pcur, h->pnext, h->r2, h->grid, h->bnd, h->cmp, h->coef, h->fl, h->partial);
    } else {
      k_adjoint_c<false, A, F, false><<<nbk, h->ctpb, 0, h->stream>>>(h->pcur, h->pnext, h->r2, h->grid, h->bnd, h->cmp, h->coef, h->fl, nullptr);
    }
  }
}

template <int A, bool F>
void launch_collide_only(lbm_solid *h) {
  if (h->periodic)
    k_collide_only<false, A, F><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->fnext, h->g2, h->grid, h->bnd, h->coef, h->fl);
  else
    k_collide_only<true, A, F><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->fnext, h->g2, h->grid, h->bnd, h->coef, h->fl);
}

// ---- cluster-resident sweeps ---------------------------------------------------------
// Measured on B300 (time to gradient, us per sweep, cluster vs graph-replayed launches):
// periodic 10^2 .. 40^2: 2.15-2.35 vs 2.6-2.8; 80^2: 4.0 vs 2.8; plates at N_x = 64: no
// gain; 128^2 plate with a modulus field: 8.4 vs 6.6.  Inside one launch a sweep still
// costs an L2 round trip plus the cluster barrier (~2 us); only the smallest lattices,
// where a graph launch costs more than that, gain.  So: periodic lattices up to 2048
// nodes.
constexpr long kClusterMaxItems = 2048;
constexpr int kClusterMaxCta = 16;            // one GPC (non-portable cluster size)
constexpr long kClusterChunk = 512;           // sweeps per launch (fixed-step runs)

template <int KIND, bool BOUNDED, int ARITH, bool FIELD, bool PAIR = false>
cudaError_t launch_cluster(lbm_solid *h, int nsweeps, bool monitor, bool probe = false,
                           int *fits = nullptr, int chunk = 0, long long max_iters = 0,
                           double tol = 0.0, int first = 0) {
  auto kern = k_sweeps_cl<KIND, BOUNDED, ARITH, FIELD, PAIR>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)h->cl_ncta);
  cfg.blockDim = dim3((unsigned)h->cl_threads);
  cfg.stream = h->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)h->cl_ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (probe) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveClusters(fits, kern, &cfg);
  }
  double *a = KIND == 0 ? h->fcur : h->pcur, *b = KIND == 0 ? h->fnext : h->pnext;
  const double *src = KIND == 0 ? h->g2 : h->r2;
  return cudaLaunchKernelEx(&cfg, kern, a, b, src, h->grid, h->bnd, h->cmp, h->coef, h->fl,
                            h->cw, nsweeps, monitor ? 1 : 0, h->partial, h->nmon, chunk,
                            first, max_iters, tol, h->dloop);
}

// (periodic lattices only: bounded grids measured no gain, see kClusterMaxItems)
template <int KIND>
cudaError_t launch_cluster_any(lbm_solid *h, int nsweeps, bool monitor, bool probe = false,
                               int *fits = nullptr, int chunk = 0, long long max_iters = 0,
                               double tol = 0.0, int first = 0) {
  const bool fp = h->kernel == LBM_KERNEL_FP64;
  if (h->field)
    return fp ? launch_cluster<KIND, false, 0, true>(h, nsweeps, monitor, probe, fits, chunk, max_iters, tol, first)
              : h->cl_pair
                    ? launch_cluster<KIND, false, 1, true, true>(h, nsweeps, monitor, probe, fits, chunk, max_iters, tol, first)
                    : launch_cluster<KIND, false, 1, true>(h, nsweeps, monitor, probe, fits, chunk, max_iters, tol, first);
  return fp ? launch_cluster<KIND, false, 0, false>(h, nsweeps, monitor, probe, fits, chunk, max_iters, tol, first)
            : h->cl_pair
                  ? launch_cluster<KIND, false, 1, false, true>(h, nsweeps, monitor, probe, fits, chunk, max_iters, tol, first)
                  : launch_cluster<KIND, false, 1, false>(h, nsweeps, monitor, probe, fits, chunk, max_iters, tol, first);
}

// Launch shape of the compact sweep of a bounded grid.  Below ~32 warps per SM the sweep
// is latency-bound and its critical path is the warps of boundary records: blocks of 32
// threads spread them (and the interior chunks) over more SMs, and the HOIST kernels
// issue all of a record's loads before its arithmetic (~120 registers, which a grid of
// that size can afford).  Measured per primal sweep on the clamped / tensioned plate
// (128-thread blocks -> 32-thread hoisted): N_x = 64 5.6 -> 4.6 us, 256 6.2 -> 4.7 us,
// 512 7.1 -> 5.3 us; at N_x = 1024 (10.9 k warps) 128-thread blocks without it stay
// faster (10.6 us against 13.1 us).
int compact_block_size(long nb, long nchunk) {
  const long warps = (nb + 31) / 32 + nchunk;
  return warps <= 148L * 32 ? 32 : kCompactThreads;
}
bool compact_hoist(long nb, long nchunk) { return compact_block_size(nb, nchunk) == 32; }

// ---- lattices resident in distributed shared memory (k_sweeps_dsm) -------------------
// Measured on B300 (us per sweep, graph-replayed / L2 cluster / distributed shared
// memory): 16^2 2.19 / 1.61 / 1.72, 32^2 2.20 / 1.63 / 1.69, 40^2 2.22 / 1.73 / 2.10,
// 64^2 2.24 / 2.50 / 2.06, 80^2 2.25 / 3.34 / 3.14, 128^2 2.31 / 5.79 / 5.79.  A sweep of
// a cluster-resident lattice costs one warp's collisions plus the cluster barrier, and
// the L2 round trip the shared-memory lattice saves is a small part of it; one GPC's 16
// SMs fall behind the whole GPU from ~80^2.  So: the L2 cluster up to 2048 nodes, the
// shared-memory lattice above that up to 4096 nodes (64^2: time to gradient 5.36 -> 5.05
// ms), graph-replayed launches beyond.
constexpr long kDsmMaxNodes = 4096;
constexpr long kDsmBandNodes = 128;

template <int KIND, int ARITH>
cudaError_t launch_dsm(lbm_solid *h, int nsweeps, bool monitor, bool probe = false,
                       int *fits = nullptr, int chunk = 0, long long max_iters = 0,
                       double tol = 0.0, int first = 0) {
  auto kern = k_sweeps_dsm<KIND, ARITH>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)h->dsm_ncta);
  cfg.blockDim = dim3((unsigned)h->dsm_threads);
  cfg.dynamicSmemBytes = h->dsm_smem;
  cfg.stream = h->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)h->dsm_ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (probe) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->dsm_smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveClusters(fits, kern, &cfg);
  }
  double *a = KIND == 0 ? h->fcur : h->pcur, *b = KIND == 0 ? h->fnext : h->pnext;
  const double *src = KIND == 0 ? h->g2 : h->r2;
  return cudaLaunchKernelEx(&cfg, kern, a, b, src, h->grid, h->coef, h->dsm_h, nsweeps,
                            monitor ? 1 : 0, h->partial, h->nmon, chunk, first, max_iters,
                            tol, h->dloop);
}

template <int KIND>
cudaError_t launch_dsm_any(lbm_solid *h, int nsweeps, bool monitor, bool probe = false,
                           int *fits = nullptr, int chunk = 0, long long max_iters = 0,
                           double tol = 0.0, int first = 0) {
  return h->kernel == LBM_KERNEL_FP64
             ? launch_dsm<KIND, 0>(h, nsweeps, monitor, probe, fits, chunk, max_iters, tol, first)
             : launch_dsm<KIND, 1>(h, nsweeps, monitor, probe, fits, chunk, max_iters, tol, first);
}

// Chooses the cluster for a lattice held in distributed shared memory: C CTAs with C
// dividing ny (bands of whole rows), at most one GPC's worth, the fewest CTAs whose band
// holds at most 128 nodes (one warp per SM sub-partition: a sweep is the latency of one
// warp's collisions plus the barrier) when there is one, else the most that fit; checks
// that such a cluster can be scheduled with its shared memory.
void setup_dsm(lbm_solid *h) {
  h->dsm_ncta = 0;
  if (!h->periodic || h->field || h->N <= kClusterMaxItems || h->N > kDsmMaxNodes) return;
  int dev = 0, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess)
    return;
  smem_max -= 1024;  // the kernel's static reduction scratch
  std::vector<int> order;
  for (int c = 1; c <= kClusterMaxCta; ++c)
    if (h->ny % c == 0 && (long)(h->ny / c) * h->nx <= kDsmBandNodes) order.push_back(c);
  for (int c = kClusterMaxCta; c >= 1; --c)
    if (h->ny % c == 0 && (long)(h->ny / c) * h->nx > kDsmBandNodes) order.push_back(c);
  for (int c : order) {
    const long L = (long)(h->ny / c) * h->nx;
    const size_t bytes = (size_t)L * kDsmDoublesPerNode * sizeof(double);
    if (bytes > (size_t)smem_max) continue;
    h->dsm_ncta = c;
    h->dsm_h = h->ny / c;
    h->dsm_threads = (int)std::min<long>(512, (L + 31) / 32 * 32);
    h->dsm_smem = bytes;
    int f0 = 0, f1 = 0;
    if (launch_dsm_any<0>(h, 0, false, true, &f0) == cudaSuccess && f0 > 0 &&
        launch_dsm_any<1>(h, 0, false, true, &f1) == cudaSuccess && f1 > 0) {
      if (h->nmon < c) h->nmon = c;
      return;
    }
    cudaGetLastError();  // clear a refused configuration, try the next
  }
  h->dsm_ncta = 0;
}

// Chooses the cluster shape for a small lattice (CTAs of whole warps, about one item per
// thread, as many CTAs as a GPC allows) and checks that such a cluster can be scheduled;
// otherwise the handle keeps the graph-replayed launches.  With at most 64 nodes per CTA
// (2 warps: half the SM sub-partitions idle) the fixed-point sweeps run in pair form, two
// lanes per node.
void setup_cluster(lbm_solid *h, long items) {
  h->cl_ncta = 0;
  if (items < 1 || items > kClusterMaxItems) return;
  for (int ncta = (int)std::min<long>(kClusterMaxCta, (items + 31) / 32); ncta >= 1; ncta /= 2) {
    const long per = (items + ncta - 1) / ncta;
    h->cl_ncta = ncta;
    h->cl_pair = h->periodic && h->kernel != LBM_KERNEL_FP64 && per <= 64;
    h->cl_threads = (int)std::min<long>(256, ((h->cl_pair ? 2 : 1) * per + 31) / 32 * 32);
    int f0 = 0, f1 = 0;
    if (launch_cluster_any<0>(h, 0, false, true, &f0) == cudaSuccess && f0 > 0 &&
        launch_cluster_any<1>(h, 0, false, true, &f1) == cudaSuccess && f1 > 0) {
      if (h->nmon < ncta) h->nmon = ncta;
      return;
    }
    cudaGetLastError();  // clear a refused configuration, try a smaller cluster
  }
  h->cl_ncta = 0;
}

// Kernel variant of a sweep: FP64 pipe for LBM_KERNEL_FP64, fixed-point bulk nodes
// otherwise; per-node constants for modulus fields.
void launch_primal_any(lbm_solid *h, bool monitor) {
  const bool fp = h->kernel == LBM_KERNEL_FP64;
  if (h->field) {
    if (fp) launch_primal<0, true>(h, monitor);
    else launch_primal<1, true>(h, monitor);
  } else {
    if (fp) launch_primal<0, false>(h, monitor);
    else launch_primal<1, false>(h, monitor);
  }
}

void launch_adjoint_any(lbm_solid *h, bool monitor) {
  const bool fp = h->kernel == LBM_KERNEL_FP64;
  if (h->field) {
    if (fp) launch_adjoint<0, true>(h, monitor);
    else launch_adjoint<1, true>(h, monitor);
  } else {
    if (fp) launch_adjoint<0, false>(h, monitor);
    else launch_adjoint<1, false>(h, monitor);
  }
}

// One primal sweep; optional monitor partials (nmon sums of |d|^2).
lbm_status primal_sweep(lbm_solid *h, bool monitor) {
  const bool fp = h->kernel == LBM_KERNEL_FP64;
  if (h->fcur_is_fs) {
    if (h->field) {
      if (fp) launch_collide_only<0, true>(h);
      else launch_collide_only<1, true>(h);
    } else if (fp) {
      launch_collide_only<0, false>(h);
    } else {
      launch_collide_only<1, false>(h);
    }
  } else {
    launch_primal_any(h, monitor);
  }
  LAUNCHED(h);
  std::swap(h->fcur, h->fnext);
  h->fcur_is_fs = false;
  return LBM_OK;
}

lbm_status adjoint_sweep(lbm_solid *h, bool monitor) {
  launch_adjoint_any(h, monitor);
  LAUNCHED(h);
  std::swap(h->pcur, h->pnext);
  return LBM_OK;
}

constexpr long kGraphMin = 4, kGraphMax = 128;

// Sweeps that are replayed from a captured graph: k plain sweeps starting from buffer
// parity `parity`, the last one with monitor partials when mon is set.
lbm_status graph_for(lbm_solid *h, int kind, long k, bool mon, cudaGraphExec_t &exec) {
  const int parity = kind == 0 ? (h->fcur == h->fA ? 0 : 1) : (h->pcur == h->pA ? 0 : 1);
  for (const auto &g : h->graphs)
    if (g.kind == kind && g.k == k && g.parity == parity && g.mon == (int)mon &&
        g.version == h->version) {
      exec = g.exec;
      return LBM_OK;
    }
  if (!h->cap) CK(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  double *f0 = h->fcur, *f1 = h->fnext, *p0 = h->pcur, *p1 = h->pnext;
  cudaStream_t user = h->stream;
  const long launches = h->launches;
  CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  h->stream = h->cap;
  lbm_status st = LBM_OK;
  for (long i = 0; i < k && st == LBM_OK; ++i) {
    const bool m = mon && i == k - 1;
    // the kernels themselves (primal_sweep / adjoint_sweep without the launch check,
    // which would see the capture state)
    if (kind == 0) {
      launch_primal_any(h, m);
      std::swap(h->fcur, h->fnext);
    } else {
      launch_adjoint_any(h, m);
      std::swap(h->pcur, h->pnext);
    }
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
  h->stream = user;
  h->fcur = f0; h->fnext = f1; h->pcur = p0; h->pnext = p1;
  h->launches = launches;
  if (ec != cudaSuccess || !graph)
    return fail(h, LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess)
    return fail(h, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  if (h->graphs.size() >= 16) {
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(lbm_solid::GraphEnt{kind, parity, (int)mon, k, h->version, ex});
  exec = ex;
  return st;
}

// k sweeps (kind 0 primal, 1 adjoint), monitor partials on the last one if mon.
lbm_status run_sweeps(lbm_solid *h, int kind, long k, bool mon) {
  if (kind == 0 && k > 0) ++h->pstate;
  if (kind == 0 && h->fcur_is_fs && k > 0) {  // first sweep from an explicit f_S
    lbm_status st = primal_sweep(h, false);
    if (st) return st;
    --k;
  }
  if (kind == 1 && h->pcur_rest && k > 0) {  // first adjoint sweep from rest: -j
    if (h->periodic)
      k_adjoint_rest<false><<<148 * 8, 256, 0, h->stream>>>(h->r2, h->pnext, h->grid, h->bnd);
    else
      k_adjoint_rest<true><<<148 * 8, 256, 0, h->stream>>>(h->r2, h->pnext, h->grid, h->bnd);
    LAUNCHED(h);
    std::swap(h->pcur, h->pnext);
    h->pcur_rest = false;
    --k;
  }
  if (h->dsm_ncta > 0 || h->cl_ncta > 0) {  // small lattice: cluster launches of <= 512 sweeps
    const bool dsm = h->dsm_ncta > 0;
    while (k > 0) {
      const long c = k > kClusterChunk ? kClusterChunk : k;
      const bool m = mon && c == k;
      const cudaError_t e =
          dsm ? (kind == 0 ? launch_dsm_any<0>(h, (int)c, m) : launch_dsm_any<1>(h, (int)c, m))
              : (kind == 0 ? launch_cluster_any<0>(h, (int)c, m)
                           : launch_cluster_any<1>(h, (int)c, m));
      if (e != cudaSuccess)
        return fail(h, LBM_ERR_CUDA, std::string("cluster launch: ") + cudaGetErrorString(e));
      LAUNCHED(h);
      if (c & 1) {
        if (kind == 0) std::swap(h->fcur, h->fnext);
        else std::swap(h->pcur, h->pnext);
      }
      k -= c;
    }
    return LBM_OK;
  }
  while (k > 0) {
    long c = k > kGraphMax ? kGraphMax : k;
    if (k > kGraphMax && k - c < kGraphMin) c = k - kGraphMin;  // keep the tail graphable
    const bool m = mon && c == k;
    if (c < kGraphMin) {
      for (long i = 0; i < c; ++i) {
        lbm_status st = kind == 0 ? primal_sweep(h, m && i == c - 1) : adjoint_sweep(h, m && i == c - 1);
        if (st) return st;
      }
    } else {
      cudaGraphExec_t ex = nullptr;
      lbm_status st = graph_for(h, kind, c, m, ex);
      if (st) return st;
      CK(h, cudaGraphLaunch(ex, h->stream));
      h->launches += c;
      if (c & 1) {
        if (kind == 0) std::swap(h->fcur, h->fnext);
        else std::swap(h->pcur, h->pnext);
      }
    }
    k -= c;
  }
  return LBM_OK;
}

lbm_status set_field(lbm_solid *h) {
  k_set_young_field<<<148 * 4, 256, 0, h->stream>>>(h->alphaN, h->nu, h->N, h->qfield, h->qfix);
  LAUNCHED(h);
  return setup_boundary(h);
}

lbm_status residual(lbm_solid *h, const double *a, const double *b, double &res) {
  long blocks;
  if (h->periodic) {
    const long total = 8 * h->N;
    blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    k_residual<<<(unsigned)blocks, 256, 0, h->stream>>>(a, b, total, h->partial);
  } else {  // active nodes only
    blocks = h->cblocks;
    k_residual_c<<<(unsigned)blocks, h->ctpb, 0, h->stream>>>(a, b, h->grid, h->cmp, h->partial);
  }
  LAUNCHED(h);
  lbm_status st = finish(h, blocks, 2, 1, 1.0, h->dres);
  if (st) return st;
  if ((st = fetch(h, 2))) return st;
  res = h->hres[1] > 0.0 ? h->hres[0] / h->hres[1] : (h->hres[0] > 0.0 ? INFINITY : 0.0);
  if (!std::isfinite(h->hres[0]) || !std::isfinite(h->hres[1])) res = NAN;
  return LBM_OK;
}

// The device-side solve loop for the residual rule: a graph whose conditional WHILE node
// runs [c sweeps (c even, so the buffers return to the same roles), residual partials,
// their reduction, k_loop_decide] until the residual is below tol, not finite, or the
// chunk limit in the state block is reached.  No host round trip per chunk.
lbm_status loop_graph_for(lbm_solid *h, int kind, long c, cudaGraphExec_t &exec) {
  const int parity = kind == 0 ? (h->fcur == h->fA ? 0 : 1) : (h->pcur == h->pA ? 0 : 1);
  for (const auto &g : h->loops)
    if (g.kind == kind && g.k == c && g.parity == parity && g.version == h->version) {
      exec = g.exec;
      return LBM_OK;
    }
  if (!h->cap) CK(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  CK(h, cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle hnd;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphConditionalHandleCreate(&hnd, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  }
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(h->cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {  // refused: the caller keeps the host loop (handle stays usable)
    cudaGraphDestroy(graph);
    cudaGetLastError();
    h->err = std::string("loop graph: ") + cudaGetErrorString(e);
    return LBM_ERR_STATE;
  }
  double *f0 = h->fcur, *f1 = h->fnext, *p0 = h->pcur, *p1 = h->pnext;
  cudaStream_t user = h->stream;
  h->stream = h->cap;
  cudaError_t el = cudaSuccess;
  if (h->dsm_ncta > 0 || h->cl_ncta > 0) {  // one cluster launch of c sweeps
    el = h->dsm_ncta > 0
             ? (kind == 0 ? launch_dsm_any<0>(h, (int)c, false) : launch_dsm_any<1>(h, (int)c, false))
             : (kind == 0 ? launch_cluster_any<0>(h, (int)c, false)
                          : launch_cluster_any<1>(h, (int)c, false));
  } else {
    for (long i = 0; i < c; ++i) {
      if (kind == 0) {
        launch_primal_any(h, false);
        std::swap(h->fcur, h->fnext);
      } else {
        launch_adjoint_any(h, false);
        std::swap(h->pcur, h->pnext);
      }
    }
  }
  // residual of the chunk's last two states (as residual(), without the fetch)
  const double *ra = kind == 0 ? f0 : p0, *rb = kind == 0 ? f1 : p1;
  long blocks;
  if (h->periodic) {
    const long total = 8 * h->N;
    blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    k_residual<<<(unsigned)blocks, 256, 0, h->stream>>>(ra, rb, total, h->partial);
  } else {
    blocks = h->cblocks;
    k_residual_c<<<(unsigned)blocks, h->ctpb, 0, h->stream>>>(ra, rb, h->grid, h->cmp, h->partial);
  }
  k_finish<<<1, 256, 0, h->stream>>>(h->partial, blocks, 2, 1, 1.0, h->dres);
  k_loop_decide<<<1, 1, 0, h->stream>>>(h->dres, h->dloop, hnd);
  cudaGraph_t body = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(h->cap, &body);
  h->stream = user;
  h->fcur = f0; h->fnext = f1; h->pcur = p0; h->pnext = p1;
  cudaGraphExec_t ex = nullptr;
  cudaError_t ei = (el == cudaSuccess && ec == cudaSuccess) ? cudaGraphInstantiate(&ex, graph, 0)
                                                             : (el != cudaSuccess ? el : ec);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {  // as above
    cudaGetLastError();
    h->err = std::string("loop graph: ") + cudaGetErrorString(ei);
    return LBM_ERR_STATE;
  }
  if (h->loops.size() >= 8) {
    cudaGraphExecDestroy(h->loops.front().exec);
    h->loops.erase(h->loops.begin());
  }
  h->loops.push_back(lbm_solid::GraphEnt{kind, parity, 0, c, h->version, ex});
  exec = ex;
  return LBM_OK;
}

// Runs up to max_iters chunks on the device (residual rule): a first chunk of `first`
// sweeps (cluster-resident lattices only; c otherwise), then chunks of c; returns the
// chunks run and the last residual.  ok = false when no loop graph can be built (the
// caller keeps the host loop).
lbm_status device_loop(lbm_solid *h, int kind, long c, long first, long max_iters, double tol,
                       long &iters, double &metric, bool &ok) {
  ok = false;
  if (h->no_dloop) return LBM_OK;
  if (!h->dloop) {
    CK(h, cudaMalloc((void **)&h->dloop, sizeof(LoopState)));
    CK(h, cudaMallocHost((void **)&h->hloop, sizeof(LoopState)));
  }
  *h->hloop = LoopState{tol, max_iters, 0, 0.0};
  const bool cluster = h->dsm_ncta > 0 || h->cl_ncta > 0;
  if (cluster) {
    // a cluster-resident lattice: the kernel itself loops over the chunks
    if (c > INT32_MAX || first < 1 || first > c) return LBM_OK;
    CK(h, cudaMemcpyAsync(h->dloop, h->hloop, sizeof(LoopState), cudaMemcpyHostToDevice, h->stream));
    const int ci = (int)c, fi = (int)first;
    const cudaError_t e =
        h->dsm_ncta > 0
            ? (kind == 0 ? launch_dsm_any<0>(h, 0, false, false, nullptr, ci, max_iters, tol, fi)
                         : launch_dsm_any<1>(h, 0, false, false, nullptr, ci, max_iters, tol, fi))
            : (kind == 0 ? launch_cluster_any<0>(h, 0, false, false, nullptr, ci, max_iters, tol, fi)
                         : launch_cluster_any<1>(h, 0, false, false, nullptr, ci, max_iters, tol, fi));
    if (e != cudaSuccess)
      return fail(h, LBM_ERR_CUDA, std::string("cluster loop launch: ") + cudaGetErrorString(e));
    ++h->launches;
  } else {
    if (first != c) return LBM_OK;
    cudaGraphExec_t ex = nullptr;
    const lbm_status ls = loop_graph_for(h, kind, c, ex);
    if (ls == LBM_ERR_STATE) {  // capture into a conditional body refused: host loop
      h->no_dloop = true;
      h->err.clear();
      return LBM_OK;
    }
    if (ls) return ls;
    CK(h, cudaMemcpyAsync(h->dloop, h->hloop, sizeof(LoopState), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaGraphLaunch(ex, h->stream));
  }
  CK(h, cudaMemcpyAsync(h->hloop, h->dloop, sizeof(LoopState), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  iters = (long)h->hloop->iters;
  metric = h->hloop->metric;
  if (!cluster) h->launches += iters * (c + 3);
  if (cluster && iters > 0 && ((first + (iters - 1) * c) & 1)) {  // state ended in b
    if (kind == 0) std::swap(h->fcur, h->fnext);
    else std::swap(h->pcur, h->pnext);
  }
  if (kind == 0) ++h->pstate;
  ok = true;
  return LBM_OK;
}

// Shared stopping loop of the primal and adjoint solves.
template <class Resid>
lbm_status solve_loop(lbm_solid *h, const lbm_solve_opts *o, lbm_solve_info *info, int kind,
                      Resid resid) {
  const auto t0 = std::chrono::steady_clock::now();
  long steps = 0;
  double metric = 0.0;
  lbm_status result = LBM_OK;
  if (o->fixed_steps) {
    lbm_status st = run_sweeps(h, kind, o->max_steps, false);
    if (st) return st;
    steps = o->max_steps;
  } else {
    std::deque<double> win;
    h->samples.clear();
    bool done = false;
    // residual rule on a cluster-resident lattice: one launch runs every whole chunk (the
    // collide-only or from-rest first sweep, when due, is launched just before and
    // counts towards the first chunk)
    const long ce = o->check_every;
    if (o->criterion == 1 && (h->dsm_ncta > 0 || h->cl_ncta > 0) && ce % 2 == 0 &&
        ce <= INT32_MAX && o->max_steps >= ce) {
      long pre = 0;
      if ((kind == 0 && h->fcur_is_fs) || (kind == 1 && h->pcur_rest)) {
        lbm_status st = run_sweeps(h, kind, 1, false);
        if (st) return st;
        pre = 1;
      }
      long iters = 0;
      double mv = 0.0;
      bool ok = false;
      lbm_status st = device_loop(h, kind, ce, ce - pre, o->max_steps / ce, o->tol, iters, mv, ok);
      if (st) return st;
      steps = ok ? iters * ce : pre;
      if (ok) {
        metric = mv;
        if (std::isnan(mv)) result = LBM_ERR_DIVERGED;
        else if (mv < o->tol) done = true;
      }
    }
    while (result == LBM_OK && !done && steps < o->max_steps) {
      long k = o->check_every;
      if (k > o->max_steps - steps) k = o->max_steps - steps;
      // a chunk whose only sweep is the collide-only first sweep has no monitor value
      const bool first_only = kind == 0 && h->fcur_is_fs && k == 1;
      lbm_status st = run_sweeps(h, kind, k, o->criterion == 0);
      if (st) return st;
      steps += k;
      if (steps < 2 || first_only) continue;
      double v = 0.0;
      if (o->criterion == 0) {
        lbm_status st = finish(h, h->nmon, 1, 0, h->n_active ? 1.0 / h->n_active : 0.0, h->dres);
        if (st) return st;
        if ((st = fetch(h, 1))) return st;
        v = h->hres[0];
        h->samples.push_back(v);
        if (!std::isfinite(v)) { metric = v; result = LBM_ERR_DIVERGED; break; }
        win.push_back(v);
        if ((long)win.size() > o->window) win.pop_front();
        if ((long)win.size() == o->window) {
          double mean = 0.0, var = 0.0;
          for (double c : win) mean += c;
          mean /= (double)win.size();
          for (double c : win) var += (c - mean) * (c - mean);
          const double sd = std::sqrt(var / (double)win.size());
          metric = mean > 0.0 ? sd / mean : (sd == 0.0 ? 0.0 : INFINITY);
          if (metric < o->tol) done = true;
        }
      } else {
        lbm_status st = resid(v);
        if (st) return st;
        metric = v;
        if (std::isnan(v)) { result = LBM_ERR_DIVERGED; break; }
        if (v < o->tol) { done = true; break; }
        // the remaining whole chunks on the device (the first chunk, which may hold the
        // collide-only or from-rest first sweep, ran above)
        const long c = o->check_every, iters_max = (o->max_steps - steps) / c;
        if (c % 2 == 0 && iters_max >= 1) {
          long iters = 0;
          double mv = 0.0;
          bool ok = false;
          if ((st = device_loop(h, kind, c, c, iters_max, o->tol, iters, mv, ok))) return st;
          if (ok) {
            steps += iters * c;
            metric = mv;
            if (std::isnan(mv)) { result = LBM_ERR_DIVERGED; break; }
            if (mv < o->tol) { done = true; break; }
          }
        }
      }
    }
    if (result == LBM_OK && !done) result = LBM_ERR_NOT_CONVERGED;
  }
  if (info) {
    info->steps = steps;
    info->last_metric = metric;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (result == LBM_ERR_NOT_CONVERGED) h->err = "max_steps reached before the stopping rule held";
  if (result == LBM_ERR_DIVERGED) h->err = "non-finite monitor value";
  return result;
}

lbm_status check_opts(lbm_solid *h, const lbm_solve_opts *o) {
  if (!o) return fail(h, LBM_ERR_ARG, "opts is NULL");
  if (o->max_steps < 1) return fail(h, LBM_ERR_ARG, "max_steps must be >= 1");
  if (!o->fixed_steps) {
    if (o->check_every < 1) return fail(h, LBM_ERR_ARG, "check_every must be >= 1");
    if (o->criterion == 0 && o->window < 2) return fail(h, LBM_ERR_ARG, "window must be >= 2");
    if (o->criterion != 0 && o->criterion != 1) return fail(h, LBM_ERR_ARG, "criterion must be 0 or 1");
    if (!(o->tol > 0.0)) return fail(h, LBM_ERR_ARG, "tol must be > 0");
  }
  return LBM_OK;
}

// Grid of the integer-pipe objective and gradient passes of periodic lattices.
constexpr int kFixPassBlocks = 148 * 4;  // one wave at 64 registers, 256 threads

// Objective partials and r; returns through obj_parts the number of partials written.
lbm_status objective_partials(lbm_solid *h) {
  h->r_at = h->pstate;
  const double scale = h->dx * h->dx / h->cbar;
  h->obj_parts = h->nblocks2d;
  if (h->periodic && !h->fcur_is_fs && h->kernel != LBM_KERNEL_FP64) {
    h->obj_parts = kFixPassBlocks;
    if (h->obs)
      k_objective_fix<true><<<kFixPassBlocks, 256, 0, h->stream>>>(h->fcur, h->g2, h->dstar, h->obs, h->r2, scale, h->grid, h->partial);
    else
      k_objective_fix<false><<<kFixPassBlocks, 256, 0, h->stream>>>(h->fcur, h->g2, h->dstar, nullptr, h->r2, scale, h->grid, h->partial);
  } else if (h->periodic) {
    if (h->fcur_is_fs)
      k_objective<false, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->g2, h->dstar, h->obs, h->r2, scale, h->grid, h->bnd, h->partial);
    else
      k_objective<false, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->g2, h->dstar, h->obs, h->r2, scale, h->grid, h->bnd, h->partial);
  } else {
    if (h->fcur_is_fs)
      k_objective<true, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->g2, h->dstar, h->obs, h->r2, scale, h->grid, h->bnd, h->partial);
    else
      k_objective<true, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->g2, h->dstar, h->obs, h->r2, scale, h->grid, h->bnd, h->partial);
  }
  LAUNCHED(h);
  return LBM_OK;
}

void free_all(lbm_solid *h) {
  void *bufs[] = {h->fA, h->fB, h->pA, h->pB, h->g2, h->r2, h->dstar, h->obs, h->basis, h->Fbase,
                  h->type, h->regmask, h->bidx, h->Q, h->s, h->dQ, h->ds, h->bnodes,
                  h->partial, h->dres, h->qfield, h->alphaN, h->gamf, h->bnode, h->tA, h->tB,
                  h->qdot, h->qfix, h->chunk, h->negmask, h->R, h->bfix, h->bok};
  for (void *p : bufs)
    if (p) cudaFree(p);
  if (h->hres) cudaFreeHost(h->hres);
}

}  // namespace

extern "C" {

const char *lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_STATE: return "call out of order";
    case LBM_ERR_NOT_CONVERGED: return "not converged";
    case LBM_ERR_DIVERGED: return "diverged";
  }
  return "unknown status";
}

const char *lbm_solid_last_error(const lbm_solid *h) { return h ? h->err.c_str() : "null handle"; }

long lbm_solid_launch_count(const lbm_solid *h) { return h ? h->launches : -1; }

long lbm_solid_monitor_samples(const lbm_solid *h, double *dst, long cap) {
  if (!h) return -1;
  const long n = (long)h->samples.size();
  if (dst)
    for (long i = 0; i < n && i < cap; ++i) dst[i] = h->samples[i];
  return n;
}

lbm_status lbm_solid_create(const lbm_solid_desc *d, void *stream, lbm_solid **out) {
  if (!out || !d) return LBM_ERR_ARG;
  *out = nullptr;
  if (d->nx < 3 || d->ny < 3) return LBM_ERR_ARG;
  if ((long)d->nx * d->ny > (1L << 31) / 8) return LBM_ERR_ARG;  // 8N plane offsets fit int64 and index math
  if (!(d->dx > 0.0) || !std::isfinite(d->dx)) return LBM_ERR_ARG;
  if (d->control < LBM_CTRL_FORCE_FIELD || d->control > LBM_CTRL_YOUNG_FIELD) return LBM_ERR_ARG;
  if (d->kernel != LBM_KERNEL_AUTO && d->kernel != LBM_KERNEL_FP64) return LBM_ERR_ARG;
  if (d->control == LBM_CTRL_FORCE_BASIS2 && !d->force_basis) return LBM_ERR_ARG;
  lbm_solid *h = new (std::nothrow) lbm_solid();
  if (!h) return LBM_ERR_OOM;
  h->nx = d->nx; h->ny = d->ny; h->N = (long)d->nx * d->ny; h->dx = d->dx;
  h->periodic = d->periodic ? 1 : 0; h->nu = d->nu; h->control = d->control; h->kernel = d->kernel;
  h->stream = (cudaStream_t)stream;
  h->grid = Grid{d->nx, d->ny, h->N};
  const long N = h->N;
  auto bail = [&](lbm_status st) { free_all(h); delete h; return st; };

  // ---- geometry (host validation, compact boundary records) -----------------------
  std::vector<uint8_t> type(N, 1);
  std::vector<int> bidx(N, -1);
  std::vector<BoundaryNode> bn;
  std::vector<uint8_t> regm, negm;
  std::vector<int> bnode_h;
  std::vector<int2> chunks;
  if (h->periodic) {
    if (d->link_bc) return bail(LBM_ERR_ARG);
    if (d->node_mask)
      for (long n = 0; n < N; ++n)
        if (d->node_mask[n] != 1) return bail(LBM_ERR_ARG);
    h->n_active = N;
  } else {
    if (!d->link_bc) return bail(LBM_ERR_ARG);
    for (long n = 0; n < N; ++n) type[n] = d->node_mask ? (d->node_mask[n] ? 1 : 0) : 1;
    const int cx[8] = {1, 0, -1, 0, 1, -1, -1, 1}, cy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
    h->n_active = 0;
    for (long n = 0; n < N; ++n) {
      if (!type[n]) continue;
      ++h->n_active;
      const int x = (int)(n % d->nx), y = (int)(n / d->nx);
      BoundaryNode b{};
      uint8_t reg = 0, neg = 0;
      bool any = false;
      for (int k = 0; k < 8; ++k) {
        const int xs = x - cx[k], ys = y - cy[k];
        const bool src_active = xs >= 0 && xs < d->nx && ys >= 0 && ys < d->ny &&
                                type[(long)ys * d->nx + xs] != 0;
        const uint8_t code = d->link_bc[(long)k * N + n];
        if (code > 2) return bail(LBM_ERR_ARG);
        if (src_active != (code == 0)) return bail(LBM_ERR_ARG);
        b.code[k] = code;
        if (code == 0) reg |= (uint8_t)(1u << k);
        if (code == 2) neg |= (uint8_t)(1u << k);
        if (code == 1) {
          if (!d->wall_d) return bail(LBM_ERR_ARG);
          b.wd[0] = d->wall_d[n]; b.wd[1] = d->wall_d[N + n];
        }
        if (code == 2) {
          if (!d->wall_T || !d->wall_n) return bail(LBM_ERR_ARG);
          b.T[0] = d->wall_T[n]; b.T[1] = d->wall_T[N + n];
          b.nrm[0] = d->wall_n[n]; b.nrm[1] = d->wall_n[N + n];
          h->has_neumann = true;
        }
        any |= code != 0;
      }
      if (any) {
        type[n] = 2;
        bidx[n] = (int)bn.size();
        bn.push_back(b);
        regm.push_back(reg);
        negm.push_back(neg);
        bnode_h.push_back((int)n);
      }
    }
    if (h->n_active == 0) return bail(LBM_ERR_ARG);
    // interior nodes as chunks of up to 32 consecutive nodes of one row
    for (int y = 0; y < d->ny; ++y) {
      int x = 0;
      while (x < d->nx) {
        if (type[(long)y * d->nx + x] != 1) { ++x; continue; }
        int e = x;
        while (e < d->nx && e - x < 32 && type[(long)y * d->nx + e] == 1) ++e;
        chunks.push_back(make_int2((int)((long)y * d->nx + x), e - x));
        x = e;
      }
    }
  }
  h->nb = (long)bn.size();

  // ---- device buffers ---------------------------------------------------------------
  const size_t pop = sizeof(double) * 8 * N, two = sizeof(double) * 2 * N;
  unsigned bx = 128;
  while (bx > 32 && bx / 2 >= (unsigned)d->nx) bx /= 2;
  h->blk = dim3(bx, 256 / bx);
  h->grd = dim3((d->nx + h->blk.x - 1) / h->blk.x, (d->ny + h->blk.y - 1) / h->blk.y);
  // small lattices are latency-bound: smaller blocks spread the nodes (and the FP64
  // boundary nodes) over more of the 148 SMs
  while ((long)h->grd.x * h->grd.y < 148 && h->blk.x * h->blk.y > 64) {
    if (h->blk.y > 1) h->blk.y /= 2;
    else h->blk.x /= 2;
    h->grd = dim3((d->nx + h->blk.x - 1) / h->blk.x, (d->ny + h->blk.y - 1) / h->blk.y);
  }
  h->nblocks2d = (long)h->grd.x * h->grd.y;
  h->nmon = h->nblocks2d;
  if (!h->periodic) {
    h->ctpb = compact_block_size(h->nb, (long)chunks.size());
    h->hoist = compact_hoist(h->nb, (long)chunks.size());
    const long bblocks = (h->nb + h->ctpb - 1) / h->ctpb;
    const long cw = h->ctpb / 32;
    h->cblocks = bblocks + ((long)chunks.size() + cw - 1) / cw;
    h->nmon = h->cblocks;
    h->cmp.nchunk = (long)chunks.size();
    h->cmp.nb = h->nb;
    h->cmp.bblocks = (int)bblocks;
  }
  long pmax = h->nblocks2d > h->cblocks ? h->nblocks2d : h->cblocks;
  if (pmax < 148 * 8) pmax = 148 * 8;
  h->partial_cap = 4 * pmax;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes))
  ALLOC(h->fA, pop); ALLOC(h->fB, pop); ALLOC(h->pA, pop); ALLOC(h->pB, pop);
  ALLOC(h->g2, two); ALLOC(h->r2, two); ALLOC(h->dstar, two);
  ALLOC(h->partial, sizeof(double) * h->partial_cap);
  ALLOC(h->dres, sizeof(double) * 8);
  if (d->obs_mask) ALLOC(h->obs, sizeof(double) * N);
  if (d->control == LBM_CTRL_FORCE_BASIS2) ALLOC(h->basis, 2 * two);
  if (d->control >= LBM_CTRL_YOUNG_SCALAR) ALLOC(h->Fbase, two);
  h->field = d->control == LBM_CTRL_YOUNG_FIELD;
  if (h->field) {
    ALLOC(h->qfield, 3 * sizeof(double) * N);
    ALLOC(h->qfix, 3 * sizeof(FixC) * N);
    ALLOC(h->alphaN, sizeof(double) * N);
    if (!h->periodic && h->nb) {
      ALLOC(h->gamf, sizeof(double) * h->nb);
      ALLOC(h->bfix, 2 * sizeof(FixC) * h->nb);
      ALLOC(h->bok, h->nb);
    }
  }
  if (!h->periodic) {
    ALLOC(h->type, N);
    ALLOC(h->bidx, sizeof(int) * N);
    if (!chunks.empty()) ALLOC(h->chunk, sizeof(int2) * chunks.size());
    if (h->nb) {
      ALLOC(h->regmask, h->nb);
      ALLOC(h->negmask, h->nb);
      ALLOC(h->bnode, sizeof(int) * h->nb);
      ALLOC(h->R, sizeof(double) * 32 * h->nb);
      ALLOC(h->bnodes, sizeof(BoundaryNode) * h->nb);
      ALLOC(h->Q, sizeof(double) * 64 * h->nb);
      ALLOC(h->s, sizeof(double) * 8 * h->nb);
      if (d->control >= LBM_CTRL_YOUNG_SCALAR) {
        ALLOC(h->dQ, sizeof(double) * 64 * h->nb);
        ALLOC(h->ds, sizeof(double) * 8 * h->nb);
      }
    }
  }
#undef ALLOC
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hres, sizeof(double) * 8);
  if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA);

  // ---- uploads (synchronous: desc arrays are pageable host memory) -----------------
  auto up = [&](void *dst, const void *src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  if (d->obs_mask) {
    std::vector<double> ob(d->obs_mask, d->obs_mask + N);
    for (long n = 0; n < N; ++n)
      if (!type[n]) ob[n] = 0.0;
    up(h->obs, ob.data(), sizeof(double) * N);
  }
  if (h->basis) {
    std::vector<double> bs(d->force_basis, d->force_basis + 4 * N);
    up(h->basis, bs.data(), 2 * two);
  }
  if (!h->periodic) {
    up(h->type, type.data(), N);
    up(h->bidx, bidx.data(), sizeof(int) * N);
    if (h->nb) {
      up(h->regmask, regm.data(), h->nb);
      up(h->negmask, negm.data(), h->nb);
      up(h->bnodes, bn.data(), sizeof(BoundaryNode) * h->nb);
      up(h->bnode, bnode_h.data(), sizeof(int) * h->nb);
    }
    if (!chunks.empty()) up(h->chunk, chunks.data(), sizeof(int2) * chunks.size());
    h->bnd = Bounded{h->type, h->bidx, h->Q, h->s, h->regmask, h->dQ, h->ds};
    h->cmp.chunk = h->chunk;
    h->cmp.bnode = h->bnode;
    h->cmp.R = h->R;
    h->cmp.negmask = h->negmask;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->fA, 0, pop, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->fB, 0, pop, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->pA, 0, pop, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->pB, 0, pop, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->g2, 0, two, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->r2, 0, two, h->stream);
  if (e != cudaSuccess) return bail(LBM_ERR_CUDA);
  h->fcur = h->fA; h->fnext = h->fB; h->pcur = h->pA; h->pnext = h->pB;
  h->fcur_is_fs = true;

  // ---- material and fixed force -----------------------------------------------------
  if (set_material(h, d->E) != LBM_OK) return bail(LBM_ERR_ARG);
  if (h->field) {
    // uniform start: alpha_n = sqrt(E) everywhere
    std::vector<double> a0(N, std::sqrt(d->E));
    up(h->alphaN, a0.data(), sizeof(double) * N);
    if (e != cudaSuccess) return bail(LBM_ERR_CUDA);
    h->fl = Field{h->qfield, h->qfix, h->gamf, h->bfix, h->bok, h->alphaN, h->nu};
    if (set_field(h) != LBM_OK) return bail(LBM_ERR_CUDA);
  }
  if (h->Fbase) {
    if (d->force) {
      std::vector<double> F(d->force, d->force + 2 * N);
      for (long n = 0; n < N; ++n)
        if (!type[n]) F[n] = F[N + n] = 0.0;
      up(h->Fbase, F.data(), two);
      if (e != cudaSuccess) return bail(LBM_ERR_CUDA);
    } else if (cudaMemsetAsync(h->Fbase, 0, two, h->stream) != cudaSuccess) {
      return bail(LBM_ERR_CUDA);
    }
    k_set_force<<<148 * 4, 256, 0, h->stream>>>(h->g2, h->Fbase, nullptr, nullptr, 0.25 * h->dx * h->dx, N,
                                              h->periodic ? nullptr : h->type);
    ++h->launches;
    if (cudaGetLastError() != cudaSuccess) return bail(LBM_ERR_CUDA);
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(LBM_ERR_CUDA);
  if (h->periodic) {
    h->cw = ClusterWork{nullptr, N};
    setup_cluster(h, N);
    if (h->cl_ncta == 0) setup_dsm(h);
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_solid_destroy(lbm_solid *h) {
  if (!h) return LBM_ERR_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  for (auto &g : h->loops) cudaGraphExecDestroy(g.exec);
  h->loops.clear();
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->dloop) cudaFree(h->dloop);
  if (h->hloop) cudaFreeHost(h->hloop);
  free_all(h);
  delete h;
  return LBM_OK;
}

lbm_status lbm_solid_set_control(lbm_solid *h, const double *alpha, size_t n, int keep_state) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!alpha) return fail(h, LBM_ERR_ARG, "alpha is NULL");
  const double dx2 = 0.25 * h->dx * h->dx;  // q = g / 4
  const uint8_t *tp = h->periodic ? nullptr : h->type;
  switch (h->control) {
    case LBM_CTRL_FORCE_FIELD:
      if (n != (size_t)(2 * h->N)) return fail(h, LBM_ERR_ARG, "FORCE_FIELD control needs 2N values");
      k_set_force<<<148 * 4, 256, 0, h->stream>>>(h->g2, alpha, nullptr, nullptr, dx2, h->N, tp);
      LAUNCHED(h);
      break;
    case LBM_CTRL_FORCE_BASIS2:
      if (n != 2) return fail(h, LBM_ERR_ARG, "FORCE_BASIS2 control needs 2 values");
      k_set_force<<<148 * 4, 256, 0, h->stream>>>(h->g2, nullptr, h->basis, alpha, dx2, h->N, tp);
      LAUNCHED(h);
      break;
    case LBM_CTRL_YOUNG_SCALAR: {
      if (n != 1) return fail(h, LBM_ERR_ARG, "YOUNG_SCALAR control needs 1 value");
      CK(h, cudaMemcpyAsync(h->hres, alpha, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(h, cudaStreamSynchronize(h->stream));
      const lbm_status st = set_material(h, h->hres[0] * h->hres[0]);
      if (st) return st;
      h->alpha = h->hres[0];
      break;
    }
    case LBM_CTRL_YOUNG_FIELD: {
      if (n != (size_t)h->N) return fail(h, LBM_ERR_ARG, "YOUNG_FIELD control needs N values");
      // validate on the host: every active modulus alpha_n^2 must give a valid material
      std::vector<double> a(h->N), tp(h->N, 1.0);
      CK(h, cudaMemcpyAsync(a.data(), alpha, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
      std::vector<uint8_t> ty;
      if (!h->periodic) {
        ty.resize(h->N);
        CK(h, cudaMemcpyAsync(ty.data(), h->type, h->N, cudaMemcpyDeviceToHost, h->stream));
      }
      CK(h, cudaStreamSynchronize(h->stream));
      for (long i = 0; i < h->N; ++i) {
        if (!h->periodic && ty[i] == 0) continue;
        Coef c{};
        Material m{};
        YoungDeriv yd{};
        std::string why;
        if (!material_coefs(a[i] * a[i], h->nu, !h->periodic && ty[i] == 2, h->has_neumann, c, m, yd, why))
          return fail(h, LBM_ERR_ARG, "node " + std::to_string(i) + ": " + why);
      }
      CK(h, cudaMemcpyAsync(h->alphaN, alpha, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->stream));
      const lbm_status st = set_field(h);
      if (st) return st;
      break;
    }
    default:
      return fail(h, LBM_ERR_ARG, "unsupported control kind");
  }
  if (!keep_state) {
    CK(h, cudaMemsetAsync(h->fcur, 0, sizeof(double) * 8 * h->N, h->stream));
    h->fcur_is_fs = true;
  }
  ++h->pstate;
  h->adjoint_valid = false;
  h->adj_warm = false;
  return LBM_OK;
}

lbm_status lbm_solid_set_target(lbm_solid *h, const double *dstar) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!dstar) return fail(h, LBM_ERR_ARG, "dstar is NULL");
  CK(h, cudaMemcpyAsync(h->dstar, dstar, sizeof(double) * 2 * h->N, cudaMemcpyDeviceToDevice, h->stream));
  long blocks = (h->N + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (h->periodic)
    k_cbar<false><<<(unsigned)blocks, 256, 0, h->stream>>>(h->dstar, h->obs, h->grid, h->bnd, h->partial);
  else
    k_cbar<true><<<(unsigned)blocks, 256, 0, h->stream>>>(h->dstar, h->obs, h->grid, h->bnd, h->partial);
  LAUNCHED(h);
  lbm_status st = finish(h, blocks, 1, 0, h->dx * h->dx, h->dres);
  if (st) return st;
  if ((st = fetch(h, 1))) return st;
  if (!(h->hres[0] > 0.0) || !std::isfinite(h->hres[0]))
    return fail(h, LBM_ERR_ARG, "target has zero norm on the observation domain (Cbar = 0)");
  h->cbar = h->hres[0];
  ++h->pstate;
  h->have_target = true;
  h->adjoint_valid = false;
  return LBM_OK;
}

lbm_status lbm_solid_primal_solve(lbm_solid *h, const lbm_solve_opts *o, lbm_solve_info *info) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  lbm_status st = check_opts(h, o);
  if (st) return st;
  h->adjoint_valid = false;
  h->adj_warm = false;
  auto resid = [h](double &v) { return residual(h, h->fcur, h->fnext, v); };
  return solve_loop(h, o, info, 0, resid);
}

lbm_status lbm_solid_objective(lbm_solid *h, double *J) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!J) return fail(h, LBM_ERR_ARG, "J is NULL");
  if (!h->have_target) return fail(h, LBM_ERR_STATE, "objective needs set_target first");
  lbm_status st = objective_partials(h);
  if (st) return st;
  if ((st = finish(h, h->obj_parts, 1, 0, 0.5 * h->dx * h->dx / h->cbar, h->dres))) return st;
  if ((st = fetch(h, 1))) return st;
  *J = h->hres[0];
  return LBM_OK;
}

lbm_status lbm_solid_adjoint_source(lbm_solid *h, double *r) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!r) return fail(h, LBM_ERR_ARG, "r is NULL");
  if (!h->have_target) return fail(h, LBM_ERR_STATE, "adjoint_source needs set_target first");
  lbm_status st = objective_partials(h);
  if (st) return st;
  CK(h, cudaMemcpyAsync(r, h->r2, sizeof(double) * 2 * h->N, cudaMemcpyDeviceToDevice, h->stream));
  return LBM_OK;
}

lbm_status lbm_solid_adjoint_solve(lbm_solid *h, const lbm_solve_opts *o, lbm_solve_info *info) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  lbm_status st = check_opts(h, o);
  if (st) return st;
  if (!h->have_target) return fail(h, LBM_ERR_STATE, "adjoint needs set_target first");
  // constant terms of Algorithm 1: r from the current primal state (unless the last
  // objective already computed it for this state)
  if (h->r_at != h->pstate && (st = objective_partials(h))) return st;
  h->pcur_rest = !h->adj_warm;  // from rest: the first sweep writes -j directly
  h->adj_warm = false;
  auto resid = [h](double &v) { return residual(h, h->pcur, h->pnext, v); };
  st = solve_loop(h, o, info, 1, resid);
  if (st == LBM_OK || st == LBM_ERR_NOT_CONVERGED) h->adjoint_valid = true;
  return st;
}

lbm_status lbm_solid_gradient(lbm_solid *h, double *grad, size_t n, int project) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!grad) return fail(h, LBM_ERR_ARG, "grad is NULL");
  if (!h->adjoint_valid) return fail(h, LBM_ERR_STATE, "gradient needs an adjoint solve at the current primal state");
  const double dx2 = h->dx * h->dx;
  const bool fix = h->kernel != LBM_KERNEL_FP64;  // integer-pipe pass (periodic lattices)
  lbm_status st;
  if (h->control == LBM_CTRL_FORCE_FIELD) {
    if (n != (size_t)(2 * h->N)) return fail(h, LBM_ERR_ARG, "FORCE_FIELD gradient has 2N values");
    long parts = h->nblocks2d;
    if (h->periodic && fix) {
      parts = kFixPassBlocks;
      k_grad_force_fix<0><<<kFixPassBlocks, 256, 0, h->stream>>>(h->pcur, h->r2, nullptr, grad, dx2, h->grid, h->partial);
    } else if (h->periodic) {
      k_grad_force<false, 0><<<h->grd, h->blk, 0, h->stream>>>(h->pcur, h->r2, nullptr, grad, dx2, h->grid, h->bnd, h->partial);
    } else {
      k_grad_force<true, 0><<<h->grd, h->blk, 0, h->stream>>>(h->pcur, h->r2, nullptr, grad, dx2, h->grid, h->bnd, h->partial);
    }
    LAUNCHED(h);
    if (project) {
      if ((st = finish(h, parts, 2, 0, 1.0 / (double)h->n_active, h->dres))) return st;
      if (h->periodic)
        k_subtract_mean<false><<<h->grd, h->blk, 0, h->stream>>>(grad, h->dres, h->grid, h->bnd);
      else
        k_subtract_mean<true><<<h->grd, h->blk, 0, h->stream>>>(grad, h->dres, h->grid, h->bnd);
      LAUNCHED(h);
    }
    return LBM_OK;
  }
  if (h->control == LBM_CTRL_FORCE_BASIS2) {
    if (n != 2) return fail(h, LBM_ERR_ARG, "FORCE_BASIS2 gradient has 2 values");
    long parts = h->nblocks2d;
    if (h->periodic && fix) {
      parts = kFixPassBlocks;
      k_grad_force_fix<1><<<kFixPassBlocks, 256, 0, h->stream>>>(h->pcur, h->r2, h->basis, nullptr, dx2, h->grid, h->partial);
    } else if (h->periodic) {
      k_grad_force<false, 1><<<h->grd, h->blk, 0, h->stream>>>(h->pcur, h->r2, h->basis, nullptr, dx2, h->grid, h->bnd, h->partial);
    } else {
      k_grad_force<true, 1><<<h->grd, h->blk, 0, h->stream>>>(h->pcur, h->r2, h->basis, nullptr, dx2, h->grid, h->bnd, h->partial);
    }
    LAUNCHED(h);
    return finish(h, parts, 2, 0, 1.0, grad);
  }
  if (h->control == LBM_CTRL_YOUNG_SCALAR) {
    if (n != 1) return fail(h, LBM_ERR_ARG, "YOUNG_SCALAR gradient has 1 value");
    if (h->fcur_is_fs) return fail(h, LBM_ERR_STATE, "Young gradient needs a primal solve");
    if (h->periodic)
      k_grad_young<false, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->pcur, h->grid, h->bnd, h->coef, h->yd, h->fl, nullptr, h->partial);
    else
      k_grad_young<true, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->pcur, h->grid, h->bnd, h->coef, h->yd, h->fl, nullptr, h->partial);
    LAUNCHED(h);
    // E = alpha^2 (Eq. E_substitution): dJ/dalpha = 2 alpha dJ/dE
    return finish(h, h->nblocks2d, 1, 0, 2.0 * h->alpha, grad);
  }
  if (h->control == LBM_CTRL_YOUNG_FIELD) {
    if (n != (size_t)h->N) return fail(h, LBM_ERR_ARG, "YOUNG_FIELD gradient has N values");
    if (h->fcur_is_fs) return fail(h, LBM_ERR_STATE, "Young gradient needs a primal solve");
    if (h->periodic)
      k_grad_young<false, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->pcur, h->grid, h->bnd, h->coef, h->yd, h->fl, grad, nullptr);
    else
      k_grad_young<true, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->pcur, h->grid, h->bnd, h->coef, h->yd, h->fl, grad, nullptr);
    LAUNCHED(h);
    return LBM_OK;
  }
  return fail(h, LBM_ERR_ARG, "gradient for this control kind is not built");
}

lbm_status lbm_solid_tangent(lbm_solid *h, const double *seed, size_t n,
                             const lbm_solve_opts *o, double *dJ, lbm_solve_info *info) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!seed || !dJ) return fail(h, LBM_ERR_ARG, "seed or dJ is NULL");
  lbm_status st = check_opts(h, o);
  if (st) return st;
  if (!h->have_target) return fail(h, LBM_ERR_STATE, "tangent needs set_target first");
  if (h->fcur_is_fs) return fail(h, LBM_ERR_STATE, "tangent needs a primal solve");
  const long N = h->N;
  const size_t pop = sizeof(double) * 8 * N;
  if (!h->tA) {
    CK(h, cudaMalloc(&h->tA, pop));
    CK(h, cudaMalloc(&h->tB, pop));
    CK(h, cudaMalloc(&h->qdot, sizeof(double) * 2 * N));
  }
  const uint8_t *tp = h->periodic ? nullptr : h->type;
  const double q4 = 0.25 * h->dx * h->dx;
  bool young = false;
  double Edot = 0.0;
  if (h->control == LBM_CTRL_FORCE_FIELD) {
    if (n != (size_t)(2 * N)) return fail(h, LBM_ERR_ARG, "FORCE_FIELD seed has 2N values");
    k_set_force<<<148 * 4, 256, 0, h->stream>>>(h->qdot, seed, nullptr, nullptr, q4, N, tp);
    LAUNCHED(h);
  } else if (h->control == LBM_CTRL_FORCE_BASIS2) {
    if (n != 2) return fail(h, LBM_ERR_ARG, "FORCE_BASIS2 seed has 2 values");
    k_set_force<<<148 * 4, 256, 0, h->stream>>>(h->qdot, nullptr, h->basis, seed, q4, N, tp);
    LAUNCHED(h);
  } else if (h->control == LBM_CTRL_YOUNG_SCALAR) {
    if (n != 1) return fail(h, LBM_ERR_ARG, "YOUNG_SCALAR seed has 1 value");
    CK(h, cudaMemcpyAsync(h->hres, seed, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    young = true;
    Edot = 2.0 * h->alpha * h->hres[0];  // E = alpha^2
  } else {
    return fail(h, LBM_ERR_ARG, "tangent is built for force controls and the scalar modulus");
  }
  const double *qd = young ? nullptr : h->qdot;
  // both buffers: the sweep never writes inactive nodes, which the residual still reads
  CK(h, cudaMemsetAsync(h->tA, 0, pop, h->stream));
  CK(h, cudaMemsetAsync(h->tB, 0, pop, h->stream));
  double *tcur = h->tA, *tnext = h->tB;
  const auto t0 = std::chrono::steady_clock::now();
  auto sweep = [&]() -> lbm_status {
    if (h->periodic) {
      if (young) k_tangent<false, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, tcur, tnext, qd, h->grid, h->bnd, h->coef, h->yd, Edot);
      else k_tangent<false, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, tcur, tnext, qd, h->grid, h->bnd, h->coef, h->yd, Edot);
    } else {
      if (young) k_tangent<true, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, tcur, tnext, qd, h->grid, h->bnd, h->coef, h->yd, Edot);
      else k_tangent<true, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, tcur, tnext, qd, h->grid, h->bnd, h->coef, h->yd, Edot);
    }
    LAUNCHED(h);
    std::swap(tcur, tnext);
    return LBM_OK;
  };
  long steps = 0;
  double metric = 0.0;
  lbm_status result = LBM_OK;
  if (o->fixed_steps) {
    for (; steps < o->max_steps; ++steps)
      if ((st = sweep())) return st;
  } else {
    bool done = false;
    while (!done && steps < o->max_steps) {
      long k = o->check_every < o->max_steps - steps ? o->check_every : o->max_steps - steps;
      for (long i = 0; i < k; ++i)
        if ((st = sweep())) return st;
      steps += k;
      if (steps < 2) continue;
      if ((st = residual(h, tcur, tnext, metric))) return st;
      if (std::isnan(metric)) { result = LBM_ERR_DIVERGED; break; }
      if (metric < o->tol) done = true;
    }
    if (result == LBM_OK && !done) result = LBM_ERR_NOT_CONVERGED;
  }
  if (h->periodic) {
    if (young) k_tangent_objective<false, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, tcur, h->g2, qd, h->dstar, h->obs, h->grid, h->bnd, Edot, h->partial);
    else k_tangent_objective<false, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, tcur, h->g2, qd, h->dstar, h->obs, h->grid, h->bnd, Edot, h->partial);
  } else {
    if (young) k_tangent_objective<true, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, tcur, h->g2, qd, h->dstar, h->obs, h->grid, h->bnd, Edot, h->partial);
    else k_tangent_objective<true, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, tcur, h->g2, qd, h->dstar, h->obs, h->grid, h->bnd, Edot, h->partial);
  }
  LAUNCHED(h);
  if ((st = finish(h, h->nblocks2d, 1, 0, h->dx * h->dx / h->cbar, h->dres))) return st;
  if ((st = fetch(h, 1))) return st;
  *dJ = h->hres[0];
  if (info) {
    info->steps = steps;
    info->last_metric = metric;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (result == LBM_ERR_NOT_CONVERGED) h->err = "max_steps reached before the stopping rule held";
  if (result == LBM_ERR_DIVERGED) h->err = "non-finite tangent residual";
  return result;
}

lbm_status lbm_solid_get_populations(lbm_solid *h, int which, double *dst) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!dst) return fail(h, LBM_ERR_ARG, "dst is NULL");
  const size_t pop = sizeof(double) * 8 * h->N;
  if (which == 0) {
    if (h->fcur_is_fs) {
      CK(h, cudaMemcpyAsync(dst, h->fcur, pop, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      if (h->periodic)
        k_pull_primal<false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, dst, h->grid, h->bnd);
      else
        k_pull_primal<true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, dst, h->grid, h->bnd);
      LAUNCHED(h);
    }
    return LBM_OK;
  }
  if (which == 1) {
    if (h->periodic)
      k_pull_adjoint<false><<<h->grd, h->blk, 0, h->stream>>>(h->pcur, dst, h->grid, h->bnd);
    else
      k_pull_adjoint<true><<<h->grd, h->blk, 0, h->stream>>>(h->pcur, dst, h->grid, h->bnd);
    LAUNCHED(h);
    return LBM_OK;
  }
  if (which == 2) {
    CK(h, cudaMemcpyAsync(dst, h->pcur, pop, cudaMemcpyDeviceToDevice, h->stream));
    return LBM_OK;
  }
  return fail(h, LBM_ERR_ARG, "which must be 0, 1 or 2");
}

lbm_status lbm_solid_set_populations(lbm_solid *h, int which, const double *src) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!src) return fail(h, LBM_ERR_ARG, "src is NULL");
  const size_t pop = sizeof(double) * 8 * h->N;
  if (which == 0) {
    CK(h, cudaMemcpyAsync(h->fcur, src, pop, cudaMemcpyDeviceToDevice, h->stream));
    h->fcur_is_fs = true;
    ++h->pstate;
    h->adjoint_valid = false;
    return LBM_OK;
  }
  if (which == 2) {
    CK(h, cudaMemcpyAsync(h->pcur, src, pop, cudaMemcpyDeviceToDevice, h->stream));
    h->adj_warm = true;
    h->pcur_rest = false;
    return LBM_OK;
  }
  return fail(h, LBM_ERR_ARG, "which must be 0 (f_S) or 2 (phi_C)");
}

lbm_status lbm_solid_displacement(lbm_solid *h, double *d) {
  if (!h) return LBM_ERR_ARG;
  if (h->broken) return fail(h, LBM_ERR_CUDA, "handle unusable after a CUDA error");
  if (!d) return fail(h, LBM_ERR_ARG, "d is NULL");
  if (h->periodic) {
    if (h->fcur_is_fs)
      k_displacement<false, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->g2, d, h->grid, h->bnd);
    else
      k_displacement<false, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->g2, d, h->grid, h->bnd);
  } else {
    if (h->fcur_is_fs)
      k_displacement<true, false><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->g2, d, h->grid, h->bnd);
    else
      k_displacement<true, true><<<h->grd, h->blk, 0, h->stream>>>(h->fcur, h->g2, d, h->grid, h->bnd);
  }
  LAUNCHED(h);
  return LBM_OK;
}

}  // extern "C"

// ---- Batches of one bounded geometry (per-instance modulus fields) ------------------
struct lbm_plate_batch {
  lbm_solid *geo = nullptr;  // geometry, compact lists, shared force and constants
  int count = 0;
  cudaStream_t stream = nullptr, cap = nullptr;
  double *fA = nullptr, *fB = nullptr, *fcur = nullptr, *fnext = nullptr;
  bool fs = true;  // fcur holds explicit f_S (all instances)
  double *q = nullptr, *alpha = nullptr, *gam = nullptr, *R = nullptr;
  FixC *qfix = nullptr, *bfix = nullptr;
  uint8_t *bok = nullptr;
  Field fl{};
  Compact cmp{};
  struct G {
    long k;
    int parity;
    cudaGraphExec_t exec;
  };
  std::vector<G> graphs;
};

namespace {

void plate_batch_free(lbm_plate_batch *b) {
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  void *bufs[] = {b->fA, b->fB, b->q, b->alpha, b->gam, b->R, b->qfix, b->bfix, b->bok};
  for (void *p : bufs)
    if (p) cudaFree(p);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->geo) lbm_solid_destroy(b->geo);
}

void plate_batch_sweep(lbm_plate_batch *b, cudaStream_t st) {
  lbm_solid *h = b->geo;
  const dim3 grid((unsigned)h->cblocks, (unsigned)b->count);
  if (h->kernel == LBM_KERNEL_FP64)
    k_primal_cb<0><<<grid, h->ctpb, 0, st>>>(b->fcur, b->fnext, h->g2, h->grid, h->bnd, b->cmp, h->coef, b->fl);
  else
    k_primal_cb<1><<<grid, h->ctpb, 0, st>>>(b->fcur, b->fnext, h->g2, h->grid, h->bnd, b->cmp, h->coef, b->fl);
  std::swap(b->fcur, b->fnext);
}

}  // namespace

extern "C" {

lbm_status lbm_plate_batch_create(const lbm_solid_desc *d, int count, void *stream,
                                  lbm_plate_batch **out) {
  if (!out || !d) return LBM_ERR_ARG;
  *out = nullptr;
  if (d->periodic || d->control != LBM_CTRL_YOUNG_FIELD || count < 1 || count > 65535)
    return LBM_ERR_ARG;
  lbm_plate_batch *b = new (std::nothrow) lbm_plate_batch();
  if (!b) return LBM_ERR_OOM;
  b->count = count;
  b->stream = (cudaStream_t)stream;
  lbm_status st = lbm_solid_create(d, stream, &b->geo);
  if (st != LBM_OK) {
    b->geo = nullptr;
    delete b;
    return st;
  }
  lbm_solid *h = b->geo;
  const long N = h->N, nb = h->nb, C = count;
  if ((long)h->cblocks > 0x7fffffffL || 8 * N * C > (1L << 40)) {
    plate_batch_free(b);
    delete b;
    return LBM_ERR_ARG;
  }
  cudaError_t e = cudaSuccess;
#define PALLOC(ptr, bytes) \
  if (e == cudaSuccess && (bytes) > 0) e = cudaMalloc((void **)&(ptr), (bytes))
  PALLOC(b->fA, sizeof(double) * 8 * N * C);
  PALLOC(b->fB, sizeof(double) * 8 * N * C);
  PALLOC(b->q, sizeof(double) * 3 * N * C);
  PALLOC(b->qfix, sizeof(FixC) * 3 * N * C);
  PALLOC(b->alpha, sizeof(double) * N * C);
  PALLOC(b->gam, sizeof(double) * nb * C);
  PALLOC(b->R, sizeof(double) * 32 * nb * C);
  PALLOC(b->bfix, sizeof(FixC) * 2 * nb * C);
  PALLOC(b->bok, nb * C);
#undef PALLOC
  if (e == cudaSuccess) e = cudaMemsetAsync(b->fA, 0, sizeof(double) * 8 * N * C, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->fB, 0, sizeof(double) * 8 * N * C, b->stream);
  if (e != cudaSuccess) {
    plate_batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
  }
  b->fcur = b->fA;
  b->fnext = b->fB;
  b->fl = Field{b->q, b->qfix, b->gam, b->bfix, b->bok, b->alpha, h->nu};
  b->cmp = h->cmp;
  b->cmp.R = b->R;
  // initial control: the description's modulus everywhere
  std::vector<double> a0((size_t)(N * C), std::sqrt(d->E));
  double *tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(double) * N * C) != cudaSuccess) {
    plate_batch_free(b);
    delete b;
    return LBM_ERR_OOM;
  }
  st = cudaMemcpy(tmp, a0.data(), sizeof(double) * N * C, cudaMemcpyHostToDevice) == cudaSuccess
           ? lbm_plate_batch_set_control(b, tmp)
           : LBM_ERR_CUDA;
  cudaStreamSynchronize(b->stream);
  cudaFree(tmp);
  if (st != LBM_OK) {
    plate_batch_free(b);
    delete b;
    return st;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_plate_batch_destroy(lbm_plate_batch *b) {
  if (!b) return LBM_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  plate_batch_free(b);
  delete b;
  return LBM_OK;
}

lbm_status lbm_plate_batch_set_control(lbm_plate_batch *b, const double *alpha) {
  if (!b || !alpha) return LBM_ERR_ARG;
  lbm_solid *h = b->geo;
  const long N = h->N, nb = h->nb, C = b->count;
  // validate on the host: every active modulus alpha^2 must give a valid material
  std::vector<double> a((size_t)(N * C));
  std::vector<uint8_t> ty((size_t)N);
  if (cudaMemcpyAsync(a.data(), alpha, sizeof(double) * N * C, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(ty.data(), h->type, N, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  for (long i = 0; i < N * C; ++i) {
    const uint8_t t = ty[i % N];
    if (t == 0) continue;
    Coef c{};
    Material m{};
    YoungDeriv yd{};
    std::string why;
    if (!material_coefs(a[i] * a[i], h->nu, t == 2, h->has_neumann, c, m, yd, why)) return LBM_ERR_ARG;
  }
  if (cudaMemcpyAsync(b->alpha, alpha, sizeof(double) * N * C, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  for (long i = 0; i < C; ++i) {
    k_set_young_field<<<148 * 4, 256, 0, b->stream>>>(b->alpha + N * i, h->nu, N, b->q + 3 * N * i, b->qfix + 3 * N * i);
    if (nb) {
      const unsigned blocks = (unsigned)((nb + 127) / 128);
      k_boundary_setup<<<blocks, 128, 0, b->stream>>>(
          h->bnodes, nb, h->mat, h->dx, nullptr, nullptr, nullptr, nullptr, b->alpha + N * i,
          h->bnode, h->nu, b->gam + nb * i, b->R + 32 * nb * i, nullptr, b->bfix + 2 * nb * i,
          b->bok + nb * i);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaMemsetAsync(b->fcur, 0, sizeof(double) * 8 * N * C, b->stream) != cudaSuccess) return LBM_ERR_CUDA;
  b->fs = true;
  return LBM_OK;
}

lbm_status lbm_plate_batch_primal(lbm_plate_batch *b, long sweeps) {
  if (!b || sweeps < 0) return LBM_ERR_ARG;
  lbm_solid *h = b->geo;
  if (b->fs && sweeps > 0) {  // first sweep from the explicit states
    const dim3 grid((unsigned)h->cblocks, (unsigned)b->count);
    if (h->kernel == LBM_KERNEL_FP64)
      k_collide_cb<0><<<grid, h->ctpb, 0, b->stream>>>(b->fcur, b->fnext, h->g2, h->grid, b->cmp, h->coef, b->fl);
    else
      k_collide_cb<1><<<grid, h->ctpb, 0, b->stream>>>(b->fcur, b->fnext, h->g2, h->grid, b->cmp, h->coef, b->fl);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    std::swap(b->fcur, b->fnext);
    b->fs = false;
    --sweeps;
  }
  // runs of sweeps replayed from CUDA graphs (keyed by length and buffer parity)
  constexpr long kChunk = 64;
  while (sweeps > 0) {
    const long k = sweeps >= kChunk ? kChunk : sweeps;
    if (k < 4) {
      for (long i = 0; i < k; ++i) plate_batch_sweep(b, b->stream);
      if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    } else {
      const int parity = b->fcur == b->fA ? 0 : 1;
      cudaGraphExec_t ex = nullptr;
      for (auto &g : b->graphs)
        if (g.k == k && g.parity == parity) ex = g.exec;
      if (!ex) {
        if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
          return LBM_ERR_CUDA;
        double *f0 = b->fcur, *f1 = b->fnext;
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
          return LBM_ERR_CUDA;
        for (long i = 0; i < k; ++i) plate_batch_sweep(b, b->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(b->cap, &graph);
        b->fcur = f0;
        b->fnext = f1;
        if (ec != cudaSuccess || !graph) return LBM_ERR_CUDA;
        const cudaError_t ei = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return LBM_ERR_CUDA;
        b->graphs.push_back(lbm_plate_batch::G{k, parity, ex});
      }
      if (cudaGraphLaunch(ex, b->stream) != cudaSuccess) return LBM_ERR_CUDA;
      if (k & 1) std::swap(b->fcur, b->fnext);
    }
    sweeps -= k;
  }
  return LBM_OK;
}

lbm_status lbm_plate_batch_get_populations(lbm_plate_batch *b, double *dst) {
  if (!b || !dst) return LBM_ERR_ARG;
  lbm_solid *h = b->geo;
  const size_t pop = sizeof(double) * 8 * h->N * b->count;
  if (b->fs) {
    if (cudaMemcpyAsync(dst, b->fcur, pop, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
      return LBM_ERR_CUDA;
    return LBM_OK;
  }
  if (cudaMemsetAsync(dst, 0, pop, b->stream) != cudaSuccess) return LBM_ERR_CUDA;
  const dim3 grid((unsigned)h->cblocks, (unsigned)b->count);
  k_pull_cb<<<grid, h->ctpb, 0, b->stream>>>(b->fcur, dst, h->grid, h->bnd, b->cmp);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // extern "C"
