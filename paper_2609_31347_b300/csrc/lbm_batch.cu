// Batched periodic lattices: many instances of uneven size advanced by one launch per
// sweep (a block -> instance table over all instances' tiles), replayed from CUDA graphs
// across sweeps, with per-instance objective, adjoint source and force gradient, and a
// tile-shape autotuner.  Same per-node arithmetic as the single-lattice kernels
// (lbm_kernels.cuh / lbm_fixed.cuh), so an instance of a batch reproduces the
// single-lattice result bit for bit.
//
// Layout: instance i owns nodes [off_i, off_i + N_i) of the concatenated node range;
// its population plane k is at [8 off_i + k N_i, ...), its two-component fields at
// [2 off_i + c N_i, ...).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "lbm_kernels.cuh"
#include "lbm_solid.h"

using namespace lbm;

namespace {

struct Inst {
  int nx, ny;
  long N, off;       // nodes, node offset
  long blk0;         // first block of this instance
  int tiles_x;
  double dx;
};

constexpr int kThreads = 256;

template <bool MONITOR, int ARITH>
__global__ void __launch_bounds__(kThreads) k_primal_batch(const double *__restrict__ fin,
                                                           double *__restrict__ fout,
                                                           const double *__restrict__ q,
                                                           const Inst *__restrict__ inst,
                                                           const int *__restrict__ blk_inst,
                                                           Coef c) {
  const int ib = blk_inst[blockIdx.x];
  const Inst I = inst[ib];
  const long t = blockIdx.x - I.blk0;
  const int x = (int)(t % I.tiles_x) * blockDim.x + threadIdx.x;
  const int y = (int)(t / I.tiles_x) * blockDim.y + threadIdx.y;
  if (x >= I.nx || y >= I.ny) return;
  const Grid g{I.nx, I.ny, I.N};
  const Bounded b{};
  fin += 8 * I.off;
  fout += 8 * I.off;
  q += 2 * I.off;
  const long n = (long)y * g.nx + x;
  double f[8], gsel, o[8], dxn, dyn;
  pull_primal<false>(fin, x, y, g, b, f, gsel);
  const double qx = __ldg(q + n), qy = __ldg(q + g.N + n);
  if (ARITH == 0 || !collide_fix<false, false, true, true>(f, qx, qy, c.fx, o, dxn, dyn))
    collide<false>(f, qx, qy, c, o, dxn, dyn);
#pragma unroll
  for (int k = 0; k < 8; ++k) fout[k * g.N + n] = o[k];
}

template <int ARITH>
__global__ void __launch_bounds__(kThreads) k_collide_batch(const double *__restrict__ fin,
                                                            double *__restrict__ fout,
                                                            const double *__restrict__ q,
                                                            const Inst *__restrict__ inst,
                                                            const int *__restrict__ blk_inst,
                                                            Coef c) {
  const int ib = blk_inst[blockIdx.x];
  const Inst I = inst[ib];
  const long t = blockIdx.x - I.blk0;
  const int x = (int)(t % I.tiles_x) * blockDim.x + threadIdx.x;
  const int y = (int)(t / I.tiles_x) * blockDim.y + threadIdx.y;
  if (x >= I.nx || y >= I.ny) return;
  fin += 8 * I.off;
  fout += 8 * I.off;
  q += 2 * I.off;
  const long n = (long)y * I.nx + x;
  double f[8], o[8], dxn, dyn;
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] = fin[k * I.N + n];
  if (ARITH == 0 || !collide_fix<false, false, true, true>(f, q[n], q[I.N + n], c.fx, o, dxn, dyn))
    collide<false>(f, q[n], q[I.N + n], c, o, dxn, dyn);
#pragma unroll
  for (int k = 0; k < 8; ++k) fout[k * I.N + n] = o[k];
}

template <int ARITH>
__global__ void __launch_bounds__(kThreads) k_adjoint_batch(const double *__restrict__ pin,
                                                            double *__restrict__ pout,
                                                            const double *__restrict__ r,
                                                            const Inst *__restrict__ inst,
                                                            const int *__restrict__ blk_inst,
                                                            Coef c) {
  const int ib = blk_inst[blockIdx.x];
  const Inst I = inst[ib];
  const long t = blockIdx.x - I.blk0;
  const int x = (int)(t % I.tiles_x) * blockDim.x + threadIdx.x;
  const int y = (int)(t / I.tiles_x) * blockDim.y + threadIdx.y;
  if (x >= I.nx || y >= I.ny) return;
  const Grid g{I.nx, I.ny, I.N};
  const Bounded b{};
  pin += 8 * I.off;
  pout += 8 * I.off;
  r += 2 * I.off;
  const long n = (long)y * g.nx + x;
  double p[8], gsel, o[8], ax, ay;
  pull_adjoint<false>(pin, x, y, g, b, p, gsel);
  const double rx = __ldg(r + n), ry = __ldg(r + g.N + n);
  if (ARITH == 0 || !collide_T_fix<false, false, true, true, true>(p, rx, ry, c.fx, o, ax, ay))
    collide_T<false>(p, rx, ry, c, o, ax, ay);
#pragma unroll
  for (int k = 0; k < 8; ++k) pout[k * g.N + n] = o[k];
}

// First adjoint sweep from rest: phi_C(1) = -j (the transposed collision of a zero
// state, j_k = r . c_k), written without reading the zero state.
__global__ void __launch_bounds__(kThreads) k_adjoint_rest_batch(const double *__restrict__ r,
                                                                 double *__restrict__ pout,
                                                                 const Inst *__restrict__ inst,
                                                                 const int *__restrict__ blk_inst) {
  const int ib = blk_inst[blockIdx.x];
  const Inst I = inst[ib];
  const long t = blockIdx.x - I.blk0;
  const int x = (int)(t % I.tiles_x) * blockDim.x + threadIdx.x;
  const int y = (int)(t / I.tiles_x) * blockDim.y + threadIdx.y;
  if (x >= I.nx || y >= I.ny) return;
  const long n = (long)y * I.nx + x;
  const double rx = r[2 * I.off + n], ry = r[2 * I.off + I.N + n];
  const double P1 = -rx - ry, P2 = rx - ry;
  double *p = pout + 8 * I.off;
  p[0 * I.N + n] = -rx;
  p[1 * I.N + n] = -ry;
  p[2 * I.N + n] = rx;
  p[3 * I.N + n] = ry;
  p[4 * I.N + n] = P1;
  p[5 * I.N + n] = P2;
  p[6 * I.N + n] = -P1;
  p[7 * I.N + n] = -P2;
}

// Per block: sum |d - d*|^2 (objective) and write r = (dx^2/Cbar_i)(d - d*); or, with
// dstar_only, sum |d*|^2 (Cbar).  Each block lies in one instance.
__global__ void __launch_bounds__(kThreads) k_objective_batch(
    const double *__restrict__ fc, const double *__restrict__ q, const double *__restrict__ dstar,
    double *__restrict__ r, const double *__restrict__ rscale, const Inst *__restrict__ inst,
    const int *__restrict__ blk_inst, int explicit_fs, int dstar_only,
    double *__restrict__ partial) {
  const int ib = blk_inst[blockIdx.x];
  const Inst I = inst[ib];
  const long t = blockIdx.x - I.blk0;
  const int x = (int)(t % I.tiles_x) * blockDim.x + threadIdx.x;
  const int y = (int)(t / I.tiles_x) * blockDim.y + threadIdx.y;
  double acc[1] = {0.0};
  if (x < I.nx && y < I.ny) {
    const long n = (long)y * I.nx + x;
    const double *ds = dstar + 2 * I.off;
    if (dstar_only) {
      acc[0] = ds[n] * ds[n] + ds[I.N + n] * ds[I.N + n];
    } else {
      const Grid g{I.nx, I.ny, I.N};
      const Bounded b{};
      double f[8], gsel;
      if (explicit_fs) {
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = fc[8 * I.off + k * I.N + n];
      } else {
        pull_primal<false>(fc + 8 * I.off, x, y, g, b, f, gsel);
      }
      const double *qq = q + 2 * I.off;
      const double ex = (f[0] - f[2]) + (f[4] - f[6]) - (f[5] - f[7]) + 2.0 * qq[n] - ds[n];
      const double ey = (f[1] - f[3]) + (f[4] - f[6]) + (f[5] - f[7]) + 2.0 * qq[I.N + n] - ds[I.N + n];
      acc[0] = ex * ex + ey * ey;
      const double sc = rscale[ib];
      r[2 * I.off + n] = sc * ex;
      r[2 * I.off + I.N + n] = sc * ey;
    }
  }
  __shared__ double sm[32];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.x] = acc[0];
}

// dJ/dF_n = dx_i^2 (r_n / 2 - (dC/dg)^T phi_S,n) per instance (Eq. optimality).
__global__ void __launch_bounds__(kThreads) k_grad_batch(const double *__restrict__ pc,
                                                         const double *__restrict__ r,
                                                         double *__restrict__ grad,
                                                         const Inst *__restrict__ inst,
                                                         const int *__restrict__ blk_inst) {
  const int ib = blk_inst[blockIdx.x];
  const Inst I = inst[ib];
  const long t = blockIdx.x - I.blk0;
  const int x = (int)(t % I.tiles_x) * blockDim.x + threadIdx.x;
  const int y = (int)(t / I.tiles_x) * blockDim.y + threadIdx.y;
  if (x >= I.nx || y >= I.ny) return;
  const Grid g{I.nx, I.ny, I.N};
  const Bounded b{};
  const long n = (long)y * I.nx + x;
  double p[8], gsel, sx, sy;
  pull_adjoint<false>(pc + 8 * I.off, x, y, g, b, p, gsel);
  force_sensitivity(p, sx, sy);
  const double dx2 = I.dx * I.dx;
  grad[2 * I.off + n] = dx2 * (0.5 * r[2 * I.off + n] - sx);
  grad[2 * I.off + I.N + n] = dx2 * (0.5 * r[2 * I.off + I.N + n] - sy);
}

// q = dx_i^2 F / 4 per instance; one thread per node of the concatenated range.
__global__ void k_set_force_batch(double *__restrict__ q, const double *__restrict__ F,
                                  const Inst *__restrict__ inst, const int *__restrict__ blk_inst) {
  const int ib = blk_inst[blockIdx.x];
  const Inst I = inst[ib];
  const long t = blockIdx.x - I.blk0;
  const int x = (int)(t % I.tiles_x) * blockDim.x + threadIdx.x;
  const int y = (int)(t / I.tiles_x) * blockDim.y + threadIdx.y;
  if (x >= I.nx || y >= I.ny) return;
  const long n = (long)y * I.nx + x;
  const double s = 0.25 * I.dx * I.dx;
  q[2 * I.off + n] = s * F[2 * I.off + n];
  q[2 * I.off + I.N + n] = s * F[2 * I.off + I.N + n];
}

// One block per instance: out[i] = scale_i * sum of that instance's block partials
// (fixed order).  mode 0: J_i = 0.5 dx_i^2 / Cbar_i * S; mode 1: Cbar_i = dx_i^2 S and
// rscale_i = dx_i^2 / Cbar_i.
__global__ void __launch_bounds__(kThreads) k_finish_batch(const double *__restrict__ partial,
                                                           const Inst *__restrict__ inst,
                                                           const double *__restrict__ cbar,
                                                           int count, long total_blocks, int mode,
                                                           double *__restrict__ out,
                                                           double *__restrict__ rscale) {
  const int i = blockIdx.x;
  if (i >= count) return;
  const Inst I = inst[i];
  const long end = (i + 1 < count) ? inst[i + 1].blk0 : total_blocks;
  double acc[1] = {0.0};
  for (long b = I.blk0 + threadIdx.x; b < end; b += kThreads) acc[0] += partial[b];
  __shared__ double sm[32];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) {
    const double dx2 = I.dx * I.dx;
    if (mode == 0) {
      out[i] = 0.5 * dx2 / cbar[i] * acc[0];
    } else {
      out[i] = dx2 * acc[0];
      rscale[i] = dx2 / (dx2 * acc[0]);
    }
  }
}

}  // namespace

struct lbm_batch {
  int count = 0;
  long total = 0;  // nodes
  std::vector<int> nx, ny;
  std::vector<double> dx;
  std::vector<long> off;
  Coef coef{};
  int kernel = 0;
  cudaStream_t stream = nullptr, cap = nullptr;
  int bx = 128;  // tile width (blockDim.x); blockDim.y = 256 / bx
  long nblocks = 0;
  Inst *d_inst = nullptr;
  int *d_blk = nullptr;
  // the adjoint sweep's own tile width and block table (tuned separately)
  int bx_a = 128;
  long nblocks_a = 0;
  Inst *d_inst_a = nullptr;
  int *d_blk_a = nullptr;
  double *fA = nullptr, *fB = nullptr, *pA = nullptr, *pB = nullptr;
  double *q = nullptr, *r = nullptr, *dstar = nullptr;
  double *partial = nullptr, *cbar = nullptr, *rscale = nullptr, *jbuf = nullptr;
  double *fcur = nullptr, *fnext = nullptr, *pcur = nullptr, *pnext = nullptr;
  bool fs_explicit = true, have_target = false, adjoint_valid = false;
  struct G {
    int kind, parity, bx;
    long k;
    cudaGraphExec_t exec;
  };
  std::vector<G> graphs;
};

namespace {

bool batch_coefs(double E, double nu, Coef &c) {
  if (!(E > 0.0) || !(nu > -1.0 && nu < 1.0)) return false;
  const double th = 1.0 / 3.0;
  const double mu = E / (2.0 * (1.0 + nu)), K = E / (2.0 * (1.0 - nu));
  const double w11 = 1.0 / (mu / th + 0.5), ws = 1.0 / (2.0 * K / (1.0 + th) + 0.5);
  const double wd = 1.0 / (2.0 * mu / (1.0 - th) + 0.5);
  c = Coef{};
  c.c11 = 1.0 - w11; c.cs = 1.0 - ws; c.cd = 1.0 - wd;
  c.w11 = w11; c.ws = ws; c.wd = wd; c.K = K;
  c.q11 = 0.25 * c.c11; c.qs = 0.25 * c.cs; c.qd = 0.25 * c.cd;
  auto fixc = [](double v) {
    const long long C = std::llround(std::ldexp(v, 62));
    const long long hi = C >> 31;
    return FixC{(int)hi, (int)(C - hi * (1LL << 31))};
  };
  c.fx = CoefFix{fixc(c.qs), fixc(c.qd), fixc(c.q11), fixc(1.0 / 3.0)};
  return true;
}

// Block tables for tile width bx (blockDim = (bx, 256 / bx)): which = 0 the table of the
// primal sweep and of every other kernel, which = 1 the adjoint sweep's.
lbm_status build_tables(lbm_batch *b, int which, int bx) {
  const int by = kThreads / bx;
  std::vector<Inst> inst(b->count);
  std::vector<int> blk;
  long blk0 = 0;
  for (int i = 0; i < b->count; ++i) {
    const int tx = (b->nx[i] + bx - 1) / bx, ty = (b->ny[i] + by - 1) / by;
    inst[i] = Inst{b->nx[i], b->ny[i], (long)b->nx[i] * b->ny[i], b->off[i], blk0, tx, b->dx[i]};
    blk.insert(blk.end(), (size_t)tx * ty, i);
    blk0 += (long)tx * ty;
  }
  if (blk0 > 0x7fffffffL) return LBM_ERR_ARG;
  int *&d_blk = which == 0 ? b->d_blk : b->d_blk_a;
  Inst *d_inst = which == 0 ? b->d_inst : b->d_inst_a;
  if (d_blk) cudaFree(d_blk);
  d_blk = nullptr;
  if (cudaMalloc(&d_blk, sizeof(int) * blk.size()) != cudaSuccess) return LBM_ERR_OOM;
  if (cudaMemcpy(d_blk, blk.data(), sizeof(int) * blk.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_inst, inst.data(), sizeof(Inst) * b->count, cudaMemcpyHostToDevice) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (which == 1) {
    b->nblocks_a = blk0;
    b->bx_a = bx;
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
    return LBM_OK;
  }
  if (b->partial) cudaFree(b->partial);
  b->partial = nullptr;
  if (cudaMalloc(&b->partial, sizeof(double) * blk0) != cudaSuccess) return LBM_ERR_OOM;
  b->nblocks = blk0;
  b->bx = bx;
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  return LBM_OK;
}

dim3 blk_dim(const lbm_batch *b) { return dim3(b->bx, kThreads / b->bx); }

void launch_sweep(lbm_batch *b, int kind, cudaStream_t s) {
  const dim3 bd = blk_dim(b);
  const unsigned g = (unsigned)b->nblocks;
  if (kind == 0) {
    if (b->kernel == LBM_KERNEL_FP64)
      k_primal_batch<false, 0><<<g, bd, 0, s>>>(b->fcur, b->fnext, b->q, b->d_inst, b->d_blk, b->coef);
    else
      k_primal_batch<false, 1><<<g, bd, 0, s>>>(b->fcur, b->fnext, b->q, b->d_inst, b->d_blk, b->coef);
    std::swap(b->fcur, b->fnext);
  } else {
    const dim3 ba(b->bx_a, kThreads / b->bx_a);
    const unsigned ga = (unsigned)b->nblocks_a;
    if (b->kernel == LBM_KERNEL_FP64)
      k_adjoint_batch<0><<<ga, ba, 0, s>>>(b->pcur, b->pnext, b->r, b->d_inst_a, b->d_blk_a, b->coef);
    else
      k_adjoint_batch<1><<<ga, ba, 0, s>>>(b->pcur, b->pnext, b->r, b->d_inst_a, b->d_blk_a, b->coef);
    std::swap(b->pcur, b->pnext);
  }
}

lbm_status run_batch_sweeps(lbm_batch *b, int kind, long k) {
  if (kind == 0 && b->fs_explicit && k > 0) {
    if (b->kernel == LBM_KERNEL_FP64)
      k_collide_batch<0><<<(unsigned)b->nblocks, blk_dim(b), 0, b->stream>>>(b->fcur, b->fnext, b->q, b->d_inst, b->d_blk, b->coef);
    else
      k_collide_batch<1><<<(unsigned)b->nblocks, blk_dim(b), 0, b->stream>>>(b->fcur, b->fnext, b->q, b->d_inst, b->d_blk, b->coef);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    std::swap(b->fcur, b->fnext);
    b->fs_explicit = false;
    --k;
  }
  constexpr long kChunk = 64;
  while (k > 0) {
    const long c = k >= kChunk ? kChunk : k;
    if (c < 4) {
      for (long i = 0; i < c; ++i) launch_sweep(b, kind, b->stream);
      if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    } else {
      const int parity = kind == 0 ? (b->fcur == b->fA ? 0 : 1) : (b->pcur == b->pA ? 0 : 1);
      cudaGraphExec_t ex = nullptr;
      const int bxk = kind == 0 ? b->bx : b->bx_a;
      for (auto &g : b->graphs)
        if (g.kind == kind && g.k == c && g.parity == parity && g.bx == bxk) ex = g.exec;
      if (!ex) {
        if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
          return LBM_ERR_CUDA;
        double *f0 = b->fcur, *f1 = b->fnext, *p0 = b->pcur, *p1 = b->pnext;
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
          return LBM_ERR_CUDA;
        for (long i = 0; i < c; ++i) launch_sweep(b, kind, b->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        b->fcur = f0; b->fnext = f1; b->pcur = p0; b->pnext = p1;
        if (e != cudaSuccess || !graph) return LBM_ERR_CUDA;
        const cudaError_t ei = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return LBM_ERR_CUDA;
        b->graphs.push_back(lbm_batch::G{kind, parity, bxk, c, ex});
      }
      if (cudaGraphLaunch(ex, b->stream) != cudaSuccess) return LBM_ERR_CUDA;
      if (c & 1) {
        if (kind == 0) std::swap(b->fcur, b->fnext);
        else std::swap(b->pcur, b->pnext);
      }
    }
    k -= c;
  }
  return LBM_OK;
}

void free_batch(lbm_batch *b) {
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  void *bufs[] = {b->d_inst, b->d_blk, b->fA, b->fB, b->pA, b->pB, b->q, b->r, b->dstar,
                  b->partial, b->cbar, b->rscale, b->jbuf, b->d_inst_a, b->d_blk_a};
  for (void *p : bufs)
    if (p) cudaFree(p);
  if (b->cap) cudaStreamDestroy(b->cap);
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int count, const int *nx, const int *ny, const double *dx, double E,
                            double nu, int kernel, void *stream, lbm_batch **out) {
  if (!out || count < 1 || !nx || !ny) return LBM_ERR_ARG;
  *out = nullptr;
  if (kernel != LBM_KERNEL_AUTO && kernel != LBM_KERNEL_FP64) return LBM_ERR_ARG;
  Coef c{};
  if (!batch_coefs(E, nu, c)) return LBM_ERR_ARG;
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_OOM;
  b->count = count;
  b->kernel = kernel;
  b->coef = c;
  b->stream = (cudaStream_t)stream;
  long off = 0;
  for (int i = 0; i < count; ++i) {
    if (nx[i] < 3 || ny[i] < 3) { delete b; return LBM_ERR_ARG; }
    const double h = dx ? dx[i] : 1.0 / nx[i];
    if (!(h > 0.0)) { delete b; return LBM_ERR_ARG; }
    b->nx.push_back(nx[i]);
    b->ny.push_back(ny[i]);
    b->dx.push_back(h);
    b->off.push_back(off);
    off += (long)nx[i] * ny[i];
  }
  b->total = off;
  const size_t pop = sizeof(double) * 8 * off, two = sizeof(double) * 2 * off;
  cudaError_t e = cudaSuccess;
#define BALLOC(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes))
  BALLOC(b->d_inst, sizeof(Inst) * count);
  BALLOC(b->d_inst_a, sizeof(Inst) * count);
  BALLOC(b->fA, pop); BALLOC(b->fB, pop); BALLOC(b->pA, pop); BALLOC(b->pB, pop);
  BALLOC(b->q, two); BALLOC(b->r, two); BALLOC(b->dstar, two);
  BALLOC(b->cbar, sizeof(double) * count); BALLOC(b->rscale, sizeof(double) * count);
  BALLOC(b->jbuf, sizeof(double) * count);
#undef BALLOC
  if (e != cudaSuccess) {
    free_batch(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
  }
  lbm_status st = build_tables(b, 0, 128);
  if (st == LBM_OK) st = build_tables(b, 1, 128);
  if (st) { free_batch(b); delete b; return st; }
  if (cudaMemsetAsync(b->fA, 0, pop, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->pA, 0, pop, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->q, 0, two, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    free_batch(b);
    delete b;
    return LBM_ERR_CUDA;
  }
  b->fcur = b->fA; b->fnext = b->fB; b->pcur = b->pA; b->pnext = b->pB;
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch *b) {
  if (!b) return LBM_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
  return LBM_OK;
}

long lbm_batch_offset(const lbm_batch *b, int i) {
  if (!b || i < 0 || i > b->count) return -1;
  return i == b->count ? b->total : b->off[i];
}

lbm_status lbm_batch_set_force(lbm_batch *b, const double *F) {
  if (!b || !F) return LBM_ERR_ARG;
  k_set_force_batch<<<(unsigned)b->nblocks, blk_dim(b), 0, b->stream>>>(b->q, F, b->d_inst, b->d_blk);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaMemsetAsync(b->fcur, 0, sizeof(double) * 8 * b->total, b->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  b->fs_explicit = true;
  b->adjoint_valid = false;
  return LBM_OK;
}

lbm_status lbm_batch_set_target(lbm_batch *b, const double *dstar) {
  if (!b || !dstar) return LBM_ERR_ARG;
  if (cudaMemcpyAsync(b->dstar, dstar, sizeof(double) * 2 * b->total, cudaMemcpyDeviceToDevice,
                      b->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  k_objective_batch<<<(unsigned)b->nblocks, blk_dim(b), 0, b->stream>>>(
      b->fcur, b->q, b->dstar, b->r, b->rscale, b->d_inst, b->d_blk, 1, 1, b->partial);
  k_finish_batch<<<b->count, kThreads, 0, b->stream>>>(b->partial, b->d_inst, b->cbar, b->count,
                                                       b->nblocks, 1, b->cbar, b->rscale);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  std::vector<double> cb(b->count);
  if (cudaMemcpyAsync(cb.data(), b->cbar, sizeof(double) * b->count, cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  for (double v : cb)
    if (!(v > 0.0) || !std::isfinite(v)) return LBM_ERR_ARG;
  b->have_target = true;
  return LBM_OK;
}

lbm_status lbm_batch_primal(lbm_batch *b, long sweeps) {
  if (!b || sweeps < 0) return LBM_ERR_ARG;
  b->adjoint_valid = false;
  return run_batch_sweeps(b, 0, sweeps);
}

lbm_status lbm_batch_objective(lbm_batch *b, double *J) {
  if (!b || !J) return LBM_ERR_ARG;
  if (!b->have_target) return LBM_ERR_STATE;
  k_objective_batch<<<(unsigned)b->nblocks, blk_dim(b), 0, b->stream>>>(
      b->fcur, b->q, b->dstar, b->r, b->rscale, b->d_inst, b->d_blk, b->fs_explicit ? 1 : 0, 0,
      b->partial);
  k_finish_batch<<<b->count, kThreads, 0, b->stream>>>(b->partial, b->d_inst, b->cbar, b->count,
                                                       b->nblocks, 0, J, nullptr);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_batch_adjoint(lbm_batch *b, long sweeps) {
  if (!b || sweeps < 0) return LBM_ERR_ARG;
  if (!b->have_target) return LBM_ERR_STATE;
  const lbm_status st = lbm_batch_objective(b, b->jbuf);  // r at the current primal state
  if (st) return st;
  if (sweeps == 0) {  // phi_C = 0
    if (cudaMemsetAsync(b->pcur, 0, sizeof(double) * 8 * b->total, b->stream) != cudaSuccess)
      return LBM_ERR_CUDA;
  } else {  // from rest, the first sweep gives -j
    k_adjoint_rest_batch<<<(unsigned)b->nblocks_a, dim3(b->bx_a, kThreads / b->bx_a), 0,
                           b->stream>>>(b->r, b->pnext, b->d_inst_a, b->d_blk_a);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    std::swap(b->pcur, b->pnext);
  }
  const lbm_status s2 = run_batch_sweeps(b, 1, sweeps > 0 ? sweeps - 1 : 0);
  if (s2 == LBM_OK) b->adjoint_valid = true;
  return s2;
}

lbm_status lbm_batch_gradient(lbm_batch *b, double *grad) {
  if (!b || !grad) return LBM_ERR_ARG;
  if (!b->adjoint_valid) return LBM_ERR_STATE;
  k_grad_batch<<<(unsigned)b->nblocks, blk_dim(b), 0, b->stream>>>(b->pcur, b->r, grad, b->d_inst,
                                                                   b->d_blk);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_batch_get_populations(lbm_batch *b, int which, double *dst) {
  if (!b || !dst) return LBM_ERR_ARG;
  if (which == 0 && !b->fs_explicit) {
    // f_S = S f_C(t-1): one pull per instance, through the objective kernel's pull path
    // is not a copy, so use a collide-free pass: primal pull written out
    for (int i = 0; i < b->count; ++i) {
      const Grid g{b->nx[i], b->ny[i], (long)b->nx[i] * b->ny[i]};
      const dim3 bd(b->bx, kThreads / b->bx);
      const dim3 gd((b->nx[i] + bd.x - 1) / bd.x, (b->ny[i] + bd.y - 1) / bd.y);
      k_pull_primal<false><<<gd, bd, 0, b->stream>>>(b->fcur + 8 * b->off[i], dst + 8 * b->off[i], g,
                                                     Bounded{});
    }
  } else if (which == 0) {
    if (cudaMemcpyAsync(dst, b->fcur, sizeof(double) * 8 * b->total, cudaMemcpyDeviceToDevice,
                        b->stream) != cudaSuccess)
      return LBM_ERR_CUDA;
  } else if (which == 2) {
    if (cudaMemcpyAsync(dst, b->pcur, sizeof(double) * 8 * b->total, cudaMemcpyDeviceToDevice,
                        b->stream) != cudaSuccess)
      return LBM_ERR_CUDA;
  } else {
    return LBM_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_batch_tune(lbm_batch *b, int sweeps, int *best_bx) {
  if (!b || sweeps < 1) return LBM_ERR_ARG;
  // time `sweeps` primal sweeps, then `sweeps` adjoint sweeps, for each tile width and
  // keep the fastest for each (both states restored)
  const int cands[] = {32, 64, 128, 256};
  const size_t pop = sizeof(double) * 8 * b->total;
  double *save = nullptr, *save_p = nullptr;
  if (cudaMalloc(&save, pop) != cudaSuccess) return LBM_ERR_OOM;
  if (cudaMalloc(&save_p, pop) != cudaSuccess) {
    cudaFree(save);
    return LBM_ERR_OOM;
  }
  if (cudaMemcpyAsync(save, b->fcur, pop, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(save_p, b->pcur, pop, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess) {
    cudaFree(save);
    cudaFree(save_p);
    return LBM_ERR_CUDA;
  }
  const bool was_fs = b->fs_explicit, was_adj = b->adjoint_valid;
  double *cur0 = b->fcur, *next0 = b->fnext, *pcur0 = b->pcur, *pnext0 = b->pnext;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best_w[2] = {b->bx, b->bx_a};
  lbm_status st = LBM_OK;
  for (int kind = 0; kind < 2 && st == LBM_OK; ++kind) {
    float best = 1e30f;
    for (int bx : cands) {
      if ((st = build_tables(b, kind, bx))) break;
      b->fs_explicit = false;
      run_batch_sweeps(b, kind, 4);  // capture + warm-up
      cudaEventRecord(e0, b->stream);
      run_batch_sweeps(b, kind, sweeps);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = LBM_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_w[kind] = bx; }
    }
    if (st == LBM_OK) st = build_tables(b, kind, best_w[kind]);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->fcur = cur0;
  b->fnext = next0;
  b->pcur = pcur0;
  b->pnext = pnext0;
  cudaMemcpyAsync(b->fcur, save, pop, cudaMemcpyDeviceToDevice, b->stream);
  cudaMemcpyAsync(b->pcur, save_p, pop, cudaMemcpyDeviceToDevice, b->stream);
  cudaStreamSynchronize(b->stream);
  cudaFree(save);
  cudaFree(save_p);
  b->fs_explicit = was_fs;
  b->adjoint_valid = was_adj;
  if (best_bx) *best_bx = best_w[0];
  return st;
}

}  // extern "C"
