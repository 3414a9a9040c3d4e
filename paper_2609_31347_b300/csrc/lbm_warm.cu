// Conversions between the solver's FP64 SoA populations and the warm-start network's
// FP32 NHWC tensors (see "Learned warm start" in include/lbm_solid.h).
//
// The network works on a resolution-free representation of a steady state.  On the
// periodic lattice the steady moments of f_S scale with the grid spacing dx as
//   m10, m01 = O(1) (the displacement, Eq. disp_from_moments),
//   m11, m_s, m_d, m22 = O(dx) (the stress, Eq. stress_from_moments),
//   m12 - theta m10, m21 - theta m01 = O(dx^2) (the equilibria of the third-order
//   moments are theta times the first-order ones, Section 3.1),
// so for primal states (mode 1) the network predicts z = (m10, m01, m11/dx, m_s/dx,
// m_d/dx, (m12 - theta m10)/dx^2, (m21 - theta m01)/dx^2, m22/dx).  The steady adjoint
// state phi_C (mode 2) has the same pattern with (1 - theta) in place of theta -- there
// m12 = (1 - theta) m10 and m21 = (1 - theta) m01 hold exactly at the fixed point -- and
// its size grows as 1/dx^2 for a source r ~ dx^2 (r = (dx^2/Cbar) w (d - d*)), so mode 2
// multiplies z by dx^2.  Mode 0 uses the plain moments.  Each channel is divided by a
// per-channel constant c_i (c_i = 0: the channel is not predicted and stays zero) and by
// the RMS s of the sample's input field: the states are linear in their input, so
// dividing the input by s and multiplying the output by s makes the prediction exactly
// scale-equivariant.
//
// A network trained at one resolution is used at `factor` times that resolution:
// the input field is averaged over factor x factor blocks, and the predicted moments
// are interpolated bilinearly (periodic) back to the fine nodes, with the fine dx in
// the rescaling.  Coarse node j stands for the centre of its block, fine index
// factor * j + (factor - 1) / 2.
#include <cuda_runtime.h>

#include "lbm_solid.h"

namespace {

constexpr double kTh = 1.0 / 3.0;

// D2Q8 moments (Appendix A.1, gamma = 0): velocities 0:(1,0) 1:(0,1) 2:(-1,0) 3:(0,-1)
// 4:(1,1) 5:(-1,1) 6:(-1,-1) 7:(1,-1).
__device__ __forceinline__ void moments(const double (&f)[8], double (&m)[8]) {
  const double a02 = f[0] - f[2], a13 = f[1] - f[3];
  const double b46 = f[4] - f[6], b57 = f[5] - f[7];
  const double s46 = f[4] + f[6], s57 = f[5] + f[7];
  m[0] = a02 + b46 - b57;                                // m10
  m[1] = a13 + b46 + b57;                                // m01
  m[2] = s46 - s57;                                      // m11
  m[3] = f[0] + f[1] + f[2] + f[3] + 2.0 * (s46 + s57);  // m_s
  m[4] = f[0] - f[1] + f[2] - f[3];                      // m_d
  m[5] = b46 - b57;                                      // m12
  m[6] = b46 + b57;                                      // m21
  m[7] = s46 + s57;                                      // m22
}

// Inverse of `moments`: the diagonal populations from (m22, m12, m21, m11), the axis
// populations from m_s - 2 m22, m_d, m10 - m12 and m01 - m21.
__device__ __forceinline__ void populations(const double (&m)[8], double (&f)[8]) {
  const double S = m[7], X = m[5], Y = m[6], Z = m[2];
  f[4] = 0.25 * (S + X + Y + Z);
  f[5] = 0.25 * (S - X + Y - Z);
  f[6] = 0.25 * (S - X - Y + Z);
  f[7] = 0.25 * (S + X - Y - Z);
  const double T = m[3] - 2.0 * S;
  const double p = 0.5 * (T + m[4]), q = 0.5 * (T - m[4]);
  const double ux = m[0] - X, uy = m[1] - Y;
  f[0] = 0.5 * (p + ux);
  f[2] = 0.5 * (p - ux);
  f[1] = 0.5 * (q + uy);
  f[3] = 0.5 * (q - uy);
}

// populations -> network coordinates z (before the 1 / (s c_i) normalisation)
__device__ __forceinline__ void to_z(const double (&m)[8], double dx, int mode, double (&z)[8]) {
  if (mode == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) z[i] = m[i];
    return;
  }
  const double th = mode == 1 ? kTh : 1.0 - kTh;
  const double a = mode == 1 ? 1.0 : dx * dx;
  const double idx = a / dx, idx2 = a / (dx * dx);
  z[0] = a * m[0];
  z[1] = a * m[1];
  z[2] = m[2] * idx;
  z[3] = m[3] * idx;
  z[4] = m[4] * idx;
  z[5] = (m[5] - th * m[0]) * idx2;
  z[6] = (m[6] - th * m[1]) * idx2;
  z[7] = m[7] * idx;
}

__device__ __forceinline__ void from_z(const double (&z)[8], double dx, int mode, double (&m)[8]) {
  if (mode == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) m[i] = z[i];
    return;
  }
  const double th = mode == 1 ? kTh : 1.0 - kTh;
  const double ia = mode == 1 ? 1.0 : 1.0 / (dx * dx);
  const double sx = dx * ia, sx2 = dx * dx * ia;
  m[0] = z[0] * ia;
  m[1] = z[1] * ia;
  m[2] = z[2] * sx;
  m[3] = z[3] * sx;
  m[4] = z[4] * sx;
  m[5] = th * m[0] + z[5] * sx2;
  m[6] = th * m[1] + z[6] * sx2;
  m[7] = z[7] * sx;
}

// s[b] = RMS over the 2N values of sample b of field - ref (ref NULL = 0; 1 where the
// difference is zero).  One block per sample, fixed reduction order.
__global__ void __launch_bounds__(1024) k_field_rms(const double *__restrict__ field,
                                                     const double *__restrict__ ref, long N,
                                                     float *__restrict__ s) {
  const long o = (long)blockIdx.x * 2 * N;
  double acc = 0.0;
  for (long i = threadIdx.x; i < 2 * N; i += blockDim.x) {
    const double v = field[o + i] - (ref ? ref[o + i] : 0.0);
    acc += v * v;
  }
  __shared__ double sm[1024];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double r = sqrt(sm[0] / (double)(2 * N));
    s[blockIdx.x] = r > 0.0 ? (float)r : 1.f;
  }
}

// x[b, yc, xc, c] = mean of (field - ref)[b, c, factor x factor block] / s[b]
__global__ void k_encode(const double *__restrict__ field, const double *__restrict__ ref, int nx,
                         int ny, int factor, const float *__restrict__ s, float *__restrict__ x,
                         int count) {
  const int wc = nx / factor, hc = ny / factor;
  const long N = (long)nx * ny;
  const long total = (long)count * hc * wc * 2;
  const double inv = 1.0 / ((double)factor * factor);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i & 1);
    long r = i >> 1;
    const int xc = (int)(r % wc);
    r /= wc;
    const int yc = (int)(r % hc), b = (int)(r / hc);
    const long o = ((long)b * 2 + c) * N;
    double acc = 0.0;
    for (int dy = 0; dy < factor; ++dy)
      for (int dx = 0; dx < factor; ++dx) {
        const long j = o + (long)(yc * factor + dy) * nx + xc * factor + dx;
        acc += field[j] - (ref ? ref[j] : 0.0);
      }
    x[i] = (float)(acc * inv / (double)s[b]);
  }
}

// t[b, y, x, i] = z_i(pop[b, :, node]) / (s[b] c_i)   (c = NULL: c_i = 1; c_i = 0: 0)
__global__ void k_targets(const double *__restrict__ pop, long N, double dx, int mode,
                          const float *__restrict__ s, const float *__restrict__ c,
                          float *__restrict__ t, int count) {
  const long total = (long)count * N;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const long b = i / N, n = i % N;
    const double *p = pop + b * 8 * N + n;
    double f[8], m[8], z[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = p[k * N];
    moments(f, m);
    to_z(m, dx, mode, z);
    const double is = 1.0 / (double)s[b];
    float o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double ck = c ? (double)c[k] : 1.0;
      o[k] = ck != 0.0 ? (float)(z[k] * is / ck) : 0.f;
    }
    float4 *dst = reinterpret_cast<float4 *>(t + i * 8);
    dst[0] = make_float4(o[0], o[1], o[2], o[3]);
    dst[1] = make_float4(o[4], o[5], o[6], o[7]);
  }
}

// pop[b, :, fine node] (= or +=) populations of the bilinear interpolation of y at
// that node, rescaled by s[b] c_i and the fine dx.
__global__ void k_decode(const float *__restrict__ y, int wc, int hc, int factor, double dx,
                         int mode, const float *__restrict__ s, const float *__restrict__ c,
                         double *__restrict__ pop, int count, int accumulate) {
  const int nx = wc * factor, ny = hc * factor;
  const long N = (long)nx * ny;
  const long total = (long)count * N;
  const double half = 0.5 * (factor - 1);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const long b = i / N, n = i % N;
    const int xf = (int)(n % nx), yf = (int)(n / nx);
    const double u = ((double)xf - half) / factor, v = ((double)yf - half) / factor;
    const double fu = floor(u), fv = floor(v);
    const double wx = u - fu, wy = v - fv;
    const int x0 = (((int)fu % wc) + wc) % wc, y0 = (((int)fv % hc) + hc) % hc;
    const int x1 = (x0 + 1) % wc, y1 = (y0 + 1) % hc;
    const float *base = y + b * (long)hc * wc * 8;
    const float *q00 = base + ((long)y0 * wc + x0) * 8, *q01 = base + ((long)y0 * wc + x1) * 8;
    const float *q10 = base + ((long)y1 * wc + x0) * 8, *q11 = base + ((long)y1 * wc + x1) * 8;
    double z[8], m[8], f[8];
    const double sb = (double)s[b];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double v0 = (1.0 - wx) * q00[k] + wx * q01[k];
      const double v1 = (1.0 - wx) * q10[k] + wx * q11[k];
      z[k] = ((1.0 - wy) * v0 + wy * v1) * sb * (c ? (double)c[k] : 1.0);
    }
    from_z(z, dx, mode, m);
    populations(m, f);
    double *p = pop + b * 8 * N + n;
#pragma unroll
    for (int k = 0; k < 8; ++k) p[k * N] = accumulate ? p[k * N] + f[k] : f[k];
  }
}

// Remove the Fourier components at the wavevectors (nx/2, 0) and (0, ny/2) (for even
// sizes) of one population plane per block: sum_n (-1)^x f(n) / N and sum_n (-1)^y f(n) / N
// are the coefficients of the two orthogonal sign patterns.  The primal and adjoint
// steps have the eigenvalue -1 at those wavevectors, so error there would alternate
// forever instead of decaying; the steady state of a smooth field has none.
__global__ void __launch_bounds__(1024) k_drop_half_nyquist(double *__restrict__ pop, int nx,
                                                             int ny) {
  const long N = (long)nx * ny;
  double *f = pop + (long)blockIdx.x * N;
  double sx = 0.0, sy = 0.0;
  for (long i = threadIdx.x; i < N; i += blockDim.x) {
    const int x = (int)(i % nx), y = (int)(i / nx);
    const double v = f[i];
    sx += (x & 1) ? -v : v;
    sy += (y & 1) ? -v : v;
  }
  __shared__ double sm[2][1024];
  sm[0][threadIdx.x] = sx;
  sm[1][threadIdx.x] = sy;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + o];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  const double ax = (nx % 2 == 0) ? sm[0][0] / (double)N : 0.0;
  const double ay = (ny % 2 == 0) ? sm[1][0] / (double)N : 0.0;
  for (long i = threadIdx.x; i < N; i += blockDim.x) {
    const int x = (int)(i % nx), y = (int)(i / nx);
    f[i] -= ((x & 1) ? -ax : ax) + ((y & 1) ? -ay : ay);
  }
}

// Set the conserved k = 0 components of one sample (block) to zero.  On the periodic
// lattice the mean displacement is conserved by both iterations (the eigenvalue 1 at
// k = 0, two collision invariants): from rest with a zero-mean force (source) it stays
// zero, so a warm start must start there too, or the iteration settles on a rigidly
// shifted state.  Primal (mode 1): the means of m10 = <c_x, f> and m01 = <c_y, f> are
// removed along the stationary states v_x, v_y (m10 = 1 resp. m01 = 1, third-order
// moments at equilibrium theta, all else 0).  Adjoint (mode 2): the conserved quantities
// are <v_x, phi>, <v_y, phi>, removed along c_x, c_y (<v_x, c_x> = 1, <v_y, c_x> = 0).
__global__ void __launch_bounds__(256) k_drop_conserved_mean(double *__restrict__ pop, long N,
                                                              int mode) {
  double *f = pop + (long)blockIdx.x * 8 * N;
  double acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.0;
  for (long n = threadIdx.x; n < N; n += blockDim.x)
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += f[k * N + n];
  __shared__ double sm[8][256];
#pragma unroll
  for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int k = 0; k < 8; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + o];
    __syncthreads();
  }
  const double cx[8] = {1, 0, -1, 0, 1, -1, -1, 1}, cy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
  const double a = 0.5 * (1.0 - kTh), b = 0.25 * kTh;
  const double vx[8] = {a, 0, -a, 0, b, -b, -b, b}, vy[8] = {0, a, 0, -a, b, b, -b, -b};
  const double *wx = mode == 1 ? cx : vx, *wy = mode == 1 ? cy : vy;  // conserved functionals
  const double *ux = mode == 1 ? vx : cx, *uy = mode == 1 ? vy : cy;  // removed along these
  double ax = 0.0, ay = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    ax += wx[k] * sm[k][0];
    ay += wy[k] * sm[k][0];
  }
  ax /= (double)N;
  ay /= (double)N;
  double d[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) d[k] = ax * ux[k] + ay * uy[k];
  for (long n = threadIdx.x; n < N; n += blockDim.x)
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k * N + n] -= d[k];
}

// rms[i] = sqrt(mean over the first P' pixels of t[., i]^2), P' = min(P, 2^22); one
// block per channel, fixed order.
__global__ void __launch_bounds__(1024) k_channel_rms(const float *__restrict__ t, long P,
                                                       float *__restrict__ rms) {
  const int ch = blockIdx.x;
  const long n = P < (1L << 22) ? P : (1L << 22);
  double acc = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = t[i * 8 + ch];
    acc += v * v;
  }
  __shared__ double sm[1024];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) rms[ch] = (float)sqrt(sm[0] / (double)n);
}

// ---- History of steady states: combinations and inner products --------------------

constexpr int kMaxVec = 4;                       // history vectors per call
constexpr int kDotBlocks = 296;                  // 2 blocks per SM, grid-stride
constexpr int kDotPairs = (kMaxVec + 1) * (kMaxVec + 2) / 2;

struct VecSet {
  const double *v[kMaxVec + 1];
  double w[kMaxVec];
};

// dst[i] = sum_j w_j src_j[i].  Each element reads every source before it is written, so
// dst may be one of the sources.
__global__ void __launch_bounds__(256) k_combine(VecSet vs, int count, long n,
                                                 double *__restrict__ dst) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < count; ++j) acc += vs.w[j] * vs.v[j][i];
    dst[i] = acc;
  }
}

// Per-block partial sums of u_a . u_b for a <= b < m, in the packed upper-triangle order
// p(a, b) = a * m - a (a - 1) / 2 + (b - a); grid-stride over n, fixed order.
__global__ void __launch_bounds__(256) k_dot_partial(VecSet vs, int m, long n,
                                                     double *__restrict__ part) {
  double acc[kDotPairs];
#pragma unroll
  for (int p = 0; p < kDotPairs; ++p) acc[p] = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    double u[kMaxVec + 1];
#pragma unroll
    for (int a = 0; a <= kMaxVec; ++a) u[a] = a < m ? vs.v[a][i] : 0.0;
    int p = 0;
#pragma unroll
    for (int a = 0; a <= kMaxVec; ++a)
#pragma unroll
      for (int b = a; b <= kMaxVec; ++b) acc[p++] += u[a] * u[b];
  }
  __shared__ double sm[kDotPairs][256];
#pragma unroll
  for (int p = 0; p < kDotPairs; ++p) sm[p][threadIdx.x] = acc[p];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int p = 0; p < kDotPairs; ++p) sm[p][threadIdx.x] += sm[p][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < kDotPairs) part[threadIdx.x * kDotBlocks + blockIdx.x] = sm[threadIdx.x][0];
}

// Sums the partials of each pair in block order and expands the packed triangle (full
// (kMaxVec + 1)^2 layout, only the first m x m used) into out.
__global__ void k_dot_finish(const double *__restrict__ part, int m, double *__restrict__ out) {
  const int t = threadIdx.x;
  if (t >= kDotPairs) return;
  double acc = 0.0;
  for (int b = 0; b < kDotBlocks; ++b) acc += part[t * kDotBlocks + b];
  int p = 0;
  for (int a = 0; a <= kMaxVec; ++a)
    for (int b = a; b <= kMaxVec; ++b, ++p)
      if (p == t && b < m) {
        out[a * m + b] = acc;
        out[b * m + a] = acc;
      }
}

unsigned grid_for(long n) {
  const long b = (n + 255) / 256;
  return (unsigned)(b < 148 * 16 ? (b < 1 ? 1 : b) : 148 * 16);
}

// Bounded grids (one plate geometry, network on a w x h crop of the nx_box x ny_box box):
// x[b, yc, xc, 0] = block mean of mask E_ref / E_n (the compliance: for loads that do not
// depend on E the steady displacement of a uniform modulus is proportional to it, so a
// linear network can represent that dependence), x[b, yc, xc, 1] = block mean of mask,
// E_n = alpha_n^2 (per node) or alpha_b^2 (one modulus per sample).
__global__ void k_encode_modulus(const double *__restrict__ alpha, int per_node,
                                 const uint8_t *__restrict__ mask, int nx_box, long N_box,
                                 double E_ref, int w, int h, int factor,
                                 float *__restrict__ x, int count) {
  const int wc = w / factor, hc = h / factor;
  const long total = (long)count * hc * wc;
  const double inv = 1.0 / ((double)factor * factor);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int xc = (int)(i % wc);
    const long r = i / wc;
    const int yc = (int)(r % hc), b = (int)(r / hc);
    double le = 0.0, mk = 0.0;
    for (int dy = 0; dy < factor; ++dy)
      for (int dx = 0; dx < factor; ++dx) {
        const long n = (long)(yc * factor + dy) * nx_box + xc * factor + dx;
        if (!mask[n]) continue;
        const double a = per_node ? alpha[(long)b * N_box + n] : alpha[b];
        le += E_ref / (a * a);
        mk += 1.0;
      }
    x[2 * i] = (float)(le * inv);
    x[2 * i + 1] = (float)(mk * inv);
  }
}

// Populations between the box (count, 8, ny_box, nx_box) and the crop (count, 8, h, w):
// to_box = 0 copies the crop out; to_box = 1 writes the box, zero outside the crop and at
// inactive nodes (mask NULL: all active).
__global__ void k_crop(const double *__restrict__ src, double *__restrict__ dst, int nx_box,
                       int ny_box, int w, int h, int to_box, const uint8_t *__restrict__ mask,
                       int count) {
  const long Nb = (long)nx_box * ny_box, Nc = (long)w * h;
  const long total = (long)count * 8 * (to_box ? Nb : Nc);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    if (to_box) {
      const long n = i % Nb, bk = i / Nb;
      const int x = (int)(n % nx_box), y = (int)(n / nx_box);
      const bool in = x < w && y < h && (!mask || mask[n]);
      dst[i] = in ? src[bk * Nc + (long)y * w + x] : 0.0;
    } else {
      const long n = i % Nc, bk = i / Nc;
      const int x = (int)(n % w), y = (int)(n / w);
      dst[i] = src[bk * Nb + (long)y * nx_box + x];
    }
  }
}

}  // namespace

extern "C" {

lbm_status lbm_warm_encode(int count, int nx, int ny, int factor, const double *field_dev,
                           const double *ref_dev, float *x_dev, float *scale_dev, void *stream) {
  if (count < 1 || nx < 1 || ny < 1 || factor < 1 || nx % factor || ny % factor || !field_dev ||
      !x_dev || !scale_dev)
    return LBM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long N = (long)nx * ny;
  k_field_rms<<<count, 1024, 0, st>>>(field_dev, ref_dev, N, scale_dev);
  k_encode<<<grid_for((long)count * (N / ((long)factor * factor)) * 2), 256, 0, st>>>(
      field_dev, ref_dev, nx, ny, factor, scale_dev, x_dev, count);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_warm_targets(int count, int nx, int ny, double dx, int mode, const double *pop_dev,
                            const float *scale_dev, const float *chan_dev, float *t_dev,
                            void *stream) {
  if (count < 1 || nx < 1 || ny < 1 || !(dx > 0.0) || mode < 0 || mode > 3 || !pop_dev ||
      !scale_dev || !t_dev)
    return LBM_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(t_dev) % 16) return LBM_ERR_ARG;
  const long N = (long)nx * ny;
  k_targets<<<grid_for((long)count * N), 256, 0, (cudaStream_t)stream>>>(
      pop_dev, N, dx, mode == 3 ? 1 : mode, scale_dev, chan_dev, t_dev, count);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_warm_decode(int count, int wc, int hc, int factor, double dx_fine, int mode,
                           const float *y_dev, const float *scale_dev, const float *chan_dev,
                           double *pop_dev, int accumulate, void *stream) {
  if (count < 1 || wc < 1 || hc < 1 || factor < 1 || !(dx_fine > 0.0) || mode < 0 || mode > 3 ||
      !y_dev || !scale_dev || !pop_dev)
    return LBM_ERR_ARG;
  const long N = (long)wc * hc * factor * factor;
  k_decode<<<grid_for((long)count * N), 256, 0, (cudaStream_t)stream>>>(
      y_dev, wc, hc, factor, dx_fine, mode == 3 ? 1 : mode, scale_dev, chan_dev, pop_dev, count,
      accumulate);
  if (mode == 1 || mode == 2) {
    k_drop_half_nyquist<<<count * 8, 1024, 0, (cudaStream_t)stream>>>(pop_dev, wc * factor,
                                                                     hc * factor);
    k_drop_conserved_mean<<<count, 256, 0, (cudaStream_t)stream>>>(pop_dev, N, mode);
  }
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_warm_encode_modulus(int count, int nx_box, int ny_box, int per_node,
                                   const double *alpha_dev, const uint8_t *mask_dev, double E_ref,
                                   int w, int h, int factor, float *x_dev, void *stream) {
  if (count < 1 || nx_box < 1 || ny_box < 1 || w < 1 || h < 1 || w > nx_box || h > ny_box ||
      factor < 1 || w % factor || h % factor || !(E_ref > 0.0) || !alpha_dev || !mask_dev ||
      !x_dev)
    return LBM_ERR_ARG;
  const long total = (long)count * (w / factor) * (h / factor);
  k_encode_modulus<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>(
      alpha_dev, per_node ? 1 : 0, mask_dev, nx_box, (long)nx_box * ny_box, E_ref, w, h, factor,
      x_dev, count);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_warm_crop(int count, int nx_box, int ny_box, int w, int h, int to_box,
                         const uint8_t *mask_dev, const double *src_dev, double *dst_dev,
                         void *stream) {
  if (count < 1 || nx_box < 1 || ny_box < 1 || w < 1 || h < 1 || w > nx_box || h > ny_box ||
      !src_dev || !dst_dev || src_dev == dst_dev)
    return LBM_ERR_ARG;
  const long total = (long)count * 8 * (to_box ? (long)nx_box * ny_box : (long)w * h);
  k_crop<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>(src_dev, dst_dev, nx_box, ny_box, w,
                                                            h, to_box ? 1 : 0, mask_dev, count);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_warm_channel_rms(const float *t_dev, long pixels, float *rms_dev, void *stream) {
  if (!t_dev || pixels < 1 || !rms_dev) return LBM_ERR_ARG;
  k_channel_rms<<<8, 1024, 0, (cudaStream_t)stream>>>(t_dev, pixels, rms_dev);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_warm_combine(int count, long n, const double *w, const double *const *src_dev,
                            double *dst_dev, void *stream) {
  if (count < 1 || count > kMaxVec || n < 1 || !w || !src_dev || !dst_dev) return LBM_ERR_ARG;
  VecSet vs{};
  for (int j = 0; j < count; ++j) {
    if (!src_dev[j]) return LBM_ERR_ARG;
    vs.v[j] = src_dev[j];
    vs.w[j] = w[j];
  }
  k_combine<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(vs, count, n, dst_dev);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

long lbm_warm_dot_work_size(void) { return (long)kDotPairs * kDotBlocks + kDotPairs * 2 + 64; }

lbm_status lbm_warm_dots(int m, long n, const double *const *v_dev, double *work_dev,
                         double *out_host, void *stream) {
  if (m < 1 || m > kMaxVec + 1 || n < 1 || !v_dev || !work_dev || !out_host) return LBM_ERR_ARG;
  VecSet vs{};
  for (int j = 0; j < m; ++j) {
    if (!v_dev[j]) return LBM_ERR_ARG;
    vs.v[j] = v_dev[j];
  }
  cudaStream_t st = (cudaStream_t)stream;
  double *part = work_dev, *res = work_dev + (long)kDotPairs * kDotBlocks;
  k_dot_partial<<<kDotBlocks, 256, 0, st>>>(vs, m, n, part);
  k_dot_finish<<<1, 32, 0, st>>>(part, m, res);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaMemcpyAsync(out_host, res, sizeof(double) * m * m, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LBM_ERR_CUDA;
  return LBM_OK;
}

}  // extern "C"
