// Warm-start network on the GPU: a linear 4-level U-Net (3x3 circular convolutions,
// 2x2 average pooling, bilinear upsampling with skip concatenation, 1x1 head) mapping a
// 2-channel control field to the 8 steady populations.  BF16 activations and weights,
// FP32 accumulation with mma.sync.m16n8k16 (implicit GEMM, no im2col buffer), FP32
// master weights with Adam.  Training and inference kernels are all in this file.
//
// Tensors are NHWC with the channel count padded to a multiple of 16 (the input's two
// channels live in a 16-channel tensor whose other channels are zero).  A 3x3 weight is
// stored three ways: FP32 master [tap][ci][co] (the oracle's (3,3,Cin,Cout) order),
// BF16 [tap][co][ci] for the forward pass and BF16 [tap][ci][co] for the backward pass
// (the B operand wants its k index contiguous).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "lbm_solid.h"
#include "lbm_unet_tc.cuh"

namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t pack2(bf16 a, bf16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ float ldf(const bf16 &v) { return __bfloat162float(v); }
__device__ __forceinline__ float ldf(const float &v) { return v; }
__device__ __forceinline__ void stf(bf16 &d, float v) { d = __float2bfloat16_rn(v); }
__device__ __forceinline__ void stf(float &d, float v) { d = v; }

// A-operand word (two consecutive k) from BF16 activations, or the high and low BF16
// parts of two FP32 activations (x = hi + lo to 16 significant bits).
__device__ __forceinline__ void a_word(const bf16 *p, uint32_t &hi, uint32_t &lo) {
  hi = *reinterpret_cast<const uint32_t *>(p);
  lo = 0u;
}
__device__ __forceinline__ void a_word(const float *p, uint32_t &hi, uint32_t &lo) {
  const float2 v = *reinterpret_cast<const float2 *>(p);
  const bf16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y);
  hi = pack2(h0, h1);
  lo = pack2(__float2bfloat16_rn(v.x - __bfloat162float(h0)),
             __float2bfloat16_rn(v.y - __bfloat162float(h1)));
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Convolution as implicit GEMM: out[p, n] = bias[n] + sum_tap sum_k in[p + s*tap, k] *
// W[tap][n][k] with p = (b, y, x) and circular wrap in y, x; s = +1 (forward) or -1
// (gradient w.r.t. the input, with the transposed weight copy).  One warp: 16 pixels
// along x times 32 output channels (4 n-tiles of 8); grid.y over output-channel tiles.
// TIN = bf16: BF16 activations, one mma per fragment.  TIN = float: FP32 activations,
// each A fragment split into high and low BF16 parts and multiplied twice, so that the
// only rounding left is that of the BF16 weights themselves and the FP32 sums.
// Requires W % 16 == 0, Cin % 16 == 0, Cout % 8 == 0.
template <int KS, typename TIN>
__global__ void __launch_bounds__(128) k_conv(const TIN *__restrict__ in, int Cin,
                                              const bf16 *__restrict__ w, int Cout,
                                              const float *__restrict__ bias,
                                              bf16 *__restrict__ out_bf, float *__restrict__ out_f,
                                              int B, int H, int W, int sgn) {
  constexpr bool kSplit = sizeof(TIN) == 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const long tile = (long)blockIdx.x * 4 + warp;  // 16-pixel tile
  const long tiles_per_row = W / 16;
  const long total_tiles = (long)B * H * tiles_per_row;
  if (tile >= total_tiles) return;
  const int x0 = (int)(tile % tiles_per_row) * 16;
  const long by = tile / tiles_per_row;
  const int y = (int)(by % H);
  const int b = (int)(by / H);
  const int n0 = blockIdx.y * 32;
  const int R = KS / 2;
  float acc[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
  for (int dy = -R; dy <= R; ++dy) {
    const int ys = ((y + sgn * dy) % H + H) % H;
    for (int dx = -R; dx <= R; ++dx) {
      const int tap = (dy + R) * KS + (dx + R);
      const int xa = ((x0 + g + sgn * dx) % W + W) % W;
      const int xb = ((x0 + g + 8 + sgn * dx) % W + W) % W;
      const TIN *ra = in + (((long)b * H + ys) * W + xa) * Cin;
      const TIN *rb = in + (((long)b * H + ys) * W + xb) * Cin;
      const bf16 *wt = w + (long)tap * Cout * Cin;
      for (int k0 = 0; k0 < Cin; k0 += 16) {
        uint32_t a[4], al[4];
        a_word(ra + k0 + 2 * t, a[0], al[0]);
        a_word(rb + k0 + 2 * t, a[1], al[1]);
        a_word(ra + k0 + 2 * t + 8, a[2], al[2]);
        a_word(rb + k0 + 2 * t + 8, a[3], al[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = n0 + 8 * j + g;
          if (n0 + 8 * j >= Cout) break;
          const bf16 *wr = wt + (long)n * Cin + k0 + 2 * t;
          uint32_t bb[2];
          bb[0] = *reinterpret_cast<const uint32_t *>(wr);
          bb[1] = *reinterpret_cast<const uint32_t *>(wr + 8);
          mma16816(acc[j], a, bb);
          if (kSplit) mma16816(acc[j], al, bb);
        }
      }
    }
  }
  // epilogue: rows g and g+8 (pixels x0+g, x0+g+8), columns 2t, 2t+1 of each n-tile
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int nb = n0 + 8 * j;
    if (nb >= Cout) break;
    const int n = nb + 2 * t;
    const float b0 = bias ? bias[n] : 0.f, b1 = bias ? bias[n + 1] : 0.f;
    const long pa = (((long)b * H + y) * W + x0 + g) * Cout + n;
    const long pb = (((long)b * H + y) * W + x0 + g + 8) * Cout + n;
    if (out_f) {
      *reinterpret_cast<float2 *>(out_f + pa) = make_float2(acc[j][0] + b0, acc[j][1] + b1);
      *reinterpret_cast<float2 *>(out_f + pb) = make_float2(acc[j][2] + b0, acc[j][3] + b1);
    } else {
      *reinterpret_cast<uint32_t *>(out_bf + pa) =
          pack2(__float2bfloat16_rn(acc[j][0] + b0), __float2bfloat16_rn(acc[j][1] + b1));
      *reinterpret_cast<uint32_t *>(out_bf + pb) =
          pack2(__float2bfloat16_rn(acc[j][2] + b0), __float2bfloat16_rn(acc[j][3] + b1));
    }
  }
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// Weight gradient: gw[tap][ci][co] += sum_p in[p + tap, ci] gout[p, co], a GEMM with
// M = co, N = ci, K = pixels.  A block owns 64 output x 64 input channels of one tap and
// `ppb` consecutive pixels.  Per 64-pixel stage the 128 threads copy the gout rows
// (A, [pixel][co]) and the shifted input rows (B, [pixel][ci]) into shared memory with
// cp.async (two buffers, rows padded to 144 B so that ldmatrix is conflict-free); each
// warp reads its 16 output channels transposed with ldmatrix.trans into
// mma.sync.m16n8k16 fragments (K = 16 pixels per step).  The FP32 sums of the block are
// added into the unpadded [tap][ci_real][co_real] slice with atomics; only real channels
// are written.  Needs Cin, Cout multiples of 16.
template <int KS>
__global__ void __launch_bounds__(128) k_conv_wgrad(const bf16 *__restrict__ in, int Cin,
                                                    int ci_real, const bf16 *__restrict__ gout,
                                                    int Cout, int co_real,
                                                    float *__restrict__ gw, int B, int H, int W,
                                                    long ppb) {
  constexpr int kP = 64, kLd = 72;
  __shared__ __align__(16) bf16 sA[2][kP * kLd];
  __shared__ __align__(16) bf16 sB[2][kP * kLd];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int nci = (Cin + 63) / 64;
  const int tap = blockIdx.z / nci, cit = blockIdx.z % nci;
  const int R = KS / 2, dy = tap / KS - R, dx = tap % KS - R;
  const int co0 = blockIdx.y * 64, ci0 = cit * 64;
  const int mt = Cout - co0 < 64 ? Cout - co0 : 64;  // multiples of 16
  const int ntl = Cin - ci0 < 64 ? Cin - ci0 : 64;
  const long P = (long)B * H * W;
  const long pb = (long)blockIdx.x * ppb;
  if (pb >= P) return;
  const long pe = pb + ppb < P ? pb + ppb : P;
  const int stages = (int)((pe - pb + kP - 1) / kP);
  auto load = [&](int st, int buf) {
    const long ps = pb + (long)st * kP;
    const int ca = mt / 8, cb = ntl / 8;
    for (int q = tid; q < kP * ca; q += 128) {
      const int r = q / ca, c = q - r * ca;
      const long p = ps + r;
      const bool v = p < pe;
      tc::cp16(tc::smem_u32(&sA[buf][r * kLd + c * 8]), gout + (v ? p : 0) * Cout + co0 + c * 8, v);
    }
    for (int q = tid; q < kP * cb; q += 128) {
      const int r = q / cb, c = q - r * cb;
      const long p = ps + r;
      const bool v = p < pe;
      long row = 0;
      if (v) {
        const int x = (int)(p % W);
        const long rr = p / W;
        const int y = (int)(rr % H);
        const long b = rr / H;
        int ys = y + dy, xs = x + dx;
        ys = ys < 0 ? ys + H : (ys >= H ? ys - H : ys);
        xs = xs < 0 ? xs + W : (xs >= W ? xs - W : xs);
        row = (b * H + ys) * W + xs;
      }
      tc::cp16(tc::smem_u32(&sB[buf][r * kLd + c * 8]), in + row * Cin + ci0 + c * 8, v);
    }
    asm volatile("cp.async.commit_group;");
  };
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
  const bool active = 16 * warp < mt;
  const int tile = lane >> 3, rr8 = lane & 7;
  load(0, 0);
  for (int st = 0; st < stages; ++st) {
    if (st + 1 < stages) {
      load(st + 1, (st + 1) & 1);
      asm volatile("cp.async.wait_group 1;");
    } else {
      asm volatile("cp.async.wait_group 0;");
    }
    __syncthreads();
    const bf16 *A = sA[st & 1], *Bm = sB[st & 1];
    if (active) {
#pragma unroll
      for (int k0 = 0; k0 < kP; k0 += 16) {
        // A fragment: tiles (m 0-7, k 0-7), (m 8-15, k 0-7), (m 0-7, k 8-15), (m 8-15, k 8-15)
        uint32_t a[4];
        ldsm_x4_trans(a, tc::smem_u32(&A[(k0 + rr8 + ((tile & 2) ? 8 : 0)) * kLd + 16 * warp +
                                          ((tile & 1) ? 8 : 0)]));
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          if (8 * j >= ntl) break;
          // B fragments of n-tiles j, j + 1: (k 0-7, n), (k 8-15, n), (k 0-7, n+8), (k 8-15, n+8)
          uint32_t b4[4];
          ldsm_x4_trans(b4, tc::smem_u32(&Bm[(k0 + rr8 + ((tile & 1) ? 8 : 0)) * kLd + 8 * j +
                                             ((tile & 2) ? 8 : 0)]));
          const uint32_t b0[2] = {b4[0], b4[1]}, b1[2] = {b4[2], b4[3]};
          mma16816(acc[j], a, b0);
          mma16816(acc[j + 1], a, b1);
        }
      }
    }
    __syncthreads();  // this buffer is refilled two stages on
  }
  if (!active) return;
  float *dst = gw + (long)tap * ci_real * co_real;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (8 * j >= ntl) break;
    const int ci = ci0 + 8 * j + 2 * t;
    const int ma = co0 + 16 * warp + g, mb = ma + 8;
    if (ci < ci_real && ma < co_real) atomicAdd(dst + (long)ci * co_real + ma, acc[j][0]);
    if (ci + 1 < ci_real && ma < co_real) atomicAdd(dst + (long)(ci + 1) * co_real + ma, acc[j][1]);
    if (ci < ci_real && mb < co_real) atomicAdd(dst + (long)ci * co_real + mb, acc[j][2]);
    if (ci + 1 < ci_real && mb < co_real) atomicAdd(dst + (long)(ci + 1) * co_real + mb, acc[j][3]);
  }
}

// Bias gradient: gb[c] += sum_p gout[p, c].
__global__ void k_bias_grad(const bf16 *__restrict__ gout, int C, int stride, long P,
                            float *__restrict__ gb) {
  const int c = threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (long p = blockIdx.x; p < P; p += gridDim.x) s += __bfloat162float(gout[p * stride + c]);
  atomicAdd(gb + c, s);
}

template <typename T>
__global__ void k_pool(const T *__restrict__ in, T *__restrict__ out, int C, int B, int H, int W) {
  const int Ho = H / 2, Wo = W / 2;
  const long total = (long)B * Ho * Wo * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long r = i / C;
    const int x = (int)(r % Wo);
    r /= Wo;
    const int y = (int)(r % Ho), b = (int)(r / Ho);
    const T *s = in + (((long)b * H + 2 * y) * W + 2 * x) * C + c;
    const float v = ldf(s[0]) + ldf(s[C]) + ldf(s[(long)W * C]) + ldf(s[(long)W * C + C]);
    stf(out[i], 0.25f * v);
  }
}

// Bilinear 2x upsampling, periodic: each coarse value sits at the centre of its 2x2 fine
// block, so along each axis fine cell i takes 3/4 of coarse cell i/2 and 1/4 of the
// coarse neighbour on its side (i even: i/2 - 1, i odd: i/2 + 1).
__device__ __forceinline__ int up_nbr(int i, int n) {
  const int j = i >> 1;
  return (i & 1) ? (j + 1 == n ? 0 : j + 1) : (j == 0 ? n - 1 : j - 1);
}

// out (B,H,W,Ca+Cb) = [bilinear-upsampled a (B,H/2,W/2,Ca), skip (B,H,W,Cb)].
template <typename T>
__global__ void k_up_concat(const T *__restrict__ a, int Ca, const T *__restrict__ s, int Cb,
                            T *__restrict__ out, int B, int H, int W) {
  const int C = Ca + Cb, Hc = H / 2, Wc = W / 2;
  const long total = (long)B * H * W * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W);
    const long r = p / W;
    const int y = (int)(r % H), b = (int)(r / H);
    if (c < Ca) {
      const int x0 = x >> 1, x1 = up_nbr(x, Wc), y0 = y >> 1, y1 = up_nbr(y, Hc);
      const T *ab = a + (long)b * Hc * Wc * Ca + c;
      const float v = 0.5625f * ldf(ab[((long)y0 * Wc + x0) * Ca]) +
                      0.1875f * (ldf(ab[((long)y0 * Wc + x1) * Ca]) +
                                 ldf(ab[((long)y1 * Wc + x0) * Ca])) +
                      0.0625f * ldf(ab[((long)y1 * Wc + x1) * Ca]);
      stf(out[i], v);
    } else {
      out[i] = s[p * Cb + (c - Ca)];
    }
  }
}

// Backward of k_up_concat's upsampled part: coarse cell j gathers fine cells 2j and
// 2j+1 with weight 3/4 and 2j-1, 2j+2 with 1/4 along each axis (the skip slice of the
// gradient is read by k_pool_back_add).
__global__ void k_up_concat_back(const bf16 *__restrict__ g, int Ca, int Cb, bf16 *__restrict__ ga,
                                 int B, int H, int W) {
  const int C = Ca + Cb, Hc = H / 2, Wc = W / 2;
  const long total = (long)B * Hc * Wc * Ca;
  const float wt[4] = {0.25f, 0.75f, 0.75f, 0.25f};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % Ca);
    long r = i / Ca;
    const int x = (int)(r % Wc);
    r /= Wc;
    const int y = (int)(r % Hc), b = (int)(r / Hc);
    const bf16 *gb = g + (long)b * H * W * C + c;
    float v = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int fy = 2 * y - 1 + u;
      fy = fy < 0 ? fy + H : (fy >= H ? fy - H : fy);
      float row = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        int fx = 2 * x - 1 + t;
        fx = fx < 0 ? fx + W : (fx >= W ? fx - W : fx);
        row += wt[t] * __bfloat162float(gb[((long)fy * W + fx) * C]);
      }
      v += wt[u] * row;
    }
    ga[i] = __float2bfloat16_rn(v);
  }
}

// gfine (B,H,W,C) = 0.25 * gcoarse upsampled + gskip slice of gcat (channels Ca..Ca+C).
__global__ void k_pool_back_add(const bf16 *__restrict__ gcoarse, const bf16 *__restrict__ gcat,
                                int Ca, int C, bf16 *__restrict__ out, int B, int H, int W) {
  const long total = (long)B * H * W * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W);
    const long r = p / W;
    const int y = (int)(r % H), b = (int)(r / H);
    const float v = 0.25f * __bfloat162float(gcoarse[(((long)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]) +
                    __bfloat162float(gcat[p * (Ca + C) + Ca + c]);
    out[i] = __float2bfloat16_rn(v);
  }
}

// Input (B,H,W,2) FP32 -> 16 channels (2..15 zero), BF16 or FP32.
template <typename T>
__global__ void k_pack_input(const float *__restrict__ x, T *__restrict__ out, long P) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P * 16;
       i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % 16);
    stf(out[i], c < 2 ? x[(i / 16) * 2 + c] : 0.f);
  }
}

// MSE loss 0.5 mean (y - t)^2: per-block partial sums, and gy = (y - t) / n in BF16,
// stored with 16 channels per pixel (channels 8..15 stay zero) for the mma k-chunks.
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, long n,
                      bf16 *__restrict__ gy, float *__restrict__ partial) {
  __shared__ float sm[256];
  float s = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += d * d;
    gy[(i / 8) * 16 + (i % 8)] = __float2bfloat16_rn(d / (float)n);
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void k_sum_partials(const float *__restrict__ partial, int nb, float scale,
                               float *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < nb; ++i) s += partial[i];
    out[0] = s * scale;
  }
}

// Adam on the FP32 master copy, then refresh the two BF16 layouts of every 3x3 / 1x1
// weight.  Parameters of one layer: w [taps][ci][co] then b [co].
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// master w [tap][ci][co] (ci < ci_real) -> wf [tap][co][cipad], wb [tap][cipad][copad]
// (wb's channels co..copad-1 stay zero from the allocation)
__global__ void k_weights_bf16(const float *__restrict__ w, int taps, int ci_real, int cipad,
                               int co, int copad, bf16 *__restrict__ wf, bf16 *__restrict__ wb) {
  const long total = (long)taps * cipad * co;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int o = (int)(i % co);
    long r = i / co;
    const int c = (int)(r % cipad);
    const int tap = (int)(r / cipad);
    const float val = c < ci_real ? w[((long)tap * ci_real + c) * co + o] : 0.f;
    const bf16 bv = __float2bfloat16_rn(val);
    wf[((long)tap * co + o) * cipad + c] = bv;
    // input-gradient layout: the s = -1 convolution reads gout at p - (dy, dx) with the
    // same tap's weight transposed (grad_in[q] = sum_tap gout[q - off] w[tap]^T)
    wb[((long)tap * cipad + c) * copad + o] = bv;
  }
}

struct Layer {
  int ks, ci, cipad, co, copad;
  long woff, boff;         // offsets in the flat FP32 parameter vector
  bf16 *wf = nullptr, *wb = nullptr;
  bf16 *in = nullptr;      // saved input activation (B,H,W,cipad)
  bf16 *out = nullptr;     // output activation (B,H,W,co) (not for the head)
  bf16 *gin = nullptr;     // gradient w.r.t. the input
  int H, W;
};

}  // namespace

struct lbm_unet {
  int base, levels, B, H, W;
  cudaStream_t stream;
  std::vector<Layer> L;
  long nparams = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  float *y = nullptr, *partial = nullptr;
  bf16 *x16 = nullptr, *gy = nullptr;
  std::vector<bf16 *> pooled, upcat, gcoarse;  // per level
  // FP32 activations of the exact-activation forward (allocated on first use)
  float *x32 = nullptr;
  std::vector<float *> out32, pooled32, upcat32;
  int *err = nullptr;  // set by a tensor-core convolution whose wait timed out
  long step = 0;
  std::vector<void *> allocs;
};

namespace {

template <class T>
T *dalloc(lbm_unet *u, size_t n, cudaError_t &e) {
  void *p = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&p, n * sizeof(T));
  if (e == cudaSuccess) {
    u->allocs.push_back(p);
    cudaMemsetAsync(p, 0, n * sizeof(T), u->stream);
  }
  return static_cast<T *>(p);
}

unsigned gs(long n) { long b = (n + 255) / 256; return (unsigned)(b < 148 * 16 ? (b < 1 ? 1 : b) : 148 * 16); }

// 3x3 convolution on the tensor cores (tcgen05, accumulator in TMEM): Kc-channel chunks
// (64, 32 or 16, dividing Cin), N-tiles of up to 256 output channels (384 = 2 x 192).
template <typename TIN>
void conv3_tc(lbm_unet *u, const TIN *in, int Cin, const bf16 *w, int Cout, const float *bias,
              bf16 *out_bf, float *out_f, int Hh, int Ww, int sgn) {
  const int kc = Cin % 64 == 0 ? 64 : (Cin % 32 == 0 ? 32 : 16);
  int nt = Cout <= 256 ? Cout : (Cout % 192 == 0 ? 192 : 128);
  const long P = (long)u->B * Hh * Ww;
  const long mt = (P + tc::kM - 1) / tc::kM;
  // coarse levels have few pixels: narrower N-tiles put more CTAs on the 148 SMs
  while (mt * (Cout / nt) < 148 && nt % 32 == 0 && Cout % (nt / 2) == 0) nt /= 2;
  int tcols = 32;
  while (tcols < nt) tcols *= 2;
  const bool split = sizeof(TIN) == 4;
  size_t smem = tc::kBufs * ((size_t)tc::kM * kc * 2 * (split ? 2 : 1) + (size_t)nt * kc * 2);
  // at most 512 / tcols CTAs per SM, so that their TMEM allocations always fit
  if (smem < (size_t)tcols * 456) smem = (size_t)tcols * 456;
  // the opt-in shared-memory size is per device: set it on every launch (cheap)
  cudaFuncSetAttribute(tc::k_conv3<TIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  dim3 grid((unsigned)mt, (unsigned)(Cout / nt));
  tc::k_conv3<TIN><<<grid, tc::kThreads, smem, u->stream>>>(in, Cin, w, Cout, bias, out_bf, out_f,
                                                           u->B, Hh, Ww, sgn, kc, nt, tcols, u->err);
}

template <typename TIN>
void conv_fwd(lbm_unet *u, const Layer &l, const TIN *in, bf16 *out_bf, float *out_f, int Hh, int Ww) {
  const float *bias = u->p + l.boff;
  if (l.ks == 3) {
    conv3_tc<TIN>(u, in, l.cipad, l.wf, l.co, bias, out_bf, out_f, Hh, Ww, 1);
    return;
  }
  const long tiles = (long)u->B * Hh * (Ww / 16);
  dim3 grid((unsigned)((tiles + 3) / 4), (unsigned)((l.co + 31) / 32));
  k_conv<1, TIN><<<grid, 128, 0, u->stream>>>(in, l.cipad, l.wf, l.co, bias, out_bf, out_f, u->B, Hh, Ww, 1);
}

// a layer's output in the activation type of the pass
void conv_out(lbm_unet *u, const Layer &l, const bf16 *in, bf16 *out, int Hh, int Ww) {
  conv_fwd<bf16>(u, l, in, out, nullptr, Hh, Ww);
}
void conv_out(lbm_unet *u, const Layer &l, const float *in, float *out, int Hh, int Ww) {
  conv_fwd<float>(u, l, in, nullptr, out, Hh, Ww);
}

// Forward pass with activations of type T: BF16 (training; the layer inputs are kept
// for the backward pass) or FP32 (exact activations).  outs[i]: output of layer i.
template <typename T>
void forward_t(lbm_unet *u, const float *x, T *xin, const std::vector<T *> &outs,
               const std::vector<T *> &pooled, const std::vector<T *> &upcat, bool save) {
  const int lv = u->levels;
  const long P = (long)u->B * u->H * u->W;
  k_pack_input<T><<<gs(P * 16), 256, 0, u->stream>>>(x, xin, P);
  const T *h = xin;
  int li = 0;
  auto keep = [&](Layer &ly, const T *in) {
    if (save) ly.in = reinterpret_cast<bf16 *>(const_cast<T *>(in));
  };
  for (int l = 0; l < lv; ++l) {
    const int ia = li++, ib = li++;
    Layer &a = u->L[ia], &b = u->L[ib];
    keep(a, h);
    conv_out(u, a, h, outs[ia], a.H, a.W);
    keep(b, outs[ia]);
    conv_out(u, b, outs[ia], outs[ib], b.H, b.W);
    h = outs[ib];
    if (l + 1 < lv) {
      k_pool<T><<<gs((long)u->B * b.H * b.W * b.co / 4), 256, 0, u->stream>>>(h, pooled[l], b.co,
                                                                              u->B, b.H, b.W);
      h = pooled[l];
    }
  }
  for (int l = lv - 2; l >= 0; --l) {
    const int ia = li++, ib = li++;
    Layer &a = u->L[ia], &b = u->L[ib];
    const int cu = a.ci - u->L[2 * l + 1].co;  // channels of the upsampled path
    k_up_concat<T><<<gs((long)u->B * a.H * a.W * a.ci), 256, 0, u->stream>>>(
        h, cu, outs[2 * l + 1], a.ci - cu, upcat[l], u->B, a.H, a.W);
    keep(a, upcat[l]);
    conv_out(u, a, upcat[l], outs[ia], a.H, a.W);
    keep(b, outs[ia]);
    conv_out(u, b, outs[ia], outs[ib], b.H, b.W);
    h = outs[ib];
  }
  Layer &hd = u->L[li];
  keep(hd, h);
  conv_fwd<T>(u, hd, h, nullptr, u->y, hd.H, hd.W);
}

// gradient w.r.t. the input of layer l (output in gin, cipad channels), and weight/bias
// grads; gout has copad channels (the head's 8 output channels padded to 16 with zeros)
void conv_bwd(lbm_unet *u, Layer &l, const bf16 *gout, int Hh, int Ww, bool need_gin) {
  const long P = (long)u->B * Hh * Ww;
  if (need_gin) {
    const long tiles = P / 16;
    dim3 grid((unsigned)((tiles + 3) / 4), (unsigned)((l.cipad + 31) / 32));
    if (l.ks == 3)
      conv3_tc<bf16>(u, gout, l.copad, l.wb, l.cipad, nullptr, l.gin, nullptr, Hh, Ww, -1);
    else
      k_conv<1, bf16><<<grid, 128, 0, u->stream>>>(gout, l.copad, l.wb, l.cipad, nullptr, l.gin, nullptr, u->B, Hh, Ww, -1);
  }
  const long ppb = 1024;  // pixels per block (K range); partial sums meet in atomics
  const unsigned nci = (unsigned)((l.cipad + 63) / 64);
  dim3 grid((unsigned)((P + ppb - 1) / ppb), (unsigned)((l.copad + 63) / 64),
            (unsigned)(l.ks * l.ks) * nci);
  if (l.ks == 3)
    k_conv_wgrad<3><<<grid, 128, 0, u->stream>>>(l.in, l.cipad, l.ci, gout, l.copad, l.co, u->g + l.woff, u->B, Hh, Ww, ppb);
  else
    k_conv_wgrad<1><<<grid, 128, 0, u->stream>>>(l.in, l.cipad, l.ci, gout, l.copad, l.co, u->g + l.woff, u->B, Hh, Ww, ppb);
  k_bias_grad<<<148 * 4, l.co, 0, u->stream>>>(gout, l.co, l.copad, P, u->g + l.boff);
}

}  // namespace

extern "C" {

lbm_status lbm_unet_create(int base, int levels, int batch, int H, int W, unsigned long long seed,
                           void *stream, lbm_unet **out) {
  if (!out || base < 16 || base % 16 || levels < 1 || levels > 5 || batch < 1) return LBM_ERR_ARG;
  const int div = 16 << (levels - 1);  // coarsest level still has W % 16 == 0
  if (H % (1 << (levels - 1)) || W % div || base << (levels - 1) > 256) return LBM_ERR_ARG;
  *out = nullptr;
  lbm_unet *u = new (std::nothrow) lbm_unet();
  if (!u) return LBM_ERR_OOM;
  u->base = base; u->levels = levels; u->B = batch; u->H = H; u->W = W;
  u->stream = (cudaStream_t)stream;
  // layers in execution order (same as the CPU reference)
  std::vector<int> ch(levels);
  for (int l = 0; l < levels; ++l) ch[l] = base << l;
  auto add = [&](int ks, int ci, int co, int h, int w) {
    Layer ly;
    ly.ks = ks; ly.ci = ci; ly.cipad = (ci + 15) / 16 * 16; ly.co = co; ly.H = h; ly.W = w;
    ly.copad = (co + 15) / 16 * 16;
    ly.woff = u->nparams;
    u->nparams += (long)ks * ks * ci * co;
    ly.boff = u->nparams;
    u->nparams += co;
    u->L.push_back(ly);
  };
  int c = 2;
  for (int l = 0; l < levels; ++l) {
    add(3, c, ch[l], H >> l, W >> l);
    add(3, ch[l], ch[l], H >> l, W >> l);
    c = ch[l];
  }
  for (int l = levels - 2; l >= 0; --l) {
    add(3, ch[l + 1] + ch[l], ch[l], H >> l, W >> l);
    add(3, ch[l], ch[l], H >> l, W >> l);
  }
  add(1, ch[0], 8, H, W);
  cudaError_t e = cudaSuccess;
  u->p = dalloc<float>(u, u->nparams, e);
  u->g = dalloc<float>(u, u->nparams, e);
  u->m = dalloc<float>(u, u->nparams, e);
  u->v = dalloc<float>(u, u->nparams, e);
  const long P = (long)batch * H * W;
  u->y = dalloc<float>(u, P * 8, e);
  u->err = dalloc<int>(u, 1, e);
  u->partial = dalloc<float>(u, 148 * 16, e);
  u->x16 = dalloc<bf16>(u, P * 16, e);
  u->gy = dalloc<bf16>(u, P * 16, e);
  for (auto &ly : u->L) {
    const long Pl = (long)batch * ly.H * ly.W;
    ly.wf = dalloc<bf16>(u, (size_t)ly.ks * ly.ks * ly.cipad * ly.co, e);
    ly.wb = dalloc<bf16>(u, (size_t)ly.ks * ly.ks * ly.cipad * ly.copad, e);
    ly.out = dalloc<bf16>(u, Pl * ly.co, e);
    ly.gin = dalloc<bf16>(u, Pl * ly.cipad, e);
  }
  for (int l = 0; l < levels; ++l) {
    const long Pl = (long)batch * (H >> l) * (W >> l);
    u->pooled.push_back(l + 1 < levels ? dalloc<bf16>(u, Pl / 4 * ch[l], e) : nullptr);
    u->upcat.push_back(l + 1 < levels ? dalloc<bf16>(u, Pl * (ch[l] + ch[l + 1]), e) : nullptr);
    u->gcoarse.push_back(l + 1 < levels ? dalloc<bf16>(u, Pl / 4 * ch[l + 1], e) : nullptr);
  }
  if (e != cudaSuccess) {
    for (void *q : u->allocs) cudaFree(q);
    delete u;
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
  }
  // fan-in scaled normal weights, zero biases (host RNG, uploaded once)
  std::vector<float> hp(u->nparams, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  for (auto &ly : u->L) {
    const float sc = std::sqrt(1.f / (ly.ks * ly.ks * ly.ci));
    for (long i = 0; i < (long)ly.ks * ly.ks * ly.ci * ly.co; ++i) hp[ly.woff + i] = sc * nd(rng);
  }
  if (cudaMemcpy(u->p, hp.data(), sizeof(float) * u->nparams, cudaMemcpyHostToDevice) != cudaSuccess) {
    for (void *q : u->allocs) cudaFree(q);
    delete u;
    return LBM_ERR_CUDA;
  }
  for (auto &ly : u->L)
    k_weights_bf16<<<gs((long)ly.ks * ly.ks * ly.cipad * ly.co), 256, 0, u->stream>>>(
        u->p + ly.woff, ly.ks * ly.ks, ly.ci, ly.cipad, ly.co, ly.copad, ly.wf, ly.wb);
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) {
    for (void *q : u->allocs) cudaFree(q);
    delete u;
    return LBM_ERR_CUDA;
  }
  *out = u;
  return LBM_OK;
}

lbm_status lbm_unet_destroy(lbm_unet *u) {
  if (!u) return LBM_ERR_ARG;
  cudaStreamSynchronize(u->stream);
  for (void *q : u->allocs) cudaFree(q);
  delete u;
  return LBM_OK;
}

long lbm_unet_param_count(const lbm_unet *u) { return u ? u->nparams : -1; }

lbm_status lbm_unet_status(lbm_unet *u) {
  if (!u) return LBM_ERR_ARG;
  int h = 0;
  if (cudaMemcpyAsync(&h, u->err, sizeof(int), cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
      cudaStreamSynchronize(u->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (h && cudaMemsetAsync(u->err, 0, sizeof(int), u->stream) != cudaSuccess) return LBM_ERR_CUDA;
  return h ? LBM_ERR_CUDA : LBM_OK;
}

lbm_status lbm_unet_get_params(lbm_unet *u, float *dst, int which) {
  if (!u || !dst) return LBM_ERR_ARG;
  const float *src = which == 0 ? u->p : u->g;
  return cudaMemcpyAsync(dst, src, sizeof(float) * u->nparams, cudaMemcpyDeviceToDevice, u->stream) ==
                 cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_unet_set_params(lbm_unet *u, const float *src) {
  if (!u || !src) return LBM_ERR_ARG;
  if (cudaMemcpyAsync(u->p, src, sizeof(float) * u->nparams, cudaMemcpyDeviceToDevice, u->stream) !=
      cudaSuccess)
    return LBM_ERR_CUDA;
  for (auto &ly : u->L)
    k_weights_bf16<<<gs((long)ly.ks * ly.ks * ly.cipad * ly.co), 256, 0, u->stream>>>(
        u->p + ly.woff, ly.ks * ly.ks, ly.ci, ly.cipad, ly.co, ly.copad, ly.wf, ly.wb);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// Forward pass: x (B,H,W,2) FP32 -> y (B,H,W,8) FP32 (y_dev may be NULL: kept inside).
// exact_acts = 0: BF16 activations (the training pass); 1: FP32 activations.
lbm_status lbm_unet_forward(lbm_unet *u, const float *x, float *y_out, int exact_acts) {
  if (!u || !x) return LBM_ERR_ARG;
  const long P = (long)u->B * u->H * u->W;
  if (exact_acts) {
    if (!u->x32) {
      cudaError_t e = cudaSuccess;
      u->x32 = dalloc<float>(u, P * 16, e);
      for (auto &ly : u->L) u->out32.push_back(dalloc<float>(u, (long)u->B * ly.H * ly.W * ly.co, e));
      for (int l = 0; l < u->levels; ++l) {
        const long Pl = (long)u->B * (u->H >> l) * (u->W >> l);
        const int c = u->base << l;
        u->pooled32.push_back(l + 1 < u->levels ? dalloc<float>(u, Pl / 4 * c, e) : nullptr);
        u->upcat32.push_back(l + 1 < u->levels ? dalloc<float>(u, Pl * (c + 2 * c), e) : nullptr);
      }
      if (e != cudaSuccess) {
        u->x32 = nullptr;  // buffers stay in allocs and are freed by destroy
        u->out32.clear(); u->pooled32.clear(); u->upcat32.clear();
        return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
      }
    }
    forward_t<float>(u, x, u->x32, u->out32, u->pooled32, u->upcat32, false);
  } else {
    std::vector<bf16 *> outs;
    for (auto &ly : u->L) outs.push_back(ly.out);
    forward_t<bf16>(u, x, u->x16, outs, u->pooled, u->upcat, true);
  }
  if (y_out &&
      cudaMemcpyAsync(y_out, u->y, sizeof(float) * P * 8, cudaMemcpyDeviceToDevice, u->stream) !=
          cudaSuccess)
    return LBM_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// One training step on a batch: forward, loss 0.5 mean (y - t)^2 (written to loss_dev),
// backward into the gradient vector, and (lr > 0) one Adam step.
lbm_status lbm_unet_train_step(lbm_unet *u, const float *x, const float *t, float lr,
                               float *loss_dev) {
  if (!u || !x || !t) return LBM_ERR_ARG;
  lbm_status st = lbm_unet_forward(u, x, nullptr, 0);
  if (st) return st;
  const int lv = u->levels;
  const long P = (long)u->B * u->H * u->W;
  const unsigned nb = 148 * 4;
  k_mse<<<nb, 256, 0, u->stream>>>(u->y, t, P * 8, u->gy, u->partial);
  if (loss_dev) k_sum_partials<<<1, 32, 0, u->stream>>>(u->partial, nb, 0.5f / (float)(P * 8), loss_dev);
  cudaMemsetAsync(u->g, 0, sizeof(float) * u->nparams, u->stream);
  int li = (int)u->L.size() - 1;
  Layer &hd = u->L[li--];
  conv_bwd(u, hd, u->gy, hd.H, hd.W, true);
  const bf16 *g = hd.gin;
  std::vector<const bf16 *> gskip(lv, nullptr);
  for (int l = 0; l < lv - 1; ++l) {  // decoder, reverse execution order
    Layer &b = u->L[li--], &a = u->L[li--];
    conv_bwd(u, b, g, b.H, b.W, true);
    conv_bwd(u, a, b.gin, a.H, a.W, true);
    const int cskip = u->L[2 * l + 1].co, cu = a.ci - cskip;
    // gradient of the upsampled part -> coarse level; the skip slice stays in a.gin
    k_up_concat_back<<<gs((long)u->B * (a.H / 2) * (a.W / 2) * cu), 256, 0, u->stream>>>(
        a.gin, cu, cskip, u->gcoarse[l], u->B, a.H, a.W);
    gskip[l] = a.gin;
    g = u->gcoarse[l];
  }
  for (int l = lv - 1; l >= 0; --l) {
    Layer &b = u->L[2 * l + 1], &a = u->L[2 * l];
    const bf16 *gl = g;
    if (l < lv - 1) {
      // gradient of enc_b output = 0.25 * upsampled (pooling) gradient + skip slice
      const int cu = u->L[2 * (l + 1) + 1].co;  // C_{l+1}: the upsampled part of dec_a(l)
      k_pool_back_add<<<gs((long)u->B * b.H * b.W * b.co), 256, 0, u->stream>>>(
          g, gskip[l], cu, b.co, u->upcat[l], u->B, b.H, b.W);
      gl = u->upcat[l];  // reuse the concat buffer (large enough) as scratch
    }
    conv_bwd(u, b, gl, b.H, b.W, true);
    conv_bwd(u, a, b.gin, a.H, a.W, l > 0);
    g = a.gin;
  }
  if (lr > 0.f) {
    ++u->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)u->step), c2 = 1.f - std::pow(b2, (float)u->step);
    k_adam<<<gs(u->nparams), 256, 0, u->stream>>>(u->p, u->g, u->m, u->v, u->nparams, lr, b1, b2,
                                                  1e-8f, c1, c2);
    for (auto &ly : u->L)
      k_weights_bf16<<<gs((long)ly.ks * ly.ks * ly.cipad * ly.co), 256, 0, u->stream>>>(
          u->p + ly.woff, ly.ks * ly.ks, ly.ci, ly.cipad, ly.co, ly.copad, ly.wf, ly.wb);
  }
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // extern "C"
