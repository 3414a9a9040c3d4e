// 3x3 circular convolution of the warm-start network on the 5th-generation tensor cores:
// an implicit GEMM whose 128-pixel x N accumulator lives in tensor memory.
//
//   out[p, n] = bias[n] + sum_tap sum_k in[p + s (dy, dx)_tap, k] W[tap][n][k]
//
// p = flattened pixel (b, y, x) of an NHWC tensor with circular wrap in y and x; s = +1
// (forward) or -1 (gradient w.r.t. the input, with the transposed weight copy).  One
// CTA owns 128 consecutive pixels (the M = 128 rows of tcgen05.mma, one TMEM lane each)
// and an N-tile of output channels (TMEM columns).  The K loop runs over taps and
// Kc-channel chunks: the 128 threads stage the im2col rows of A and the weight rows of B
// into shared memory (cp.async, 16 B per copy; FP32 activations are split into high and
// low BF16 parts on the way, two A tiles, two MMAs), in the no-swizzle K-major layout of
// 8-row x 16-byte core matrices; one thread issues Kc/16 tcgen05.mma (kind::f16, BF16
// inputs, FP32 accumulation) per chunk and commits them to the buffer's mbarrier.  Three
// buffers: the copies of chunk i + 1 are in flight while chunks i - 1 and i multiply, so
// the tensor core gets chunk i without waiting for chunk i - 1 to finish.  The epilogue
// reads the accumulator with tcgen05.ld (warp w: lanes 32w..32w+31), adds the bias and
// stores BF16 or FP32 rows.
//
// Every mbarrier wait is bounded; on a timeout the CTA sets *err, stops issuing, waits
// (bounded) for what it issued, writes NaN to its outputs, frees its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace tc {

constexpr int kM = 128;        // pixels per CTA = TMEM lanes
constexpr int kThreads = 128;  // four warps
constexpr long kSpin = 1L << 22;
constexpr int kBufs = 3;       // operand buffers: chunk i + 1 loads while i and i - 1 multiply

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: start address, LBO = byte distance between
// core matrices adjacent along K, SBO = between adjacent 8-row groups; fixed 0b001 at 46.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(bar)));
}

// bounded wait for the phase with parity `par`; false on timeout
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t par) {
  const uint32_t a = smem_u32(bar);
  for (long i = 0; i < kSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(par));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(valid ? 16 : 0));
}

__device__ __forceinline__ uint32_t bfpack(float a, float b) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// Byte offset of (row r, 16-byte chunk c8) in a no-swizzle K-major tile of kc channels:
// core matrix (r / 8, c8) at (r / 8) * SBO + c8 * 128, SBO = kc * 16; row r % 8 at 16 B.
__device__ __forceinline__ uint32_t tile_off(int r, int c8, int kc) {
  return (uint32_t)((r & 7) * 16 + (r >> 3) * (kc * 16) + c8 * 128);
}

// TIN = bf16 (activations copied as they are) or float (split into hi + lo BF16).
// Layout of the dynamic shared memory: per buffer [A_hi | A_lo (float only) | B].
template <typename TIN>
__global__ void __launch_bounds__(kThreads) k_conv3(
    const TIN *__restrict__ in, int Cin, const __nv_bfloat16 *__restrict__ w, int Cout,
    const float *__restrict__ bias, __nv_bfloat16 *__restrict__ out_bf, float *__restrict__ out_f,
    int B, int H, int W, int sgn, int kc, int nt, int tcols, int *__restrict__ err) {
  constexpr bool kSplit = sizeof(TIN) == 4;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[kBufs];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long P = (long)B * H * W;
  const long p0 = (long)blockIdx.x * kM;
  const int n0 = blockIdx.y * nt;
  const uint32_t a_bytes = (uint32_t)kM * kc * 2, b_bytes = (uint32_t)nt * kc * 2;
  const uint32_t buf_bytes = a_bytes * (kSplit ? 2 : 1) + b_bytes;
  const uint32_t sbase = smem_u32(smem);

  if (tid == 0) {
    for (int b2 = 0; b2 < kBufs; ++b2)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[b2])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;

  // the 128 rows' pixel coordinates are fixed; per tap only the shift changes
  const int cpr = kc / 8;  // 16-byte chunks per row of a tile
  const int ksteps = Cin / kc;
  const int iters = 9 * ksteps;
  const uint32_t id = idesc(nt);
  bool ok = true;
  // the pixel (b, y, x) of each A row this thread copies: rows q / cpr for
  // q = tid, tid + 128, ... (at most 8 of them); -1 = beyond the last pixel
  constexpr int kMaxRows = kM * 8 / kThreads;
  long rb[kMaxRows];
  int ry[kMaxRows], rx[kMaxRows];
#pragma unroll
  for (int i = 0; i < kMaxRows; ++i) {
    const int q = tid + i * kThreads;
    const long p = p0 + q / cpr;
    rb[i] = -1;
    ry[i] = rx[i] = 0;
    if (q < kM * cpr && p < P) {
      rx[i] = (int)(p % W);
      const long t = p / W;
      ry[i] = (int)(t % H);
      rb[i] = (t / H) * H;
    }
  }
  // stage the operands of K-chunk `it` into buffer it % kBufs
  auto load = [&](int it) {
    const int buf = it % kBufs;
    const int tap = it / ksteps, k0 = (it % ksteps) * kc;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const uint32_t abase = sbase + buf * buf_bytes;
    const uint32_t bbase = abase + a_bytes * (kSplit ? 2 : 1);
    // A: kM rows x kc channels of the shifted pixels
#pragma unroll
    for (int i = 0; i < kMaxRows; ++i) {
      const int q = tid + i * kThreads;
      if (q >= kM * cpr) break;
      const int r = q / cpr, c8 = q - r * cpr;
      const bool valid = rb[i] >= 0;
      long src = 0;
      if (valid) {
        int ys = ry[i] + sgn * dy, xs = rx[i] + sgn * dx;
        ys = ys < 0 ? ys + H : (ys >= H ? ys - H : ys);
        xs = xs < 0 ? xs + W : (xs >= W ? xs - W : xs);
        src = ((rb[i] + ys) * W + xs) * Cin + k0 + c8 * 8;
      }
      const uint32_t off = tile_off(r, c8, kc);
      if (!kSplit) {
        cp16(abase + off, in + src, valid);
      } else {
        float v[8];
        if (valid) {
          const float4 u0 = *reinterpret_cast<const float4 *>(in + src);
          const float4 u1 = *reinterpret_cast<const float4 *>(in + src + 4);
          v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
          v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = 0.f;
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float h0 = __bfloat162float(__float2bfloat16_rn(v[2 * j]));
          const float h1 = __bfloat162float(__float2bfloat16_rn(v[2 * j + 1]));
          hi[j] = bfpack(h0, h1);
          lo[j] = bfpack(v[2 * j] - h0, v[2 * j + 1] - h1);
        }
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(abase + off), "r"(hi[0]),
                     "r"(hi[1]), "r"(hi[2]), "r"(hi[3]));
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(abase + a_bytes + off),
                     "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]));
      }
    }
    // B: nt weight rows x kc channels
    const __nv_bfloat16 *wt = w + ((long)tap * Cout + n0) * Cin + k0;
    for (int q = tid; q < nt * cpr; q += kThreads) {
      const int n = q / cpr, c8 = q - n * cpr;
      cp16(bbase + tile_off(n, c8, kc), wt + (long)n * Cin + c8 * 8, true);
    }
    asm volatile("cp.async.commit_group;");
  };
  load(0);
  for (int it = 0; it < iters; ++it) {
    // prefetch chunk it + 1 once the MMAs of chunk it + 1 - kBufs, the last to read its
    // buffer, are done (block-uniform decision); chunk it's MMAs then never wait for
    // chunk it - 1's
    if (it + 1 < iters) {
      const int prev = it + 1 - kBufs;
      const bool w_ok = prev < 0 || wait_bar(&bar[(it + 1) % kBufs], (uint32_t)((prev / kBufs) & 1));
      if (!__syncthreads_and(w_ok)) {
        ok = false;
        break;
      }
      load(it + 1);
      asm volatile("cp.async.wait_group 1;");  // chunk it has landed, it + 1 may be in flight
    } else {
      asm volatile("cp.async.wait_group 0;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      const uint32_t abase = sbase + (it % kBufs) * buf_bytes;
      const uint32_t bbase = abase + a_bytes * (kSplit ? 2 : 1);
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sbo = (uint32_t)kc * 16;
      for (int j = 0; j < kc / 16; ++j) {
        const uint64_t bd = sdesc(bbase + j * 256, 128, sbo);
        mma(tmem, sdesc(abase + j * 256, 128, sbo), bd, id, (it > 0 || j > 0) ? 1u : 0u);
        if (kSplit) mma(tmem, sdesc(abase + a_bytes + j * 256, 128, sbo), bd, id, 1u);
      }
      commit(&bar[it % kBufs]);
    }
  }
  // the last commit covers every MMA issued before it
  if (ok) ok = wait_bar(&bar[(iters - 1) % kBufs], (uint32_t)(((iters - 1) / kBufs) & 1));
  ok = __syncthreads_and(ok);
  if (!ok) {
    atomicExch(err, 1);
    // let anything still queued drain before the accumulator is released
    for (int b2 = 0; b2 < kBufs; ++b2) wait_bar(&bar[b2], 0), wait_bar(&bar[b2], 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // epilogue: warp w holds rows 32w + lane
  const long p = p0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c = 0; c < nt; c += 16) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(trow + (uint32_t)c));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (p < P) {
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        v[j] = ok ? __uint_as_float(r[j]) + (bias ? bias[n0 + c + j] : 0.f) : __int_as_float(0x7fc00000);
      const long o = p * Cout + n0 + c;
      if (out_f) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4 *>(out_f + o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      } else {
        uint4 q0, q1;
        q0.x = bfpack(v[0], v[1]); q0.y = bfpack(v[2], v[3]);
        q0.z = bfpack(v[4], v[5]); q0.w = bfpack(v[6], v[7]);
        q1.x = bfpack(v[8], v[9]); q1.y = bfpack(v[10], v[11]);
        q1.z = bfpack(v[12], v[13]); q1.w = bfpack(v[14], v[15]);
        *reinterpret_cast<uint4 *>(out_bf + o) = q0;
        *reinterpret_cast<uint4 *>(out_bf + o + 8) = q1;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

}  // namespace tc
