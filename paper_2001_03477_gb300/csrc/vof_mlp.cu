// vof_mlp.cu -- the learned interface normal on the 5th-generation tensor
// cores (tcgen05, accumulators in tensor memory).
//
// The paper reconstructs the interface normal with MYC (Sec. 3.2, Eq.
// plane_m, [Aulisa07]).  The learned-normal form replaces it by a small
// network that maps the 27 volume fractions of a cell's 3x3x3 stencil to the
// normal, 27 -> 64 -> 64 -> 3 with GELU (x Phi(x)), inputs 2 c - 1, output
// direction y / |y|_1, with MYC kept as the fallback wherever the network's
// plane fits the stencil worse than MYC's (plane residual: RMS over the 26
// neighbours of the plane's volume minus c; the network's normal is kept
// when its residual is at most 1.25 x MYC's + 1e-3).
//
// Arithmetic.  Weights are BF16 (round to nearest even of the FP32 master
// weights), accumulation FP32 in tensor memory.  The activations (inputs
// and hidden layers) enter the BF16 multiplications as the sum of three BF16
// numbers, hi + mid + lo, which carries the FP32 value to ~2^-24 relative:
// every product of the network is then formed with the BF16 weight and an
// FP32-accurate activation, so the forward pass agrees with the same network
// evaluated in FP64 with the same BF16 weights to FP32 accumulation error.
// Gradient contractions use two-term splits (hi + lo) of both operands.
//
// Tensor-core use (one CTA of 128 threads per tile of 128 stencils):
//   * operands in shared memory in the canonical K-major layout without
//     swizzle: 8-row x 16-byte core matrices, K-adjacent core matrices 128 B
//     apart (leading byte offset), 8-row groups KC x 128 B apart (stride
//     byte offset), KC = K / 8;
//   * tcgen05.mma.cta_group::1.kind::f16, M = 128, BF16 x BF16 -> FP32,
//     issued by one thread; completion through tcgen05.commit on an
//     mbarrier; row r of the accumulator is tensor-memory lane r, read back
//     by the thread of that row with tcgen05.ld 32x32b;
//   * every mbarrier wait is bounded by one second of the global timer;
//     a wait that gives up sets a device status bit, the CTA frees its
//     tensor memory and returns.
#include <cuda_bf16.h>

#include "../../include/vofgb.h"
#include "vof_launch.h"

namespace vofgb {
namespace mlp {

constexpr int kIn = 27, kK1 = 32, kH = 64, kOut = 3, kN3 = 16;
constexpr int kRows = 128;
constexpr int kThreads = 128;

// master parameter vector (FP32), the order of the C ABI
constexpr int oW1 = 0;                  // W1[64][27]
constexpr int oB1 = oW1 + kH * kIn;     // b1[64]
constexpr int oW2 = oB1 + kH;           // W2[64][64]
constexpr int oB2 = oW2 + kH * kH;      // b2[64]
constexpr int oW3 = oB2 + kH;           // W3[3][64]
constexpr int oB3 = oW3 + kOut * kH;    // b3[3]
constexpr int kParams = oB3 + kOut;     // 6147

// Byte offset of element (row r, k) in a canonical K-major image with KC
// core matrices along K.
__host__ __device__ constexpr uint32_t canon(int r, int k, int KC) {
  return ((uint32_t)((r >> 3) * KC + (k >> 3)) << 7) + ((uint32_t)(r & 7) << 4) + ((uint32_t)(k & 7) << 1);
}

// packed parameters (device buffer written by the pack / Adam kernels)
constexpr uint32_t pW1 = 0;                     // [64 rows][K 32] bf16, K-major
constexpr uint32_t pW2 = pW1 + kH * kK1 * 2;    // [64][64]: rows = output j, K = input k
constexpr uint32_t pW3 = pW2 + kH * kH * 2;     // [16][64]: rows 0..2 used
constexpr uint32_t pW2T = pW3 + kN3 * kH * 2;   // [64][64]: rows = input k, K = output j
constexpr uint32_t pW3F = pW2T + kH * kH * 2;   // W3 as FP32 [3][64] (bf16 values)
constexpr uint32_t pB = pW3F + kOut * kH * 4;   // b1[64], b2[64], b3[16] FP32
constexpr uint32_t kPackedBytes = pB + (kH + kH + kN3) * 4;
constexpr uint32_t kInferWBytes = pW2T;         // the three images inference loads

constexpr float kFallbackRatio = 1.25f;
constexpr float kFallbackTol = 1e-3f;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// shared-memory matrix descriptor: start, leading (K) and stride (8-row)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait on phase `parity`; false after one second without completion
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = su32(bar);
  const uint64_t t0 = gtimer();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (gtimer() - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// warp-wide: allocate ncols tensor-memory columns, address written to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] . B[smem]^T, one thread
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's lane, waited for in the same
// statement (the registers are valid when it returns)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// numerics
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * __expf(-0.5f * x * x) * 0.39894228040143268f;
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// x = hi + mid + lo (each BF16), exact differences in FP32
__device__ __forceinline__ void split3(float x, uint16_t& h, uint16_t& m, uint16_t& l) {
  h = bf16_bits(x);
  const float r1 = x - bf16_val(h);
  m = bf16_bits(r1);
  const float r2 = r1 - bf16_val(m);
  l = bf16_bits(r2);
}
__device__ __forceinline__ void split2(float x, uint16_t& h, uint16_t& l) {
  h = bf16_bits(x);
  l = bf16_bits(x - bf16_val(h));
}

// stores 8 consecutive K elements (one core-matrix row) of row r
__device__ __forceinline__ void st_row8(unsigned char* img, int r, int k0, int KC, const uint16_t (&v)[8]) {
  uint4 q;
  q.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
  q.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
  q.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
  q.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
  *reinterpret_cast<uint4*>(img + canon(r, k0, KC)) = q;
}

// FP32 plane geometry of the fallback test ----------------------------------
// volume below the plane m.x <= a in the unit cube (any signs of m)
__device__ __forceinline__ float volume_f(float m0, float m1, float m2, float a) {
  if (m0 < 0.f) { a -= m0; m0 = -m0; }
  if (m1 < 0.f) { a -= m1; m1 = -m1; }
  if (m2 < 0.f) { a -= m2; m2 = -m2; }
  const float l1 = m0 + m1 + m2;
  if (!(l1 > 0.f)) return a >= 0.f ? 1.f : 0.f;
  const float r = 1.f / l1;
  m0 *= r; m1 *= r; m2 *= r; a *= r;
  if (a <= 0.f) return 0.f;
  if (a >= 1.f) return 1.f;
  float t;
  if (m1 < m0) { t = m0; m0 = m1; m1 = t; }
  if (m2 < m1) { t = m1; m1 = m2; m2 = t; }
  if (m1 < m0) { t = m0; m0 = m1; m1 = t; }
  return a <= 0.5f ? vol_low_f(m0, m1, m2, a) : 1.f - vol_low_f(m0, m1, m2, 1.f - a);
}

// plane constant with volume_f(m, a) = c (m L1-normalised)
__device__ __forceinline__ float alpha_f(float m0, float m1, float m2, float c) {
  float sh = 0.f;
  if (m0 < 0.f) { sh -= m0; m0 = -m0; }
  if (m1 < 0.f) { sh -= m1; m1 = -m1; }
  if (m2 < 0.f) { sh -= m2; m2 = -m2; }
  float t;
  if (m1 < m0) { t = m0; m0 = m1; m1 = t; }
  if (m2 < m1) { t = m1; m1 = m2; m2 = t; }
  if (m1 < m0) { t = m0; m0 = m1; m1 = t; }
  if (c <= 0.f) return -sh;
  if (c >= 1.f) return 1.f - sh;
  const float a = c <= 0.5f ? alpha_guess_f(m0, m1, m2, c) : 1.f - alpha_guess_f(m0, m1, m2, 1.f - c);
  return a - sh;
}

// RMS over the 26 neighbours of (volume of the plane with normal m through
// the central cell's plane constant) - c; s: the stencil (x fastest)
__device__ __forceinline__ float plane_residual(const float* s, float m0, float m1, float m2) {
  const float l1 = fabsf(m0) + fabsf(m1) + fabsf(m2);
  const float r = 1.f / l1;
  m0 *= r; m1 *= r; m2 *= r;
  const float al = alpha_f(m0, m1, m2, s[13]);
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    if (k == 13) continue;
    const float ox = (float)(k % 3 - 1), oy = (float)((k / 3) % 3 - 1), oz = (float)(k / 9 - 1);
    const float d = volume_f(m0, m1, m2, al - (m0 * ox + m1 * oy + m2 * oz)) - s[k];
    acc += d * d;
  }
  return sqrtf(acc * (1.f / 26.f));
}

// ---------------------------------------------------------------------------
// Sources of stencils
// ---------------------------------------------------------------------------
// explicit stencils X[n][27] (x fastest within a stencil)
struct SrcX {
  const double* X;
  __device__ __forceinline__ double at(long i, int k) const { return __ldg(X + 27 * i + k); }
};
// the mixed-cell list of a sweep: stencil of cell gmix[i] with the boundary
// conditions' index mapping
struct SrcGrid {
  GridDev g;
  const double* c;
  const uint32_t* gmix;
  __device__ __forceinline__ double at(long i, int k) const {
    const size_t id = gmix[i];
    int x, y, z;
    cell_xyz(g, id, x, y, z);
    const int xx = map_idx(x + k % 3 - 1, g.n[0], g.bc[0]);
    const int yy = map_idx(y + (k / 3) % 3 - 1, g.n[1], g.bc[1]);
    const int zz = map_idx(z + k / 9 - 1, g.n[2], g.bc[2]);
    return __ldg(c + ((size_t)zz * g.n[1] + yy) * g.n[0] + xx);
  }
};

// ---------------------------------------------------------------------------
// Shared memory of the inference kernel
// ---------------------------------------------------------------------------
struct InferSmem {
  alignas(1024) unsigned char act[3][kRows * kH * 2];  // activation pieces (A operands)
  alignas(1024) unsigned char w[kInferWBytes];         // W1, W2, W3 images
  float bias[kH + kH + kN3];
  uint64_t bar;
  uint32_t tmem;
  int abort;
};

constexpr uint32_t kInferCols = 128;  // tensor-memory columns per CTA

// Issues the MMAs of one layer: D = sum over pieces p < np and K steps of
// A_p[128 x K] . B[N x K]^T.
__device__ __forceinline__ void issue_layer(uint32_t d, const unsigned char* a0, uint32_t a_piece_bytes, int np,
                                            const unsigned char* b, int K, int N) {
  const int KC = K / 8;
  const uint32_t sbo = (uint32_t)KC * 128u;
  const uint32_t id = idesc_bf16(kRows, N);
  uint32_t acc = 0;
  for (int p = 0; p < np; ++p)
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t ad = sdesc(su32(a0) + p * a_piece_bytes + ks * 256u, 128u, sbo);
      const uint64_t bd = sdesc(su32(b) + ks * 256u, 128u, sbo);
      umma(d, ad, bd, id, acc);
      acc = 1;
    }
}

// Writes this row's activations (FP32 values v of K columns starting at k0)
// as three BF16 pieces.
__device__ __forceinline__ void put_act3(InferSmem& S, int r, int k0, int KC, const float* v) {
  uint16_t h[8], m[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) split3(v[i], h[i], m[i], l[i]);
  st_row8(S.act[0], r, k0, KC, h);
  st_row8(S.act[1], r, k0, KC, m);
  st_row8(S.act[2], r, k0, KC, l);
}

// All threads: wait for the layer's MMAs (phase `ph`); false if the wait
// gave up anywhere in the CTA.
__device__ __forceinline__ bool layer_done(InferSmem& S, uint32_t& ph) {
  const bool ok = mbar_wait(&S.bar, ph);
  ph ^= 1u;
  const int all = __syncthreads_and(ok ? 1 : 0);
  tc_after_sync();
  return all != 0;
}

// MODE 0: network output y[n][3] (FP32) for explicit stencils.
// MODE 1: learned normal with MYC fallback for explicit stencils:
//         m[n][3] (L1-normalised, FP64) and flag[n] (1: MYC used).
// MODE 2: the same normal for the mixed cells of a sweep, into the planes
//         of the sweep scratch (m0, m1, m2; the plane constant follows).
template <int MODE, class Src>
__global__ void __launch_bounds__(kThreads)
k_mlp_infer(Src src, const int* __restrict__ count_dev, long n_host, const unsigned char* __restrict__ params,
            float* __restrict__ y_out, double* __restrict__ m_out, uint8_t* __restrict__ flag_out,
            double* __restrict__ plane_out, int* __restrict__ nfallback, int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, warp = t >> 5;
  const long n = count_dev ? (long)*count_dev : n_host;
  const long ntiles = (n + kRows - 1) / kRows;
  if ((long)blockIdx.x >= ntiles) return;  // uniform across the CTA

  // weights and biases (the images are already in the canonical layout)
  for (uint32_t o = t * 16; o < kInferWBytes; o += kThreads * 16)
    *reinterpret_cast<uint4*>(S.w + o) = __ldg(reinterpret_cast<const uint4*>(params + o));
  for (int i = t; i < kH + kH + kN3; i += kThreads) S.bias[i] = __ldg(reinterpret_cast<const float*>(params + pB) + i);
  if (t == 0) {
    mbar_init(&S.bar, 1);
    S.abort = 0;
  }
  if (warp == 0) tmem_alloc(&S.tmem, kInferCols);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tm = S.tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;  // this warp's tensor-memory lanes
  uint32_t ph = 0;
  bool ok = true;

  for (long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long i = tile * kRows + t;
    const bool live = i < n;
    // layer 1 input: 2 c - 1 (K padded to 32 with zeros)
    {
      float v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = (live && k < kIn) ? (float)(2.0 * src.at(i, k) - 1.0) : 0.f;
#pragma unroll
      for (int k0 = 0; k0 < 32; k0 += 8) put_act3(S, t, k0, 4, v + k0);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    if (t == 0) {
      tc_after_sync();
      issue_layer(tm + 0, S.act[0], kRows * kH * 2, 3, S.w + pW1, kK1, kH);
      umma_commit(&S.bar);
    }
    if (!(ok = layer_done(S, ph))) break;
    // layer 1 -> 2: z1 = D + b1, GELU, three pieces
#pragma unroll
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float v[16];
      tmem_ld16(tm + lane_base + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = gelu(v[j] + S.bias[c0 + j]);
      put_act3(S, t, c0, 8, v);
      put_act3(S, t, c0 + 8, 8, v + 8);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    if (t == 0) {
      tc_after_sync();
      issue_layer(tm + 64, S.act[0], kRows * kH * 2, 3, S.w + pW2, kH, kH);
      umma_commit(&S.bar);
    }
    if (!(ok = layer_done(S, ph))) break;
#pragma unroll
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float v[16];
      tmem_ld16(tm + lane_base + 64 + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = gelu(v[j] + S.bias[kH + c0 + j]);
      put_act3(S, t, c0, 8, v);
      put_act3(S, t, c0 + 8, 8, v + 8);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    if (t == 0) {
      tc_after_sync();
      issue_layer(tm + 0, S.act[0], kRows * kH * 2, 3, S.w + pW3, kH, kN3);
      umma_commit(&S.bar);
    }
    if (!(ok = layer_done(S, ph))) break;
    float y[16];
    tmem_ld16(tm + lane_base + 0, y);
    const float y0 = y[0] + S.bias[2 * kH + 0], y1 = y[1] + S.bias[2 * kH + 1], y2 = y[2] + S.bias[2 * kH + 2];
    if (live) {
      if constexpr (MODE == 0) {
        y_out[3 * i + 0] = y0;
        y_out[3 * i + 1] = y1;
        y_out[3 * i + 2] = y2;
      } else {
        double sd[27];
        float sf[27];
#pragma unroll
        for (int k = 0; k < 27; ++k) {
          sd[k] = src.at(i, k);
          sf[k] = (float)sd[k];
        }
        // the fallback: MYC as the sweeps of this precision compute it
        // (explicit stencils: the precision form's)
        double mm[3];
        if constexpr (MODE == 2) {
          if (src.g.f32) myc_normal_f(sd, mm);
          else myc_normal(sd, mm);
        } else {
          myc_normal_f(sd, mm);
        }
        const float rm = plane_residual(sf, (float)mm[0], (float)mm[1], (float)mm[2]);
        const float l1 = fabsf(y0) + fabsf(y1) + fabsf(y2);
        const float rn = plane_residual(sf, y0, y1, y2);
        // keep the network's normal only when its residual is a number
        // within the bound (a zero or non-finite output falls back)
        const bool use_mlp = l1 > 0.f && rn <= kFallbackRatio * rm + kFallbackTol;
        double m0 = mm[0], m1 = mm[1], m2 = mm[2];
        if (use_mlp) {
          const double dl1 = (double)fabsf(y0) + (double)fabsf(y1) + (double)fabsf(y2);
          m0 = (double)y0 / dl1;
          m1 = (double)y1 / dl1;
          m2 = (double)y2 / dl1;
        } else if (nfallback) {
          atomicAdd(nfallback, 1);
        }
        if constexpr (MODE == 1) {
          m_out[3 * i + 0] = m0;
          m_out[3 * i + 1] = m1;
          m_out[3 * i + 2] = m2;
          if (flag_out) flag_out[i] = use_mlp ? 0 : 1;
        } else {
          const size_t id = src.gmix[i];
          double* pl = plane_out + 4 * id;
          pl[0] = m0;
          pl[1] = m1;
          pl[2] = m2;
        }
      }
    }
    // the next tile's layer-1 MMAs overwrite columns 0..63 read above
    tc_before_sync();
    __syncthreads();
  }
  if (!ok && t == 0 && status) atomicOr(status, DEV_WAIT);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0) tmem_dealloc(tm, kInferCols);
}

// ---------------------------------------------------------------------------
// Packing: FP32 master parameters -> BF16 images (+ FP32 copies)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pack_one(const float* __restrict__ master, unsigned char* __restrict__ P, int q) {
  const float v = master[q];
  const uint16_t b = bf16_bits(v);
  if (q < oB1) {
    const int j = q / kIn, k = q % kIn;
    *reinterpret_cast<uint16_t*>(P + pW1 + canon(j, k, 4)) = b;
  } else if (q < oW2) {
    reinterpret_cast<float*>(P + pB)[q - oB1] = v;
  } else if (q < oB2) {
    const int j = (q - oW2) / kH, k = (q - oW2) % kH;
    *reinterpret_cast<uint16_t*>(P + pW2 + canon(j, k, 8)) = b;
    *reinterpret_cast<uint16_t*>(P + pW2T + canon(k, j, 8)) = b;
  } else if (q < oW3) {
    reinterpret_cast<float*>(P + pB)[kH + q - oB2] = v;
  } else if (q < oB3) {
    const int i = (q - oW3) / kH, j = (q - oW3) % kH;
    *reinterpret_cast<uint16_t*>(P + pW3 + canon(i, j, 8)) = b;
    reinterpret_cast<float*>(P + pW3F)[q - oW3] = bf16_val(b);
  } else {
    reinterpret_cast<float*>(P + pB)[2 * kH + q - oB3] = v;
  }
}

// zero the padding (whole buffer) and write every parameter
__global__ void k_mlp_zero(unsigned char* __restrict__ P) {
  for (uint32_t o = (blockIdx.x * blockDim.x + threadIdx.x) * 4; o < kPackedBytes; o += gridDim.x * blockDim.x * 4)
    *reinterpret_cast<uint32_t*>(P + o) = 0u;
}
__global__ void k_mlp_pack(const float* __restrict__ master, unsigned char* __restrict__ P) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kParams; q += gridDim.x * blockDim.x) pack_one(master, P, q);
}

// ---------------------------------------------------------------------------
// Training: forward and backward of one tile of 128 samples per CTA, the
// tile's gradient written to its own row of partial sums (reduced in tile
// order by the Adam kernel: deterministic).
// ---------------------------------------------------------------------------
constexpr int kZs = kH + 1;  // row stride of the FP32 pre-activations (no bank conflicts)
constexpr int kTB = 96;      // rows of the transposed B operand: a1 (64) then a0 (32)
constexpr uint32_t kTrainCols = 256;

struct TrainSmem {
  alignas(1024) unsigned char act[3][kRows * kH * 2];  // A pieces; later [a1; a0]^T pieces (2 x 24 KB)
  alignas(1024) unsigned char at[2][kRows * kRows * 2];  // [g_z2; g_z1]^T pieces (rows: unit, K: sample)
  alignas(1024) unsigned char w[kPackedBytes];
  float z1[kRows * kZs];
  float z2[kRows * kZs];
  float red[4][kOut * kH + kOut + 1];  // per-warp dW3, db3, loss
  uint64_t bar;
  uint32_t tmem;
};

// splitmix64: the sample index of (seed, step, slot)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool train_wait(TrainSmem& S, uint32_t& ph) {
  const bool ok = mbar_wait(&S.bar, ph);
  ph ^= 1u;
  const int all = __syncthreads_and(ok ? 1 : 0);
  tc_after_sync();
  return all != 0;
}

__device__ __forceinline__ void put3(unsigned char* const* pieces, uint32_t piece_bytes, int r, int k0, int KC,
                                     const float* v) {
  uint16_t h[8], m[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) split3(v[i], h[i], m[i], l[i]);
  st_row8(pieces[0], r, k0, KC, h);
  st_row8(pieces[0] + piece_bytes, r, k0, KC, m);
  st_row8(pieces[0] + 2 * piece_bytes, r, k0, KC, l);
}

// element (row, k = sample) of a transposed two-piece operand
__device__ __forceinline__ void put2_t(unsigned char* img, uint32_t piece_bytes, int row, int s, int KC, float v) {
  uint16_t h, l;
  split2(v, h, l);
  *reinterpret_cast<uint16_t*>(img + canon(row, s, KC)) = h;
  *reinterpret_cast<uint16_t*>(img + piece_bytes + canon(row, s, KC)) = l;
}

// X[ntrain][27] stencils, N[ntrain][3] unit normals; batch = gridDim.x * 128
// samples drawn with replacement by splitmix64(seed, step, slot).
// partial[tile][kParams] gradients of the batch-mean loss, loss_part[tile].
__global__ void __launch_bounds__(kThreads, 1)
k_mlp_train(const double* __restrict__ X, const double* __restrict__ N, long ntrain, unsigned long long seed,
            long step, const unsigned char* __restrict__ params, float* __restrict__ partial,
            float* __restrict__ loss_part, const long* __restrict__ idx_fixed, int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int B = gridDim.x * kRows;
  const float invB = 1.0f / (float)B;
  for (uint32_t o = t * 16; o < kPackedBytes; o += kThreads * 16)
    *reinterpret_cast<uint4*>(S.w + o) = __ldg(reinterpret_cast<const uint4*>(params + o));
  if (t == 0) mbar_init(&S.bar, 1);
  if (warp == 0) tmem_alloc(&S.tmem, kTrainCols);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tm = S.tmem;
  const uint32_t lb = (uint32_t)(warp * 32) << 16;
  const float* bias = reinterpret_cast<const float*>(S.w + pB);
  const float* w3f = reinterpret_cast<const float*>(S.w + pW3F);
  uint32_t ph = 0;
  bool ok = true;
  unsigned char* act[1] = {S.act[0]};
  constexpr uint32_t kActPiece = kRows * kH * 2;
  constexpr uint32_t kAtPiece = kRows * kRows * 2;
  constexpr uint32_t kBtPiece = kTB * kRows * 2;

  // sample
  const long slot = (long)blockIdx.x * kRows + t;
  const long si = idx_fixed ? idx_fixed[slot]
                            : (long)(mix64(seed ^ mix64((uint64_t)step * 0x100000001B3ull + (uint64_t)slot)) %
                                     (uint64_t)ntrain);
  float x[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) x[k] = k < kIn ? (float)(2.0 * __ldg(X + 27 * si + k) - 1.0) : (k == kIn ? 1.f : 0.f);
  // the feature after the 27 inputs is a constant 1 with zero weight: it
  // carries the bias gradients through the weight-gradient contraction
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += 8) put3(act, kActPiece, t, k0, 4, x + k0);
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  if (t == 0) {
    tc_after_sync();
    issue_layer(tm + 0, S.act[0], kActPiece, 3, S.w + pW1, kK1, kH);
    umma_commit(&S.bar);
  }
  if (!(ok = train_wait(S, ph))) goto done;
#pragma unroll
  for (int c0 = 0; c0 < kH; c0 += 16) {
    float v[16];
    tmem_ld16(tm + lb + c0, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float z = v[j] + bias[c0 + j];
      S.z1[t * kZs + c0 + j] = z;
      v[j] = gelu(z);
    }
    put3(act, kActPiece, t, c0, 8, v);
    put3(act, kActPiece, t, c0 + 8, 8, v + 8);
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  if (t == 0) {
    tc_after_sync();
    issue_layer(tm + 64, S.act[0], kActPiece, 3, S.w + pW2, kH, kH);
    umma_commit(&S.bar);
  }
  if (!(ok = train_wait(S, ph))) goto done;
#pragma unroll
  for (int c0 = 0; c0 < kH; c0 += 16) {
    float v[16];
    tmem_ld16(tm + lb + 64 + c0, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float z = v[j] + bias[kH + c0 + j];
      S.z2[t * kZs + c0 + j] = z;
      v[j] = gelu(z);
    }
    put3(act, kActPiece, t, c0, 8, v);
    put3(act, kActPiece, t, c0 + 8, 8, v + 8);
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  if (t == 0) {
    tc_after_sync();
    issue_layer(tm + 0, S.act[0], kActPiece, 3, S.w + pW3, kH, kN3);
    umma_commit(&S.bar);
  }
  if (!(ok = train_wait(S, ph))) goto done;
  {
    // loss and its gradient at the output: yh = y / |y|_2, loss = |yh - n|^2
    float yv[16];
    tmem_ld16(tm + lb + 0, yv);
    float y[3], nn[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      y[q] = yv[q] + bias[2 * kH + q];
      nn[q] = (float)__ldg(N + 3 * si + q);
    }
    const float ny = sqrtf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    float yh[3], gyh[3], gy[3];
    float loss = 0.f, dotp = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      yh[q] = y[q] / ny;
      const float d = yh[q] - nn[q];
      loss += d * d;
      gyh[q] = 2.f * d * invB;
      dotp += gyh[q] * yh[q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) gy[q] = (gyh[q] - yh[q] * dotp) / ny;
    // g_z2 = (g_y W3) * gelu'(z2): the A operand of g_a1 (three pieces, rows
    // = samples) and rows 0..63 of the transposed A of the weight gradients;
    // dW3, db3 and the loss by warp sums
#pragma unroll
    for (int c0 = 0; c0 < kH; c0 += 8) {
      float g8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = c0 + j;
        const float z = S.z2[t * kZs + k];
        const float ga = gy[0] * w3f[k] + gy[1] * w3f[kH + k] + gy[2] * w3f[2 * kH + k];
        g8[j] = ga * gelu_grad(z);
        put2_t(S.at[0], kAtPiece, k, t, 16, g8[j]);
        const float a2 = gelu(z);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float pr = gy[q] * a2;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) pr += __shfl_xor_sync(0xffffffffu, pr, o);
          if (lane == 0) S.red[warp][q * kH + k] = pr;
        }
      }
      put3(act, kActPiece, t, c0, 8, g8);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float pr = gy[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) pr += __shfl_xor_sync(0xffffffffu, pr, o);
      if (lane == 0) S.red[warp][kOut * kH + q] = pr;
    }
    float ls = loss;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
    if (lane == 0) S.red[warp][kOut * kH + kOut] = ls;
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  if (t == 0) {
    // g_a1 = g_z2 . W2 (B operand: W2 transposed, rows = a1 unit)
    tc_after_sync();
    issue_layer(tm + 0, S.act[0], kActPiece, 3, S.w + pW2T, kH, kH);
    umma_commit(&S.bar);
  }
  if (!(ok = train_wait(S, ph))) goto done;
  {
    // g_z1 = g_a1 * gelu'(z1): rows 64..127 of the transposed A; the
    // transposed B holds a1 (rows 0..63) and the inputs with the constant
    // feature (rows 64..95), two pieces each, in the activation buffer
    // (free now: the MMAs that read it are complete)
    unsigned char* bt = S.act[0];
#pragma unroll
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float v[16];
      tmem_ld16(tm + lb + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int k = c0 + j;
        const float z = S.z1[t * kZs + k];
        put2_t(S.at[0], kAtPiece, kH + k, t, 16, v[j] * gelu_grad(z));
        put2_t(bt, kBtPiece, k, t, 16, gelu(z));
      }
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) put2_t(bt, kBtPiece, kH + k, t, 16, x[k]);
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  if (t == 0) {
    // [dW2 | db2 ; . | dW1 db1] = [g_z2 ; g_z1]^T . [a1 , a0]: products of
    // the pieces hi.hi + hi.lo + lo.hi, K = 128 samples
    tc_after_sync();
    const uint32_t id = idesc_bf16(kRows, kTB);
    uint32_t acc = 0;
    const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
    for (int q = 0; q < 3; ++q)
      for (int ks = 0; ks < kRows / 16; ++ks) {
        const uint64_t ad = sdesc(su32(S.at[0]) + pa[q] * kAtPiece + ks * 256u, 128u, 16u * 128u);
        const uint64_t bd = sdesc(su32(S.act[0]) + pb[q] * kBtPiece + ks * 256u, 128u, 16u * 128u);
        umma(tm + 64, ad, bd, id, acc);
        acc = 1;
      }
    umma_commit(&S.bar);
  }
  if (!(ok = train_wait(S, ph))) goto done;
  {
    float* prow = partial + (size_t)blockIdx.x * kParams;
    // row t of the accumulator: t < 64 is unit t of layer 2, else unit
    // t - 64 of layer 1
#pragma unroll
    for (int c0 = 0; c0 < kTB; c0 += 16) {
      float v[16];
      tmem_ld16(tm + lb + 64 + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c0 + j;
        if (t < kH) {
          if (col < kH) prow[oW2 + t * kH + col] = v[j];
          else if (col == kH + kIn) prow[oB2 + t] = v[j];
        } else {
          if (col >= kH && col < kH + kIn) prow[oW1 + (t - kH) * kIn + (col - kH)] = v[j];
          else if (col == kH + kIn) prow[oB1 + (t - kH)] = v[j];
        }
      }
    }
    // dW3, db3, loss: the four warps' sums in order
    for (int q = t; q < kOut * kH + kOut + 1; q += kThreads) {
      const float v = ((S.red[0][q] + S.red[1][q]) + S.red[2][q]) + S.red[3][q];
      if (q < kOut * kH) prow[oW3 + q] = v;
      else if (q < kOut * kH + kOut) prow[oB3 + q - kOut * kH] = v;
      else loss_part[blockIdx.x] = v * invB;
    }
  }
done:
  if (!ok && t == 0 && status) atomicOr(status, DEV_WAIT);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0) tmem_dealloc(tm, kTrainCols);
}

// Adam on the FP32 master parameters from the tiles' partial gradients
// (summed in tile order), then the packed BF16 images of the new values;
// loss_out (nullable) = the batch-mean loss.
__global__ void k_mlp_adam(float* __restrict__ master, float* __restrict__ mom, float* __restrict__ vel,
                           const float* __restrict__ partial, const float* __restrict__ loss_part, int ntiles,
                           long step, float lr, float beta1, float beta2, float eps, unsigned char* __restrict__ P,
                           float* __restrict__ grad_out, float* __restrict__ loss_out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0 && loss_out) {
    float l = 0.f;
    for (int b = 0; b < ntiles; ++b) l += loss_part[b];
    *loss_out = l;
  }
  if (q >= kParams) return;
  float g = 0.f;
  for (int b = 0; b < ntiles; ++b) g += partial[(size_t)b * kParams + q];
  if (grad_out) grad_out[q] = g;
  if (!(lr > 0.f)) return;  // gradient only
  const float m = beta1 * mom[q] + (1.f - beta1) * g;
  const float v = beta2 * vel[q] + (1.f - beta2) * g * g;
  mom[q] = m;
  vel[q] = v;
  const float mh = m / (1.f - powf(beta1, (float)step));
  const float vh = v / (1.f - powf(beta2, (float)step));
  master[q] = master[q] - lr * mh / (sqrtf(vh) + eps);
  pack_one(master, P, q);
}

}  // namespace mlp

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t mlp_packed_bytes() { return mlp::kPackedBytes; }
int mlp_param_count() { return mlp::kParams; }

static size_t infer_smem() { return sizeof(mlp::InferSmem) + 1024; }
static size_t train_smem() { return sizeof(mlp::TrainSmem) + 1024; }

template <int MODE, class Src>
static cudaError_t launch_infer_t(const Src& src, const int* count_dev, long n_host, long max_n,
                                  const void* params, float* y, double* m, uint8_t* flag, double* plane,
                                  int* nfallback, cudaStream_t st) {
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(mlp::k_mlp_infer<MODE, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)infer_smem());
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const long tiles = (max_n + mlp::kRows - 1) / mlp::kRows;
  long grid = tiles < 152 * 3 ? tiles : 152 * 3;
  if (grid < 1) grid = 1;
  mlp::k_mlp_infer<MODE, Src><<<(unsigned)grid, mlp::kThreads, infer_smem(), st>>>(
      src, count_dev, n_host, static_cast<const unsigned char*>(params), y, m, flag, plane, nfallback,
      device_status_ptr());
  prof_mark(MODE == 2 ? "mlp.normals" : "mlp.infer", st);
  return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float* master, void* packed, cudaStream_t st) {
  mlp::k_mlp_zero<<<8, 256, 0, st>>>(static_cast<unsigned char*>(packed));
  mlp::k_mlp_pack<<<(mlp::kParams + 255) / 256, 256, 0, st>>>(master, static_cast<unsigned char*>(packed));
  prof_mark("mlp.pack", st);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* params, const double* X, long n, float* y, cudaStream_t st) {
  return launch_infer_t<0>(mlp::SrcX{X}, nullptr, n, n, params, y, nullptr, nullptr, nullptr, nullptr, st);
}

cudaError_t launch_mlp_normals(const void* params, const double* X, long n, double* m, uint8_t* flag,
                               int* nfallback, cudaStream_t st) {
  return launch_infer_t<1>(mlp::SrcX{X}, nullptr, n, n, params, nullptr, m, flag, nullptr, nfallback, st);
}

cudaError_t launch_mlp_sweep_normals(const GridDev& g, const double* c, const SweepScratch& sc, cudaStream_t st) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  mlp::SrcGrid src{g, c, sc.gmix};
  // the mixed-cell count (counters[0]) is read on the device; fallbacks are
  // counted in counters[3]
  return launch_infer_t<2>(src, sc.counters, 0, (long)N, g.mlp_params, nullptr, nullptr, nullptr, sc.plane,
                           sc.counters + 3, st);
}

cudaError_t launch_mlp_train_step(const double* X, const double* N, long ntrain, int batch, unsigned long long seed,
                                  long step, float* master, float* mom, float* vel, void* packed, float* partial,
                                  float* loss_part, const long* idx_fixed, float lr, float beta1, float beta2,
                                  float eps, float* grad_out, float* loss_out, cudaStream_t st) {
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(mlp::k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)train_smem());
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const int tiles = batch / mlp::kRows;
  mlp::k_mlp_train<<<tiles, mlp::kThreads, train_smem(), st>>>(X, N, ntrain, seed, step,
                                                              static_cast<const unsigned char*>(packed), partial,
                                                              loss_part, idx_fixed, device_status_ptr());
  prof_mark("mlp.train", st);
  mlp::k_mlp_adam<<<(mlp::kParams + 255) / 256, 256, 0, st>>>(master, mom, vel, partial, loss_part, tiles, step, lr,
                                                               beta1, beta2, eps,
                                                               static_cast<unsigned char*>(packed), grad_out,
                                                               loss_out);
  prof_mark("mlp.adam", st);
  return cudaGetLastError();
}

}  // namespace vofgb

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace vofgb;

namespace {
vof_status mlp_status(cudaError_t e) {
  if (e == cudaSuccess) return VOF_OK;
  set_last_cuda_error((int)e);
  return VOF_ECUDA;
}
bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }
}  // namespace

extern "C" {

size_t vof_mlp_packed_bytes(void) { return mlp_packed_bytes(); }

vof_status vof_mlp_pack(const float* master, void* packed, void* stream) {
  if (!master || !packed || !aligned16(packed)) return VOF_EINVAL;
  return mlp_status(launch_mlp_pack(master, packed, (cudaStream_t)stream));
}

vof_status vof_mlp_forward(const void* packed, const double* X, long n, float* y, void* stream) {
  if (!packed || !aligned16(packed) || n < 0 || (n > 0 && (!X || !y))) return VOF_EINVAL;
  if (n == 0) return VOF_OK;
  return mlp_status(launch_mlp_forward(packed, X, n, y, (cudaStream_t)stream));
}

vof_status vof_mlp_normals(const void* packed, const double* X, long n, double* m, uint8_t* fallback, void* stream) {
  if (!packed || !aligned16(packed) || n < 0 || (n > 0 && (!X || !m))) return VOF_EINVAL;
  if (n == 0) return VOF_OK;
  return mlp_status(launch_mlp_normals(packed, X, n, m, fallback, nullptr, (cudaStream_t)stream));
}

size_t vof_mlp_train_workspace_bytes(int batch) {
  if (batch < 128 || batch > 65536 || batch % 128) return 0;
  const size_t tiles = (size_t)batch / 128;
  return ((tiles * (size_t)mlp_param_count() * 4 + 255) & ~(size_t)255) + ((tiles * 4 + 255) & ~(size_t)255);
}

vof_status vof_mlp_train_step(const double* X, const double* N, long ntrain, int batch, unsigned long long seed,
                              long step, float lr, float* master, float* adam_m, float* adam_v, void* packed,
                              float* grad, float* loss, const int64_t* idx, void* workspace, size_t workspace_bytes,
                              void* stream) {
  const size_t need = vof_mlp_train_workspace_bytes(batch);
  if (need == 0 || ntrain < 1 || !X || !N || !packed || !aligned16(packed) || !workspace) return VOF_EINVAL;
  if (((uintptr_t)workspace & 255) != 0 || workspace_bytes < need) return VOF_EINVAL;
  if (!(lr >= 0.f)) return VOF_EINVAL;
  if (lr > 0.f && (!master || !adam_m || !adam_v || step < 1)) return VOF_EINVAL;
  const size_t tiles = (size_t)batch / 128;
  float* partial = static_cast<float*>(workspace);
  float* loss_part = reinterpret_cast<float*>(static_cast<char*>(workspace) +
                                              ((tiles * (size_t)mlp_param_count() * 4 + 255) & ~(size_t)255));
  return mlp_status(launch_mlp_train_step(X, N, ntrain, batch, seed, step, master, adam_m, adam_v, packed, partial,
                                          loss_part, reinterpret_cast<const long*>(idx), lr, 0.9f, 0.999f, 1e-8f,
                                          grad, loss, (cudaStream_t)stream));
}

}  // extern "C"
