// sur_mlp.h -- device side of the learned surrogate network shared by the
// inference kernel (surrogate.cu) and the push with drag law SURROGATE
// (kernels.cu): constants of the network's layout and one forward pass of a
// CTA's 128 rows on the tensor cores.
//
// The MLP is 4 -> 64 -> 64 -> 64 -> 2 with SiLU.  Layers 2 and 3 run as
// tcgen05 MMAs (M = 128 rows, N = 64, K = 64; BF16 operands in shared memory
// in the swizzled K-major layout of tc05.h; FP32 accumulators in TMEM);
// layers 1 (K = 4) and 4 (N = 2) run on the FP32 pipes.  The tangent of the
// outputs in the first input (forward mode) rides along: its tile goes
// through the same weights into the TMEM columns 64..127.
#pragma once
#include <cuda_bf16.h>

#include "tc05.h"

namespace pic1d {
namespace sur {

constexpr int TM = 128;        // rows per tile = TMEM lanes = threads of a CTA
constexpr int NT = 128;
constexpr float LT = -30.0f;   // clamp of the rate targets (ln N^)
constexpr float LE = -20.0f;   // floor of the scored region
constexpr double B_MID = -1.25, B_HALF = 2.75;
constexpr uint32_t kTagSur = 0x53555247u;

// image of the tensor-core operands (BF16, swizzled K-major, 8 KB each)
constexpr int IMG_W2 = 0, IMG_W3 = 8192, IMG_W2T = 16384, IMG_W3T = 24576, IMG_BYTES = 32768;
// FP32 copies of layers 1 and 4 and the biases
constexpr int S_W1 = 0, S_B1 = 256, S_B2 = 320, S_B3 = 384, S_W4 = 448, S_B4 = 576, S_N = 580;

constexpr uint32_t IDESC_128x64 = tc::idesc_bf16(128, 64);

// shared memory of a forward-pass CTA (from a 1024-aligned base)
constexpr int MF_W = 0;            // W2, W3 images (16 KB)
constexpr int MF_A = 16384;        // value tile, 128 x 64 BF16
constexpr int MF_AD = 32768;       // tangent tile
constexpr int MF_SMALL = 49152;    // S_N floats
constexpr int MF_END = MF_SMALL + 4 * S_N;
constexpr int MF_SMEM = MF_END + 1024;   // dynamic size with the alignment slack

// the logistic s = 1 / (1 + e^-z) (0 for z below about -88), SiLU z s, and
// SiLU with its derivative s (1 + z (1 - s)) from the same s
__device__ __forceinline__ float sigmoid(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigmoid(z); }
__device__ __forceinline__ void silu_d(float z, float& h, float& dh) {
  const float s = sigmoid(z);
  h = z * s;
  dh = s * fmaf(z, 1.0f - s, 1.0f);
}

// store 8 FP32 values as BF16 into chunk c of row r of a swizzled tile
__device__ __forceinline__ void store_chunk(uint8_t* tile, int r, int c, const float* v) {
  __align__(16) __nv_bfloat162 p[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
  *reinterpret_cast<uint4*>(tile + r * 128 + (((c ^ r) & 7) << 4)) = *reinterpret_cast<uint4*>(p);
}

// element (row j, k = batch index t) of a transposed tile with K = 128 (two
// 64-wide swizzle atoms of `rows` rows each)
__device__ __forceinline__ void store_t(uint8_t* tile, int rows, int j, int t, float v) {
  uint8_t* atom = tile + (t >> 6) * rows * 128;
  *reinterpret_cast<__nv_bfloat16*>(atom + tc::sw128(j, t & 63)) = __float2bfloat16_rn(v);
}

// warp sum then one shared atomic per warp
__device__ __forceinline__ void red_add(float v, float* acc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, v);
}

// one MMA chain of K = 64 (4 slices): D = A(128 x 64) * B(64 x 64)^T
__device__ __forceinline__ void mma_k64(uint32_t d, const uint8_t* A, const uint8_t* B) {
  const uint32_t a = tc::smem_addr(A), b = tc::smem_addr(B);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
    tc::mma_bf16(d, tc::desc_sw128(a + 32 * kk), tc::desc_sw128(b + 32 * kk), IDESC_128x64, kk > 0);
}

// Set-up of a forward-pass CTA: barriers, weight images by bulk copy, TMEM
// (128 columns), the small layers.  All NT threads call it.
struct MlpCta {
  uint8_t* sm;
  unsigned passes;   // forward passes made by this CTA
  unsigned passes_t; // of which with the tangent
  uint64_t* bar_ld;
  uint64_t* bar_mma;
  uint64_t* bar_end;
  uint32_t tmem;
  uint32_t ph;
  bool ok;
};

// bar: three mbarriers in shared memory (weight copies, MMA completion, teardown).
__device__ __forceinline__ void mlp_begin(MlpCta& M, uint8_t* smem_raw, uint64_t* bar, uint32_t* s_taddr,
                                          const uint8_t* img, const float* small) {
  M.sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar_ld = bar;
  M.bar_ld = bar;
  M.bar_mma = bar + 1;
  M.bar_end = bar + 2;
  const int t = threadIdx.x;
  if (t == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_init(bar + 1, 1);
    tc::mbar_init(bar + 2, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (t == 0) {
    tc::mbar_expect_tx(bar_ld, 16384);
    tc::bulk_g2s(M.sm + MF_W, img + IMG_W2, 8192, bar_ld);
    tc::bulk_g2s(M.sm + MF_W + 8192, img + IMG_W3, 8192, bar_ld);
  }
  if (t < 32) tc::tmem_alloc(s_taddr, 128);
  float* sSmall = reinterpret_cast<float*>(M.sm + MF_SMALL);
  for (int k = t; k < S_N; k += NT) sSmall[k] = small[k];
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  M.tmem = *s_taddr;
  M.ph = 0;
  M.passes = 0;
  M.passes_t = 0;
  M.ok = tc::mbar_wait(bar_ld, 0);
}

// End of a forward-pass CTA (all NT threads): returns true only if no wait of
// any thread gave up; the TMEM columns are freed once nothing is in flight.
__device__ __forceinline__ bool mlp_end(MlpCta& M) {
  return tc::cta_teardown(M.ok, M.bar_end, M.bar_ld, 0, M.tmem, 128);
}

// One forward pass of the CTA's 128 rows (thread t holds row t's inputs x):
// outputs y0, y1 and, if `tangent` (the same for every thread of the CTA),
// their derivatives g0, g1 in x[0] (else zero).  All NT threads call it; a
// wait that gives up clears M.ok (the outputs are then meaningless).
__device__ __forceinline__ void mlp_tile(MlpCta& M, const float (&x)[4], float& y0, float& y1, float& g0,
                                         float& g1, bool tangent = true) {
  const int t = threadIdx.x, warp = t >> 5;
  uint8_t* sA = M.sm + MF_A;
  uint8_t* sAd = M.sm + MF_AD;
  const float* sSmall = reinterpret_cast<const float*>(M.sm + MF_SMALL);
  const uint32_t tl = M.tmem + ((uint32_t)(warp * 32) << 16);
  for (int c = 0; c < 8; ++c) {
    float hv[8], hd[8];
    if (tangent) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = 8 * c + e;
        float z = sSmall[S_B1 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) z = fmaf(sSmall[S_W1 + 4 * j + i], x[i], z);
        float dh;
        silu_d(z, hv[e], dh);
        hd[e] = dh * sSmall[S_W1 + 4 * j];
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = 8 * c + e;
        float z = sSmall[S_B1 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) z = fmaf(sSmall[S_W1 + 4 * j + i], x[i], z);
        hv[e] = silu(z);
        hd[e] = 0.0f;
      }
    }
    store_chunk(sA, t, c, hv);
    if (tangent) store_chunk(sAd, t, c, hd);
  }
  float a0 = sSmall[S_B4], a1 = sSmall[S_B4 + 1], d0 = 0.f, d1 = 0.f;
  for (int layer = 0; layer < 2; ++layer) {
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (t == 0) {
      tc::fence_after();
      mma_k64(M.tmem, sA, M.sm + MF_W + 8192 * layer);
      if (tangent) mma_k64(M.tmem + 64, sAd, M.sm + MF_W + 8192 * layer);
      tc::mma_commit(M.bar_mma);
    }
    M.ok = M.ok && tc::mbar_wait(M.bar_mma, M.ph);
    M.ph ^= 1;
    tc::fence_after();
    const float* bias = sSmall + (layer == 0 ? S_B2 : S_B3);
    for (int c = 0; c < 4; ++c) {
      float v[16], vd[16];
      tc::tmem_ld16(tl + 16 * c, v);
      if (tangent) tc::tmem_ld16(tl + 64 + 16 * c, vd);
      float hv[16], hd[16];
      if (tangent) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          float dh;
          silu_d(v[e] + bias[16 * c + e], hv[e], dh);
          hd[e] = dh * vd[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          hv[e] = silu(v[e] + bias[16 * c + e]);
          hd[e] = 0.0f;
        }
      }
      if (layer == 0) {
        store_chunk(sA, t, 2 * c, hv);
        store_chunk(sA, t, 2 * c + 1, hv + 8);
        if (tangent) {
          store_chunk(sAd, t, 2 * c, hd);
          store_chunk(sAd, t, 2 * c + 1, hd + 8);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int j = 16 * c + e;
          a0 = fmaf(sSmall[S_W4 + j], hv[e], a0);
          a1 = fmaf(sSmall[S_W4 + 64 + j], hv[e], a1);
          d0 = fmaf(sSmall[S_W4 + j], hd[e], d0);
          d1 = fmaf(sSmall[S_W4 + 64 + j], hd[e], d1);
        }
      }
    }
  }
  y0 = a0;
  y1 = a1;
  g0 = d0;
  g1 = d1;
  ++M.passes;
  if (tangent) ++M.passes_t;
  // the next pass's writes to the tiles and to TMEM come after this barrier
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}

}  // namespace sur
}  // namespace pic1d
