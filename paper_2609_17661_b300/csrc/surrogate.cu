// surrogate.cu -- the learned surrogate of the photon-field quadrature.
//
// A small MLP, 4 -> 64 -> 64 -> 64 -> 2 with SiLU, stands in for the
// quadrature of the resonant scattering over the stellar blackbody photon
// field (Sec. 2.2, Eq. scatteringNdot with the momentum given per
// scattering).  Per photon direction a scattering gives the lepton the
// momentum gamma b mu~ along s (mu~ the aberrated cosine of the direction),
// so the drag is F^ = gamma b N^ <mu~> with <mu~> the rate-weighted mean of
// mu~, which lies in [-1, 1].  The network's two outputs are
//   y0 ~ <mu~>
//   y1 ~ max(ln N^, LT) - max(B, LT)
// where B = ln(0.9 N^_rad(mu_s) + 0.1 N^_rad(mu_e)) is a closed-form
// baseline (the single-direction form [contdrag] along the local radial and
// along the disk edge most favourable to the resonance) and LT = -30 the
// clamp of the targets; the network is scored where ln N^ > LE = -20, below
// which a rate is negligible.  Inputs: f0 = 2 log10(gamma)/G - 1,
// f1 = 2 s/L - 1, f2 = (log10 b + 1.25)/2.75, f3 = sign(u).
// The tensor-core operands (W2, W3 and the activations h1, h2) are BF16;
// layers 1 and 4 (4 inputs, 2 outputs) and the biases stay FP32.
//
// Kernels:
//   k_sur_samples  training/validation samples by FP64 quadrature at
//                  Philox-drawn points (gamma, s, sign, r_eq).
//   k_sur_train    forward + backward of one 128-sample tile: layers 2 and
//                  3 and the matching backward products (dh = dz W and
//                  dW = dz^T h) on the tensor cores (tcgen05, BF16 operands
//                  in shared memory, FP32 accumulators in TMEM); layers 1
//                  and 4 (4 inputs, 2 outputs) on the FP32 pipes.
//   k_sur_update   sums the tiles' gradients in a fixed order, Adam (FP32
//                  master weights), and writes the BF16 images the other
//                  kernels copy into shared memory.
//   k_sur_infer    forward pass and its derivative in f0 (forward mode).
//   k_sur_val      drag and rate errors of the network against quadrature.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>

#include "pic1d_internal.h"
#include "sur_mlp.h"
#include "tc05.h"

namespace pic1d {
namespace sur {

// K = 128 (two atoms): D = A(128 x 128) * B(64 x 128)^T, A atoms 16 KB apart, B atoms 8 KB apart
__device__ __forceinline__ void mma_k128(uint32_t d, const uint8_t* A, const uint8_t* B) {
  const uint32_t a = tc::smem_addr(A), b = tc::smem_addr(B);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const uint32_t ao = (kk >> 2) * 16384 + 32 * (kk & 3), bo = (kk >> 2) * 8192 + 32 * (kk & 3);
    tc::mma_bf16(d, tc::desc_sw128(a + ao), tc::desc_sw128(b + bo), IDESC_128x64, kk > 0);
  }
}

// ------------------------------------------------------------ geometry (FP64)
__device__ __forceinline__ double arcA(double c) {
  return 0.5 * c * sqrt(1.0 + 3.0 * c * c) + asinh(sqrt(3.0) * c) / (2.0 * sqrt(3.0));
}

// theta at arc length fraction sf of the line r = r_eq sin^2(theta) (App. B.2):
// Newton on the closed-form arc length, kept inside a shrinking bracket
__device__ double theta_at(double r_eq, double sf) {
  const double th0 = asin(sqrt(1.0 / r_eq)), c0 = cos(th0);
  const double L = 2.0 * r_eq * arcA(c0);
  const double s = sf * L;
  double lo = th0, hi = 3.141592653589793 - th0;
  double th = th0 + (hi - lo) * sf;
  for (int it = 0; it < 60; ++it) {
    const double c = cos(th);
    const double f = r_eq * (arcA(c0) - arcA(c)) - s;
    if (f > 0) hi = th; else lo = th;
    const double d = r_eq * sin(th) * sqrt(1.0 + 3.0 * c * c);
    double nt = (d > 0) ? th - f / d : 0.5 * (lo + hi);
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    if (fabs(nt - th) < 1e-15) { th = nt; break; }
    th = nt;
  }
  return th;
}

__device__ __forceinline__ double omb_cos(double u, double gam, double m) {  // 1 - beta m without cancellation
  const double sm = (u >= 0.0) ? m : -m;
  return (1.0 - sm) + sm / (gam * (gam + fabs(u)));
}

// --------------------------------------------------------------- samples
__global__ void __launch_bounds__(128) k_sur_samples(SurPhys Q, unsigned long long seed, unsigned long long start,
                                                     long long n, double r_lo, double r_hi, float* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long index = start + (unsigned long long)i;
  // Philox4x32-10 (Salmon et al., SC'11), counter (index, 0, TAG), key = seed
  uint32_t c0 = (uint32_t)index, c1 = (uint32_t)(index >> 32), c2 = 0u, c3 = kTagSur;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  const double U0 = (double)(c0 >> 8) * (1.0 / 16777216.0), U1 = (double)(c1 >> 8) * (1.0 / 16777216.0);
  const double U3 = (double)(c3 >> 8) * (1.0 / 16777216.0);
  const double log10g = Q.log10g_max * U0, sf = U1;
  const bool neg = (c2 >> 31) != 0u;
  const double r_eq = (r_hi > r_lo) ? r_lo * pow(r_hi / r_lo, U3) : r_lo;

  const double th = theta_at(r_eq, sf);
  const double cth = cos(th), sth = sin(th);
  const double x = r_eq * sth * sth;
  const double root = sqrt(1.0 + 3.0 * cth * cth);
  double b = Q.b_star * root / (x * x * x);
  if (Q.b_convention == 1) b *= 0.5;
  const double mu = 2.0 * cth / root;

  double gam = pow(10.0, log10g);
  const double au = sqrt(fmax(0.0, gam * gam - 1.0));
  const double u = neg ? -au : au;
  gam = sqrt(1.0 + u * u);
  const double beta = u / gam;
  const double pi = 3.141592653589793;
  const double pref = Q.pref;   // r_e R* / (4 pi lbar^2)
  double N, F, Fa, mub;
  {
    // the single-direction closed form along mu_s (solid angle pi/x^2)
    const double D = omb_cos(u, gam, mu), eps = b / (gam * D);
    const double Nr = pref * pi / (x * x) * eps * eps / expm1(eps / Q.theta_T) / gam;
    if (Q.photon_model == PIC1D_PHOTON_RADIAL) {
      N = Nr;
      F = Nr * gam * b * (mu - beta) / D;
      Fa = fabs(F);
      mub = (mu - beta) / D;
    } else {
      const double cmax = (x > 1.0) ? sqrt(1.0 - 1.0 / (x * x)) : 0.0;
      const double smu = sqrt(fmax(0.0, 1.0 - mu * mu));
      const double wphi = 2.0 * pi / Q.n_phi;
      double sN = 0.0, sF = 0.0, sFa = 0.0;
      for (int a = 0; a < Q.n_mu; ++a) {
        const double ca = cmax + (1.0 - cmax) * 0.5 * (Q.gx[a] + 1.0);
        const double wa = (1.0 - cmax) * 0.5 * Q.gw[a];
        const double sa = sqrt(fmax(0.0, 1.0 - ca * ca));
        for (int j = 0; j < Q.n_phi; ++j) {
          const double mk = ca * mu + sa * cos(pi * (j + 0.5) / Q.n_phi) * smu;
          const double Dk = omb_cos(u, gam, mk), ek = b / (gam * Dk);
          const double dN = wa * wphi * ek * ek / expm1(ek / Q.theta_T);
          const double dNP = dN * gam * b * (mk - beta) / Dk;
          sN += dN;
          sF += dNP;
          sFa += fabs(dNP);
        }
      }
      N = pref / gam * sN;
      F = pref / gam * sF;
      Fa = pref / gam * sFa;
      mub = (sN > 0.0) ? sF / (gam * b * sN) : (mu - beta) / D;
    }
    // baseline: 0.9 of the radial form + 0.1 of the form along the disk edge
    // with the largest 1 - beta mu_k
    const double ths = acos(fmax(-1.0, fmin(1.0, mu))), am = asin(fmin(1.0, 1.0 / x));
    const double me = (u >= 0.0) ? cos(fmin(pi, ths + am)) : cos(fmax(0.0, ths - am));
    const double De = omb_cos(u, gam, me), ee = b / (gam * De);
    const double Ne = pref * pi / (x * x) * ee * ee / expm1(ee / Q.theta_T) / gam;
    const double Nb = 0.9 * Nr + 0.1 * Ne;
    const double base = (Nb > 0.0) ? log(Nb) : -745.0;
    const double lnN = (N > 0.0) ? log(N) : -745.0;
    float* o = out + 16 * i;
    o[0] = (float)(2.0 * log10g / Q.log10g_max - 1.0);
    o[1] = (float)(2.0 * sf - 1.0);
    o[2] = (float)((log10(b) - B_MID) / B_HALF);
    o[3] = neg ? -1.0f : 1.0f;
    o[4] = (float)mub;
    o[5] = (float)(fmax(lnN, (double)LT) - fmax(base, (double)LT));
    o[6] = (lnN > (double)LT) ? 1.0f : 0.0f;
    o[7] = (float)base;
    o[8] = (float)lnN;
    o[9] = (float)F;
    o[10] = (float)Fa;
    o[11] = (float)gam;
    o[12] = (float)b;
    o[13] = (float)u;
    o[14] = (float)x;
    o[15] = (float)mu;
  }
}

// ------------------------------------------------------------- training
struct TrainArgs {
  const float* samples;        // n x 16 records
  long long n;                 // records
  unsigned long long perm_a, perm_c;   // row i of the step -> record (a i + c) mod n
  long long row0;              // first row of this step
  int rows;                    // rows in this step (<= tiles * 128)
  float inv_batch;             // 1 / rows (mean loss)
  const uint8_t* img;          // BF16 operand images (IMG_BYTES)
  const float* small;          // S_N FP32 values
  float* part;                 // [tile][8770] gradient partials
  float* loss_part;            // [tile]
  unsigned* err;               // error flag (waits that gave up)
};

// dynamic shared memory map (bytes from a 1024-aligned base)
constexpr int SM_W = 0;                       // 4 images, 32 KB
constexpr int SM_A = 32768;                   // activation tile 128 x 64, 16 KB
constexpr int SM_AT = 49152;                  // dz^T, 128 (64 used) x 128, 32 KB
constexpr int SM_H1T = 81920;                 // h1^T, 64 x 128, 16 KB
constexpr int SM_H2T = 98304;                 // h2^T, 64 x 128, 16 KB
constexpr int SM_D1 = 114688;                 // SiLU'(z1), FP32 [64][128], 32 KB
constexpr int SM_D2 = 147456;                 // SiLU'(z2), 32 KB
constexpr int SM_SMALL = 180224;              // S_N floats
constexpr int SM_RED = SM_SMALL + 4 * S_N;    // 579 FP32 sums (dW1, db1, db2, db3, dW4, db4, loss)
constexpr int SM_END = SM_RED + 4 * 580;
constexpr int TRAIN_SMEM = SM_END + 1024;     // + alignment slack
constexpr int R_W1 = 0, R_B1 = 256, R_B2 = 320, R_B3 = 384, R_W4 = 448, R_B4 = 576, R_LOSS = 578;

__global__ void __launch_bounds__(NT, 1) k_sur_train(TrainArgs A) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_ld, bar_mma, bar_end;
  __shared__ uint32_t s_taddr;
  const int t = threadIdx.x, warp = t >> 5;
  float* sSmall = reinterpret_cast<float*>(sm + SM_SMALL);
  float* sRed = reinterpret_cast<float*>(sm + SM_RED);
  float* sD1 = reinterpret_cast<float*>(sm + SM_D1);
  float* sD2 = reinterpret_cast<float*>(sm + SM_D2);
  uint8_t* sA = sm + SM_A;
  uint8_t* sAT = sm + SM_AT;

  if (t == 0) {
    tc::mbar_init(&bar_ld, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_init(&bar_end, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (t == 0) {
    tc::mbar_expect_tx(&bar_ld, IMG_BYTES);
    for (int k = 0; k < 4; ++k) tc::bulk_g2s(sm + SM_W + 8192 * k, A.img + 8192 * k, 8192, &bar_ld);
  }
  if (warp == 0) tc::tmem_alloc(&s_taddr, 128);
  for (int k = t; k < S_N; k += NT) sSmall[k] = A.small[k];
  for (int k = t; k < 580; k += NT) sRed[k] = 0.0f;
  // rows 64..127 of the dz^T tile stay zero (M is padded from 64 to 128)
  for (int k = t; k < 2 * 64 * 128 / 16; k += NT) {
    const int atom = k / (64 * 8), rest = k % (64 * 8);
    *reinterpret_cast<uint4*>(sAT + atom * 16384 + 64 * 128 + rest * 16) = make_uint4(0, 0, 0, 0);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_taddr;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's lanes
  uint32_t ph = 0;
  bool ok = tc::mbar_wait(&bar_ld, 0);

  // ---- this thread's sample
  const long long row = (long long)blockIdx.x * TM + t;
  const bool valid = row < A.rows;
  float x[4] = {0.f, 0.f, 0.f, 0.f}, t1 = 0.f, t2 = 0.f, m = 0.f;
  if (valid) {
    const unsigned long long r = (unsigned long long)(A.row0 + row);
    const long long idx = (long long)((A.perm_a * r + A.perm_c) % (unsigned long long)A.n);
    const float4 p = *reinterpret_cast<const float4*>(A.samples + 16 * idx);
    const float4 q = *reinterpret_cast<const float4*>(A.samples + 16 * idx + 4);
    x[0] = p.x; x[1] = p.y; x[2] = p.z; x[3] = p.w;
    t1 = q.x; t2 = q.y; m = q.z;
  }

  // ---- layer 1 (FP32): h1 = SiLU(W1 x + b1)
  {
    float hv[8];
    for (int c = 0; c < 8; ++c) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = 8 * c + e;
        float z = sSmall[S_B1 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) z = fmaf(sSmall[S_W1 + 4 * j + i], x[i], z);
        float h, dh;
        silu_d(z, h, dh);
        hv[e] = valid ? h : 0.0f;
        sD1[j * TM + t] = dh;
        store_t(sm + SM_H1T, 64, j, t, hv[e]);
      }
      store_chunk(sA, t, c, hv);
    }
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  // ---- layer 2 on the tensor cores: D[cols 0..63] = h1 W2^T
  if (t == 0) {
    tc::fence_after();
    mma_k64(tmem, sA, sm + SM_W + IMG_W2);
    tc::mma_commit(&bar_mma);
  }
  ok = ok && tc::mbar_wait(&bar_mma, ph);
  ph ^= 1;
  tc::fence_after();
  for (int c = 0; c < 4; ++c) {
    float v[16];
    tc::tmem_ld16(tl + 16 * c, v);
    float hv[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int j = 16 * c + e;
      const float z = v[e] + sSmall[S_B2 + j];
      float h, dh;
      silu_d(z, h, dh);
      hv[e] = valid ? h : 0.0f;
      sD2[j * TM + t] = dh;
      store_t(sm + SM_H2T, 64, j, t, hv[e]);
    }
    store_chunk(sA, t, 2 * c, hv);
    store_chunk(sA, t, 2 * c + 1, hv + 8);
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  // ---- layer 3: D = h2 W3^T
  if (t == 0) {
    tc::fence_after();
    mma_k64(tmem, sA, sm + SM_W + IMG_W3);
    tc::mma_commit(&bar_mma);
  }
  ok = ok && tc::mbar_wait(&bar_mma, ph);
  ph ^= 1;
  tc::fence_after();
  float h3[64], d3[64];
  for (int c = 0; c < 4; ++c) {
    float v[16];
    tc::tmem_ld16(tl + 16 * c, v);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int j = 16 * c + e;
      const float z = v[e] + sSmall[S_B3 + j];
      float h;
      silu_d(z, h, d3[j]);
      h3[j] = valid ? h : 0.0f;
    }
  }
  // ---- layer 4 (FP32), loss and its gradient
  float y0 = sSmall[S_B4], y1 = sSmall[S_B4 + 1];
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    y0 = fmaf(sSmall[S_W4 + j], h3[j], y0);
    y1 = fmaf(sSmall[S_W4 + 64 + j], h3[j], y1);
  }
  const float r0 = valid ? (y0 - t1) * m : 0.0f, r1 = valid ? (y1 - t2) : 0.0f;
  red_add(r0 * (y0 - t1) + r1 * r1, &sRed[R_LOSS]);
  const float dy0 = 2.0f * r0 * A.inv_batch, dy1 = 2.0f * r1 * A.inv_batch;
  red_add(dy0, &sRed[R_B4]);
  red_add(dy1, &sRed[R_B4 + 1]);
  for (int j = 0; j < 64; ++j) {
    red_add(dy0 * h3[j], &sRed[R_W4 + j]);
    red_add(dy1 * h3[j], &sRed[R_W4 + 64 + j]);
  }
  // dz3 = (W4^T dy) * SiLU'(z3)
  for (int c = 0; c < 8; ++c) {
    float dz[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = 8 * c + e;
      dz[e] = (sSmall[S_W4 + j] * dy0 + sSmall[S_W4 + 64 + j] * dy1) * d3[j];
      red_add(dz[e], &sRed[R_B3 + j]);
      store_t(sAT, 128, j, t, dz[e]);
    }
    store_chunk(sA, t, c, dz);
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  // ---- dh2 = dz3 W3 (cols 0..63), dW3 = dz3^T h2 (cols 64..127)
  if (t == 0) {
    tc::fence_after();
    mma_k64(tmem, sA, sm + SM_W + IMG_W3T);
    mma_k128(tmem + 64, sAT, sm + SM_H2T);
    tc::mma_commit(&bar_mma);
  }
  ok = ok && tc::mbar_wait(&bar_mma, ph);
  ph ^= 1;
  tc::fence_after();
  float* part = A.part + (size_t)blockIdx.x * W_N_PARAMS;
  for (int c = 0; c < 4; ++c) {
    float v[16];
    tc::tmem_ld16(tl + 16 * c, v);
    float dz[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int j = 16 * c + e;
      dz[e] = v[e] * sD2[j * TM + t];
      if (!valid) dz[e] = 0.0f;
      red_add(dz[e], &sRed[R_B2 + j]);
      store_t(sAT, 128, j, t, dz[e]);
    }
    store_chunk(sA, t, 2 * c, dz);
    store_chunk(sA, t, 2 * c + 1, dz + 8);
  }
  if (warp < 2) {   // lanes 0..63 hold dW3[out = lane][in]
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tc::tmem_ld16(tl + 64 + 16 * c, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) part[W_OW3 + t * 64 + 16 * c + e] = v[e];
    }
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  // ---- dh1 = dz2 W2, dW2 = dz2^T h1
  if (t == 0) {
    tc::fence_after();
    mma_k64(tmem, sA, sm + SM_W + IMG_W2T);
    mma_k128(tmem + 64, sAT, sm + SM_H1T);
    tc::mma_commit(&bar_mma);
  }
  ok = ok && tc::mbar_wait(&bar_mma, ph);
  ph ^= 1;
  tc::fence_after();
  for (int c = 0; c < 4; ++c) {
    float v[16];
    tc::tmem_ld16(tl + 16 * c, v);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int j = 16 * c + e;
      const float dz = valid ? v[e] * sD1[j * TM + t] : 0.0f;
      red_add(dz, &sRed[R_B1 + j]);
#pragma unroll
      for (int i = 0; i < 4; ++i) red_add(dz * x[i], &sRed[R_W1 + 4 * j + i]);
    }
  }
  if (warp < 2) {
    for (int c = 0; c < 4; ++c) {
      float v[16];
      tc::tmem_ld16(tl + 64 + 16 * c, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) part[W_OW2 + t * 64 + 16 * c + e] = v[e];
    }
  }
  tc::fence_before();
  __syncthreads();
  // ---- the tile's sums of the small layers
  for (int k = t; k < 256; k += NT) part[W_OW1 + k] = sRed[R_W1 + k];
  for (int k = t; k < 64; k += NT) {
    part[W_OB1 + k] = sRed[R_B1 + k];
    part[W_OB2 + k] = sRed[R_B2 + k];
    part[W_OB3 + k] = sRed[R_B3 + k];
  }
  for (int k = t; k < 128; k += NT) part[W_OW4 + k] = sRed[R_W4 + k];
  if (t < 2) part[W_OB4 + t] = sRed[R_B4 + t];
  if (t == 0) A.loss_part[blockIdx.x] = sRed[R_LOSS];
  if (!tc::cta_teardown(ok, &bar_end, &bar_ld, 0, tmem, 128) && t == 0) atomicOr(A.err, 1u);
}

// ------------------------------------------------- reduction, Adam, images
struct UpdateArgs {
  const float* part;   // [tiles][8770]
  int tiles;
  int mode;            // 0: gradient only, 1: Adam step, 2: refresh images from the master
  float* master;
  float* m;
  float* v;
  float* grad_out;     // mode 0
  float lr, beta1, beta2, eps, c1, c2;   // c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t)
  uint8_t* img;
  float* small;
  const float* loss_part;
  float* loss_out;     // sum of the tiles' loss sums
};

__global__ void __launch_bounds__(256) k_sur_update(UpdateArgs U) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && U.loss_out) {
    float s = 0.0f;
    for (int k = 0; k < U.tiles; ++k) s += U.loss_part[k];
    *U.loss_out = s;
  }
  if (p >= W_N_PARAMS) return;
  float th = U.master[p];
  if (U.mode != 2) {
    float g = 0.0f;
    for (int k = 0; k < U.tiles; ++k) g += U.part[(size_t)k * W_N_PARAMS + p];
    if (U.mode == 0) {
      U.grad_out[p] = g;
      return;
    }
    const float mm = U.beta1 * U.m[p] + (1.0f - U.beta1) * g;
    const float vv = U.beta2 * U.v[p] + (1.0f - U.beta2) * g * g;
    U.m[p] = mm;
    U.v[p] = vv;
    th -= U.lr * (mm * U.c1) / (sqrtf(vv * U.c2) + U.eps);
    U.master[p] = th;
  }
  const float wb = th;                                 // layers 1, 4 and biases: FP32
  const __nv_bfloat16 hb = __float2bfloat16_rn(th);    // tensor-core operands: BF16
  if (p < W_OB1) {
    U.small[S_W1 + p] = wb;
  } else if (p < W_OW2) {
    U.small[S_B1 + p - W_OB1] = wb;
  } else if (p < W_OB2) {
    const int q = p - W_OW2, o = q >> 6, i = q & 63;
    *reinterpret_cast<__nv_bfloat16*>(U.img + IMG_W2 + tc::sw128(o, i)) = hb;
    *reinterpret_cast<__nv_bfloat16*>(U.img + IMG_W2T + tc::sw128(i, o)) = hb;
  } else if (p < W_OW3) {
    U.small[S_B2 + p - W_OB2] = wb;
  } else if (p < W_OB3) {
    const int q = p - W_OW3, o = q >> 6, i = q & 63;
    *reinterpret_cast<__nv_bfloat16*>(U.img + IMG_W3 + tc::sw128(o, i)) = hb;
    *reinterpret_cast<__nv_bfloat16*>(U.img + IMG_W3T + tc::sw128(i, o)) = hb;
  } else if (p < W_OW4) {
    U.small[S_B3 + p - W_OB3] = wb;
  } else if (p < W_OB4) {
    U.small[S_W4 + p - W_OW4] = wb;
  } else {
    U.small[S_B4 + p - W_OB4] = wb;
  }
}

// ------------------------------------------------------------ inference
struct InferArgs {
  const float* feat;    // n rows of `stride` floats, inputs in columns 0..3
  int stride;
  long long n;
  const uint8_t* img;
  const float* small;
  float* out;           // n x 4: y0, y1, dy0/df0, dy1/df0
  unsigned* err;
};

// Forward pass of 128-row tiles with the tangent in f0 (sur_mlp.h), tiles
// taken grid-stride.
__global__ void __launch_bounds__(NT, 1) k_sur_infer(InferArgs A) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ uint32_t s_taddr;
  MlpCta M;
  mlp_begin(M, smem_raw, bars, &s_taddr, A.img, A.small);
  const int t = threadIdx.x;
  const long long ntiles = (A.n + TM - 1) / TM;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row = tile * TM + t;
    const bool valid = row < A.n;
    float x[4] = {0.f, 0.f, 0.f, 1.f};
    if (valid) {
      const float* f = A.feat + (size_t)row * A.stride;
      x[0] = f[0]; x[1] = f[1]; x[2] = f[2]; x[3] = f[3];
    }
    float y0, y1, g0, g1;
    mlp_tile(M, x, y0, y1, g0, g1);
    if (valid) *reinterpret_cast<float4*>(A.out + 4 * row) = make_float4(y0, y1, g0, g1);
  }
  if (!mlp_end(M) && t == 0) atomicOr(A.err, 1u);
}

// ------------------------------------------------------------- validation
// errors of the network against quadrature, per record: drag error
// |F_nn - F_q| / (|F_q| + F_abs) and |ln N_nn - ln N_q|; -1 where the rate is
// below the scoring floor LE
__global__ void k_sur_val(const float* rec, const float* y, long long n, float* err2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* r = rec + 16 * i;
  if (!(r[8] > LE)) {
    err2[2 * i] = -1.0f;
    err2[2 * i + 1] = -1.0f;
    return;
  }
  const double lnN = fmax((double)r[7], (double)LT) + (double)y[4 * i + 1];
  const double F = (double)r[11] * (double)r[12] * exp(lnN) * (double)y[4 * i];
  err2[2 * i] = (float)(fabs(F - (double)r[9]) / (fabs((double)r[9]) + (double)r[10]));
  err2[2 * i + 1] = (float)fabs(lnN - (double)r[8]);
}

}  // namespace sur

// ------------------------------------------------------------- host side
cudaError_t sur_launch_samples(const SurPhys& Q, unsigned long long seed, unsigned long long start, long long n,
                               double r_lo, double r_hi, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  sur::k_sur_samples<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(Q, seed, start, n, r_lo, r_hi, out);
  return cudaGetLastError();
}

static bool g_smem_set = false;

static cudaError_t set_smem() {
  if (g_smem_set) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(sur::k_sur_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       sur::TRAIN_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sur::k_sur_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, sur::MF_SMEM);
  if (e == cudaSuccess) g_smem_set = true;
  return e;
}

cudaError_t sur_launch_train(const SurBufs& B, const float* samples, long long n, unsigned long long perm_a,
                             unsigned long long perm_c, long long row0, int rows, cudaStream_t s) {
  cudaError_t e = set_smem();
  if (e != cudaSuccess) return e;
  sur::TrainArgs A;
  A.samples = samples;
  A.n = n;
  A.perm_a = perm_a;
  A.perm_c = perm_c;
  A.row0 = row0;
  A.rows = rows;
  A.inv_batch = 1.0f / (float)rows;
  A.img = B.img;
  A.small = B.small;
  A.part = B.part;
  A.loss_part = B.loss_part;
  A.err = B.err;
  const int tiles = (rows + sur::TM - 1) / sur::TM;
  sur::k_sur_train<<<tiles, sur::NT, sur::TRAIN_SMEM, s>>>(A);
  return cudaGetLastError();
}

cudaError_t sur_launch_update(const SurBufs& B, int tiles, int mode, float lr, int adam_t, float* grad_out,
                              float* loss_out, cudaStream_t s) {
  sur::UpdateArgs U;
  U.part = B.part;
  U.tiles = tiles;
  U.mode = mode;
  U.master = B.master;
  U.m = B.m;
  U.v = B.v;
  U.grad_out = grad_out;
  U.lr = lr;
  U.beta1 = 0.9f;
  U.beta2 = 0.999f;
  U.eps = 1e-8f;
  U.c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)adam_t)));
  U.c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)adam_t)));
  U.img = B.img;
  U.small = B.small;
  U.loss_part = B.loss_part;
  U.loss_out = loss_out;
  sur::k_sur_update<<<(W_N_PARAMS + 255) / 256, 256, 0, s>>>(U);
  return cudaGetLastError();
}

cudaError_t sur_launch_infer(const SurBufs& B, const float* feat, int stride, long long n, float* out, int grid,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = set_smem();
  if (e != cudaSuccess) return e;
  sur::InferArgs A;
  A.feat = feat;
  A.stride = stride;
  A.n = n;
  A.img = B.img;
  A.small = B.small;
  A.out = out;
  A.err = B.err;
  const long long tiles = (n + sur::TM - 1) / sur::TM;
  const int g = (int)std::min<long long>(tiles, grid);
  sur::k_sur_infer<<<g, sur::NT, sur::MF_SMEM, s>>>(A);
  return cudaGetLastError();
}

cudaError_t sur_launch_val(const float* rec, const float* y, long long n, float* err2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  sur::k_sur_val<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rec, y, n, err2);
  return cudaGetLastError();
}

}  // namespace pic1d
