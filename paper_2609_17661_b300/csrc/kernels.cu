// kernels.cu -- sm_103a kernels of the per-step particle loop.
//
//   k_push     gather E, Strang-split drag around the Lorentz kick (Sec. 3),
//              Monte-Carlo RICS scattering with recoil and pair creation
//              (Sec. 3, App. A), move, charge-conserving int64 deposit through
//              a shared-memory cell window with warp-segmented reduction,
//              loss flags at the conducting walls, pair append.
//   k_inject   surface supply at both footpoints (RATE mode).
//   k_field    Ampere with the external current in FP64 (Sec. 3) + totals.
//   k_finalize per-step scalars in a fixed summation order.
//   k_hist / k_scan / k_scatter   periodic cell sort (drops removed slots).
//   k_table    drag/rate table by FP64 quadrature over the stellar disk
//              (Sec. 2.2, Eq. scatteringNdot and Eq. contdrag).
//
// The particle SoA is read with 128-bit loads: one thread owns 4 consecutive
// particles, a block owns a contiguous range of tiles, so that cell-sorted
// particles of one block fall into a narrow window of cells.
#include <math.h>

#include "pic1d_internal.h"

namespace pic1d {

// --------------------------------------------------------------------------
// counter-based random numbers: Philox4x32-10 (Salmon et al., SC'11)
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ float unit24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// SplitMix64 finaliser (Steele, Lea, Flood 2014): stable ids of created particles
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long pair_child_id(unsigned long long parent, long long step, int m) {
  return mix64(parent ^ mix64((unsigned long long)step * 2ull + (unsigned long long)m)) | 0x8000000000000000ull;
}
__device__ __forceinline__ unsigned long long supply_id(long long step, int foot, long long slot, int m) {
  const unsigned long long k = ((unsigned long long)step << 24) ^ ((unsigned long long)foot << 23) ^
                               ((unsigned long long)slot << 1) ^ (unsigned long long)m;
  return mix64(k ^ 0x5A17A5EEDull) | 0x8000000000000000ull;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// --------------------------------------------------------------------------
// drag and scattering rate at one particle
// --------------------------------------------------------------------------
struct Site {        // what the push needs about the particle's place on the line
  float v;           // table coordinate in s/L
  float x, b, mu;    // r/R*, B/B_QED, cos(radial, +s) interpolated at s
};

struct DragVal {
  float F, dF, lnN;  // F^ (per R*), dF^/du, ln N^ (per R_star/c)
};

__device__ __forceinline__ DragVal table_eval(const DevParams& P, float u, float v, bool want_dF) {
  const float gam = sqrtf(fmaf(u, u, 1.0f));
  float t = log2f(gam) * P.t_scale;
  bool top = false;
  if (t > (float)(P.Ng - 1)) { t = (float)(P.Ng - 1); top = true; }
  const int i = min((int)t, P.Ng - 2);
  const float a = t - (float)i;
  const int j = min((int)v, P.Ns - 2);
  const float c = v - (float)j;
  const int sg = (u >= 0.0f) ? 0 : 1;
  const float2* r0 = P.table + ((size_t)(sg * P.Ns + j) * P.Ng);
  const float2* r1 = r0 + P.Ng;
  const float2 q00 = __ldg(r0 + i), q10 = __ldg(r0 + i + 1), q01 = __ldg(r1 + i), q11 = __ldg(r1 + i + 1);
  const float ac = 1.0f - a, cc = 1.0f - c;
  DragVal d;
  d.F = ac * cc * q00.x + a * cc * q10.x + ac * c * q01.x + a * c * q11.x;
  d.lnN = ac * cc * q00.y + a * cc * q10.y + ac * c * q01.y + a * c * q11.y;
  d.dF = 0.0f;
  if (want_dF && !top) {
    const float dFdt = cc * (q10.x - q00.x) + c * (q11.x - q01.x);
    d.dF = dFdt * (u / (gam * gam)) * P.dtdu_scale;
  }
  return d;
}

// closed form for radially streaming photons (Eq. contdrag and the matching
// rate of Eq. scatteringNdot with solid angle pi/x^2)
__device__ __forceinline__ DragVal closed_eval(const DevParams& P, float u, const Site& S, bool want_dF) {
  const float gam = sqrtf(fmaf(u, u, 1.0f));
  const float beta = u / gam;
  const float au = fabsf(u);
  const float sm = (u >= 0.0f) ? S.mu : -S.mu;
  const float omb = 1.0f / (gam * (gam + au));          // 1 - |beta|
  const float Dm = (1.0f - sm) + sm * omb;             // 1 - beta_s mu
  const float eps = S.b / (gam * Dm);
  const float y = eps / P.theta_T;
  const float em = expm1f(y);
  const float g = (y * y * y) / em;
  const float ix2 = 1.0f / (S.x * S.x);
  DragVal d;
  d.F = P.closedK * ix2 * gam * (S.mu - beta) * g;
  const float N = P.closedN * ix2 / gam * (eps * eps) / em;
  d.lnN = (N > 0.0f) ? logf(N) : -700.0f;
  d.dF = 0.0f;
  if (want_dF) {
    const float D = gam * Dm;
    const float gp = g * (3.0f / y - 1.0f / (-expm1f(-y)));
    const float dydu = -y * (beta - S.mu) / D;
    d.dF = P.closedK * ix2 * ((beta * S.mu - 1.0f) * g + gam * (S.mu - beta) * gp * dydu);
  }
  return d;
}

__device__ __forceinline__ DragVal drag_eval(const DevParams& P, float u, const Site& S, bool want_dF) {
  if (P.drag_law == PIC1D_DRAG_TABLE) return table_eval(P, u, S.v, want_dF);
  return closed_eval(P, u, S, want_dF);
}

// One drag update over dt/2 at fixed s (Sec. 3): limiter test |F| tau_min <
// |u0|, then the implicit midpoint [Eq. implicit] by 4 Newton iterations or
// exponential damping toward p~ = mu / sqrt(1 - mu^2).
__device__ __forceinline__ float drag_half(const DevParams& P, const Site& S, float u0, unsigned& n_lim,
                                           unsigned& n_newt) {
  const float h = P.half_dt;
  const DragVal d0 = drag_eval(P, u0, S, true);
  const float F0 = P.drag_k * d0.F;
  bool newton = true;
  if (P.limiter_on) newton = fabsf(F0) * P.tau_min < fabsf(u0);
  if (newton) {
    ++n_newt;
    float u1 = fmaf(h, F0, u0);
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
      const DragVal d1 = drag_eval(P, u1, S, true);
      const float F1 = P.drag_k * d1.F;
      const float G = u1 - u0 - 0.5f * h * (F0 + F1);
      const float dG = fmaxf(1.0f - 0.5f * h * P.drag_k * d1.dF, 0.5f);
      u1 -= G / dG;
    }
    return u1;
  }
  ++n_lim;
  const float ut = S.mu / sqrtf(1.0f - S.mu * S.mu);
  return ut + (u0 - ut) * P.damp;
}

// de-excitation angle with density (3/8)(1 + c^2): Cardano root of c^3 + 3c + 4 - 8U = 0
__device__ __forceinline__ float dipole_cos(float U) {
  const float a = 4.0f * U - 2.0f;
  const float t = cbrtf(a + sqrtf(fmaf(a, a, 1.0f)));
  return t - 1.0f / t;
}

// RICS event (App. A): excitation by a photon arriving along d (= +-1 along s)
// in the lepton rest frame, de-excitation at cos(theta~) = ct; returns the
// recoiled momentum, the photon's lab energy and momentum along s.
__device__ __forceinline__ void rics_event(float b, float d, float ui, float ct, float& uf, float& Eg,
                                           float& Pg) {
  const float EB = sqrtf(fmaf(2.0f, b, 1.0f));
  const float iEB = 1.0f / EB;
  const float gs = 0.5f * (EB + iEB);
  const float gbs = b * iEB;
  const float gi = sqrtf(fmaf(ui, ui, 1.0f));
  const float ge = gs * gi + d * gbs * ui;
  const float ue = gs * ui + d * gbs * gi;
  const float st2 = 1.0f - ct * ct;
  const float Ep = (EB - iEB) / (1.0f + sqrtf(ct * ct + st2 * iEB * iEB));
  const float Ee = EB - Ep, pe = -Ep * ct;
  uf = ue * Ee + ge * pe;
  Eg = Ep * (ge + ue * ct);
  Pg = Ep * (ue + ge * ct);
}

// --------------------------------------------------------------------------
// deposit helpers: a thread accumulates the currents of its particles into
// three registers for cells c_ref-1, c_ref, c_ref+1; anything else goes
// straight to the window (shared) or to global memory.
// --------------------------------------------------------------------------
__device__ __forceinline__ void add_cell(long long* sWin, int win_lo, long long* g, int N, int cell, long long v) {
  if (v == 0 || cell < 0 || cell >= N) return;
  const int o = cell - win_lo;
  if (o >= 0 && o < kWindow)
    atomicAdd(reinterpret_cast<unsigned long long*>(sWin + o), (unsigned long long)v);
  else
    atomicAdd(reinterpret_cast<unsigned long long*>(g + cell), (unsigned long long)v);
}

__device__ __forceinline__ void acc_cell(long long (&a)[3], int c_ref, long long* sWin, int win_lo, long long* g,
                                         int N, int cell, long long v) {
  const int o = cell - c_ref + 1;
  if (o == 0) a[0] += v;
  else if (o == 1) a[1] += v;
  else if (o == 2) a[2] += v;
  else add_cell(sWin, win_lo, g, N, cell, v);
}

// path [a, b] in fixed point (both inside [0, top]): signed length inside each
// cell times wq, the 1D charge-conserving current of Sec. 3.
__device__ __forceinline__ void deposit_path(long long (&acc)[3], int c_ref, long long* sWin, int win_lo,
                                             long long* g, const DevParams& P, long long a, long long b,
                                             long long wq) {
  if (a == b) return;
  const long long lo = a < b ? a : b, hi = a < b ? b : a;
  const long long sw = (b > a) ? wq : -wq;
  const int c0 = (int)(lo >> P.F), c1 = (int)((hi - 1) >> P.F);
  if (c0 == c1) {
    acc_cell(acc, c_ref, sWin, win_lo, g, P.N, c0, sw * (hi - lo));
  } else {
    const long long k = (long long)c1 << P.F;
    acc_cell(acc, c_ref, sWin, win_lo, g, P.N, c0, sw * (k - lo));
    acc_cell(acc, c_ref, sWin, win_lo, g, P.N, c1, sw * (hi - k));
  }
}

// warp-level segmented reduction of the per-thread registers keyed by c_ref
// (valid when c_ref is non-decreasing along the lanes: cell-sorted data),
// then one atomic per segment and cell.
__device__ __forceinline__ void warp_flush(long long (&a)[3], int c_ref, long long* sWin, int win_lo,
                                           long long* g, int N) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(full, c_ref, 1);
  const bool ok = (lane == 0) || (prev <= c_ref);
  if (__all_sync(full, ok)) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int kd = __shfl_up_sync(full, c_ref, d);
      const long long v0 = __shfl_up_sync(full, a[0], d);
      const long long v1 = __shfl_up_sync(full, a[1], d);
      const long long v2 = __shfl_up_sync(full, a[2], d);
      if (lane >= d && kd == c_ref) { a[0] += v0; a[1] += v1; a[2] += v2; }
    }
    const int next = __shfl_down_sync(full, c_ref, 1);
    if (lane == 31 || next != c_ref) {
      add_cell(sWin, win_lo, g, N, c_ref - 1, a[0]);
      add_cell(sWin, win_lo, g, N, c_ref, a[1]);
      add_cell(sWin, win_lo, g, N, c_ref + 1, a[2]);
    }
  } else {
    add_cell(sWin, win_lo, g, N, c_ref - 1, a[0]);
    add_cell(sWin, win_lo, g, N, c_ref, a[1]);
    add_cell(sWin, win_lo, g, N, c_ref + 1, a[2]);
  }
  a[0] = a[1] = a[2] = 0;
}

// --------------------------------------------------------------------------
// the push: one PIC cycle for every particle slot
// --------------------------------------------------------------------------
enum { C_SCAT, C_CLAMP, C_LIM, C_NEWT, C_NONFIN, C_LOSTN, C_LOSTS, C_PAIRS, C_DROP, C_REJ, C_WALL, C_DRAW, C_COUNT };

template <bool NMAX>
__global__ void __launch_bounds__(kBlock) k_push(DevParams P) {
  __shared__ long long sJ[kWindow];
  __shared__ long long sD[NMAX ? kWindow : 1];
  __shared__ unsigned sCtr[C_COUNT];
  __shared__ double sRed[2][kBlock / 32];

  const long long n = P.st->n_slots;
  const int lane = threadIdx.x & 31;
  const long long ntiles = (n + kTile - 1) / kTile;
  const long long tpb = (ntiles + gridDim.x - 1) / gridDim.x;
  const long long t0 = (long long)blockIdx.x * tpb;
  const long long t1 = min(ntiles, t0 + tpb);

  int win_lo = 0;
  if (t0 < t1) {
    const int c = (int)(P.pos[t0 * kTile] >> P.F);
    win_lo = max(0, min(c, P.N - 1) - kWindow / 8);
  }
  for (int i = threadIdx.x; i < kWindow; i += kBlock) {
    sJ[i] = 0;
    if (NMAX) sD[i] = 0;
  }
  if (threadIdx.x < C_COUNT) sCtr[threadIdx.x] = 0;
  __syncthreads();

  unsigned cnt[C_COUNT];
#pragma unroll
  for (int k = 0; k < C_COUNT; ++k) cnt[k] = 0;
  unsigned n_lim = 0, n_newt = 0;     // scalars: references into cnt[] would force it to local memory
  // Kahan-compensated FP32 sums (FP64 adds per particle would cost a
  // noticeable share of the step on this part's FP64 rate)
  float ke = 0.0f, ke_c = 0.0f, kl = 0.0f, kl_c = 0.0f;
  const float two_F = (float)(1u << P.F);
  const unsigned long long fmask = (1ull << P.F) - 1ull;

  for (long long t = t0; t < t1; ++t) {
    const long long base = t * kTile + (long long)threadIdx.x * kPerThread;
    uint4 p4 = *reinterpret_cast<const uint4*>(P.pos + base);
    float4 u4 = *reinterpret_cast<const float4*>(P.u + base);
    const float4 w4 = *reinterpret_cast<const float4*>(P.w + base);
    const uchar4 s4 = *reinterpret_cast<const uchar4*>(P.sp + base);
    uint32_t pp[4] = {p4.x, p4.y, p4.z, p4.w};
    float uu[4] = {u4.x, u4.y, u4.z, u4.w};
    const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
    uint8_t ss[4] = {s4.x, s4.y, s4.z, s4.w};
    const int c_ref = min((int)(pp[0] >> P.F), P.N - 1);
    long long aJ[3] = {0, 0, 0};
    long long aD[3] = {0, 0, 0};
    bool dirty = false;

#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      const long long idx = base + k;
      const bool valid = (idx < n) && (ss[k] != PIC1D_SP_DEAD);
      bool want_pair = false;
      float child_u = 0.0f;
      long long p1 = 0;
      unsigned long long pid = 0;
      if (valid) {
        const int sp = ss[k] & 3;
        const uint32_t pos0 = pp[k];
        float u = uu[k];
        const float w = ww[k];
        const bool lep = (sp != PIC1D_SP_ION);
        const int cell = min((int)(pos0 >> P.F), P.N - 1);
        // 1. gather E linearly between cell centres
        float Ep;
        {
          const long long xg = (long long)pos0 - (1ll << (P.F - 1));
          const int ig = (int)(xg >> P.F);
          if (ig < 0) Ep = __ldg(P.E32);
          else if (ig >= P.N - 1) Ep = __ldg(P.E32 + P.N - 1);
          else {
            const float f = (float)((unsigned long long)xg & fmask) * P.inv2F;
            const float e0 = __ldg(P.E32 + ig), e1 = __ldg(P.E32 + ig + 1);
            Ep = fmaf(f, e1 - e0, e0);
          }
        }
        const bool zone = __ldg(P.zone + cell) != 0;
        const bool cont = lep && P.drag_law != PIC1D_DRAG_OFF && (P.rics_mode == PIC1D_RICS_DRAG_PLUS_PAIRS || !zone);
        const bool mc = lep && P.mc_on && P.drag_law != PIC1D_DRAG_OFF && zone;
        Site S;
        if (cont || mc) {
          const float f = (float)(pos0 & (uint32_t)fmask) * P.inv2F;
          const int cn = cell;
          const float b0 = __ldg(P.nb + cn), b1 = __ldg(P.nb + cn + 1);
          const float m0 = __ldg(P.nmu + cn), m1 = __ldg(P.nmu + cn + 1);
          S.b = fmaf(f, b1 - b0, b0);
          S.mu = fmaf(f, m1 - m0, m0);
          if (P.drag_law == PIC1D_DRAG_CLOSED) {
            const float x0 = __ldg(P.nx + cn), x1 = __ldg(P.nx + cn + 1);
            S.x = fmaf(f, x1 - x0, x0);
          } else {
            S.x = 1.0f;
          }
          S.v = fminf((float)pos0 * P.v_scale, (float)(P.Ns - 1));
        }
        // 2-4. Strang split: drag dt/2, Lorentz kick dt, drag dt/2
        if (cont) u = drag_half(P, S, u, n_lim, n_newt);
        u = fmaf(P.qm[sp] * Ep, P.dt, u);
        if (cont) u = drag_half(P, S, u, n_lim, n_newt);
        // 5. Monte-Carlo RICS in the pair zone
        bool make_pair = false;
        float Pg = 0.0f;
        if (mc) {
          const DragVal dv = drag_eval(P, u, S, false);
          float psc = P.drag_k * expf(dv.lnN) * P.dt;
          if (psc > 1.0f) { psc = 1.0f; ++cnt[C_CLAMP]; }
          if (psc > 0.0f) {
            ++cnt[C_DRAW];
            pid = P.id[idx];
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)P.step, kTagRics), P.key0, P.key1);
            if (unit24(r.x) < psc) {
              ++cnt[C_SCAT];
              const float gam = sqrtf(fmaf(u, u, 1.0f));
              const float d = (S.mu > u / gam) ? 1.0f : -1.0f;
              const float ct = dipole_cos(unit24(r.y));
              float uf, Eg;
              rics_event(S.b, d, u, ct, uf, Eg, Pg);
              if (P.rics_mode == PIC1D_RICS_SPLIT) u = uf;
              if (P.pairs_on && Eg >= P.pair_e_thr) make_pair = true;
            }
          }
        }
        // 6. move
        bool lost;
        if (!isfinite(u)) {
          ++cnt[C_NONFIN];
          u = 0.0f;
          p1 = (long long)pos0;
          lost = true;
          make_pair = false;
        } else {
          const float gam = sqrtf(fmaf(u, u, 1.0f));
          const float ds = P.dt * (u / gam);
          p1 = (long long)pos0 + __float2ll_rn(ds * two_F);
          lost = (p1 < 0) || (p1 >= P.top);
          const float gm1 = (u * u) / (gam + 1.0f);
          const float e = w * P.mass[sp] * gm1;
          if (lost) {
            const float y = e - kl_c, t = kl + y;
            kl_c = (t - kl) - y;
            kl = t;
            if (p1 < 0) ++cnt[C_LOSTN]; else ++cnt[C_LOSTS];
          } else {
            const float y = e - ke_c, t = ke + y;
            ke_c = (t - ke) - y;
            ke = t;
          }
        }
        // 7. charge-conserving deposit along the path, clamped at the walls
        const long long pc = p1 < 0 ? 0 : (p1 > P.top ? P.top : p1);
        const long long wint = __float2ll_rn(w * 4096.0f);
        deposit_path(aJ, c_ref, sJ, win_lo, P.J, P, (long long)pos0, pc, (long long)P.qs[sp] * wint);
        if (NMAX && lep && !lost) acc_cell(aD, c_ref, sD, win_lo, P.dens_next, P.N, (int)(p1 >> P.F), wint);
        pp[k] = lost ? (uint32_t)min(pc, P.top - 1) : (uint32_t)p1;
        uu[k] = u;
        if (lost) { ss[k] = PIC1D_SP_DEAD; dirty = true; }
        if (make_pair) {
          if (lost) {
            ++cnt[C_WALL];
          } else if (NMAX && P.dens_cur[(int)(p1 >> P.F)] >= P.nmax_int) {
            ++cnt[C_REJ];
          } else {
            want_pair = true;
            child_u = 0.5f * Pg;
          }
        }
      }
      // pair append, warp-aggregated (uniform control flow)
      const unsigned m = __ballot_sync(0xffffffffu, want_pair);
      if (m) {
        const int leader = __ffs(m) - 1;
        long long slot0 = 0;
        if (lane == leader) slot0 = atomicAdd(reinterpret_cast<unsigned long long*>(&P.st->append),
                                              (unsigned long long)(2 * __popc(m)));
        slot0 = __shfl_sync(0xffffffffu, slot0, leader);
        if (want_pair) {
          const long long dst = n + slot0 + 2ll * __popc(m & lanemask_lt());
          if (dst + 2 > P.cap) {
            ++cnt[C_DROP];
          } else {
            ++cnt[C_PAIRS];
            const uint32_t cpos = (uint32_t)p1;
#pragma unroll
            for (int mm = 0; mm < 2; ++mm) {
              P.pos[dst + mm] = cpos;
              P.u[dst + mm] = child_u;
              P.w[dst + mm] = ww[k];
              P.sp[dst + mm] = (mm == 0) ? PIC1D_SP_ELECTRON : PIC1D_SP_POSITRON;
              P.id[dst + mm] = pair_child_id(pid, P.step, mm);
            }
            if (NMAX)
              atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + (int)(p1 >> P.F)),
                        (unsigned long long)(2ll * __float2ll_rn(ww[k] * 4096.0f)));
          }
        }
      }
    }
    // write back
    if (base + kPerThread <= n) {
      *reinterpret_cast<uint4*>(P.pos + base) = make_uint4(pp[0], pp[1], pp[2], pp[3]);
      *reinterpret_cast<float4*>(P.u + base) = make_float4(uu[0], uu[1], uu[2], uu[3]);
    } else {
#pragma unroll
      for (int k = 0; k < kPerThread; ++k)
        if (base + k < n) { P.pos[base + k] = pp[k]; P.u[base + k] = uu[k]; }
    }
    if (dirty) {
#pragma unroll
      for (int k = 0; k < kPerThread; ++k)
        if (base + k < n && ss[k] == PIC1D_SP_DEAD) P.sp[base + k] = PIC1D_SP_DEAD;
    }
    warp_flush(aJ, c_ref, sJ, win_lo, P.J, P.N);
    if (NMAX) warp_flush(aD, c_ref, sD, win_lo, P.dens_next, P.N);
  }

  // counters and energy totals of the block
  cnt[C_LIM] = n_lim;
  cnt[C_NEWT] = n_newt;
#pragma unroll
  for (int k = 0; k < C_COUNT; ++k) {
    const unsigned v = __reduce_add_sync(0xffffffffu, cnt[k]);
    if (lane == 0 && v) atomicAdd(&sCtr[k], v);
  }
  double ked = (double)ke - (double)ke_c, kld = (double)kl - (double)kl_c;
  for (int d = 16; d > 0; d >>= 1) {
    ked += __shfl_down_sync(0xffffffffu, ked, d);
    kld += __shfl_down_sync(0xffffffffu, kld, d);
  }
  if (lane == 0) { sRed[0][threadIdx.x >> 5] = ked; sRed[1][threadIdx.x >> 5] = kld; }
  __syncthreads();
  // flush the window
  for (int i = threadIdx.x; i < kWindow; i += kBlock) {
    const int cell = win_lo + i;
    if (cell < P.N) {
      if (sJ[i]) atomicAdd(reinterpret_cast<unsigned long long*>(P.J + cell), (unsigned long long)sJ[i]);
      if (NMAX && sD[i]) atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + cell), (unsigned long long)sD[i]);
    }
  }
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) { a += sRed[0][i]; b += sRed[1][i]; }
    P.ke_partial[blockIdx.x] = a;
    if (b != 0.0) atomicAdd(&P.st->ke_lost, b);
    Counters* C = P.ctr;
    unsigned long long* dst[C_COUNT] = {&C->scatters, &C->psc_clamped, &C->limiter_branch, &C->newton_branch,
                                        &C->nonfinite, &C->lost_north, &C->lost_south, &C->pairs_created,
                                        &C->pairs_dropped_cap, &C->pairs_rejected_nmax, &C->pairs_lost_wall,
                                        &C->rng_draws};
    for (int k = 0; k < C_COUNT; ++k)
      if (sCtr[k]) atomicAdd(dst[k], (unsigned long long)sCtr[k]);
  }
}

// --------------------------------------------------------------------------
// surface supply: neutral e- (atmospheric) + ion pairs at both footpoints
// --------------------------------------------------------------------------
__global__ void k_inject(DevParams P, double carriers, float sig_e, float sig_i) {
  __shared__ long long cnt[2];
  __shared__ long long slot0;
  if (threadIdx.x == 0) {
    for (int f = 0; f < 2; ++f) {
      const double acc = P.st->inj_acc[f] + carriers;
      const double c = floor(acc);
      P.st->inj_acc[f] = acc - c;
      cnt[f] = (long long)c;
    }
    slot0 = atomicAdd(reinterpret_cast<unsigned long long*>(&P.st->append),
                      (unsigned long long)(2 * (cnt[0] + cnt[1])));
  }
  __syncthreads();
  const long long n = P.st->n_slots;
  const long long total = cnt[0] + cnt[1];
  unsigned ok = 0, drop = 0;
  for (long long k = threadIdx.x; k < total; k += blockDim.x) {
    const int foot = (k < cnt[0]) ? 0 : 1;
    const long long slot = foot ? k - cnt[0] : k;
    const long long dst = n + slot0 + 2 * k;
    if (dst + 2 > P.cap) { ++drop; continue; }
    const uint4 r = philox4x32_10(make_uint4((uint32_t)slot, (uint32_t)foot, (uint32_t)P.step, kTagInj), P.key0, P.key1);
    const long long q = (long long)(r.x >> 16);
    long long pfix;
    if (P.F >= 16) pfix = foot == 0 ? (q << (P.F - 16)) : P.top - ((q + 1) << (P.F - 16));
    else pfix = foot == 0 ? (q >> (16 - P.F)) : P.top - 1 - (q >> (16 - P.F));
    const float rad = sqrtf(-2.0f * logf(1.0f - unit24(r.y)));
    const float ang = 6.283185307179586f * unit24(r.z);
    const float dir = foot == 0 ? 1.0f : -1.0f;
    const float ue = dir * fabsf(sig_e * rad * cosf(ang));
    const float ui = dir * fabsf(sig_i * rad * sinf(ang));
    for (int m = 0; m < 2; ++m) {
      P.pos[dst + m] = (uint32_t)pfix;
      P.u[dst + m] = m == 0 ? ue : ui;
      P.w[dst + m] = 1.0f;
      P.sp[dst + m] = m == 0 ? PIC1D_SP_ATMO : PIC1D_SP_ION;
      P.id[dst + m] = supply_id(P.step, foot, slot, m);
    }
    if (P.use_nmax)
      atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + (int)(pfix >> P.F)), 4096ull);
    ++ok;
  }
  if (ok) atomicAdd(&P.ctr->injected, 2ull * ok);
  if (drop) atomicAdd(&P.ctr->injected_dropped, 2ull * drop);
}

// --------------------------------------------------------------------------
// field update, FP64: E += 4 pi dt j_ext - 4 pi q_p 2^(-F-12) J_int (J_int is kept
// until the next step clears it, so that it can be read back)
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_field(DevParams P, double* E64, float* E32, double a, double cJ,
                                               double* partial) {
  double so = 0.0, sn = 0.0, s2 = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < P.N; c += gridDim.x * blockDim.x) {
    const double Eo = E64[c];
    const double En = Eo + (a - cJ * (double)P.J[c]);
    E64[c] = En;
    E32[c] = (float)En;
    if (P.use_nmax) P.dens_cur[c] = 0;     // becomes the next step's accumulator
    so += Eo;
    sn += En;
    s2 += En * En;
  }
  __shared__ double red[3][8];
  for (int d = 16; d > 0; d >>= 1) {
    so += __shfl_down_sync(0xffffffffu, so, d);
    sn += __shfl_down_sync(0xffffffffu, sn, d);
    s2 += __shfl_down_sync(0xffffffffu, s2, d);
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][wid] = so; red[1][wid] = sn; red[2][wid] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0, z = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { x += red[0][i]; y += red[1][i]; z += red[2][i]; }
    partial[3 * blockIdx.x + 0] = x;
    partial[3 * blockIdx.x + 1] = y;
    partial[3 * blockIdx.x + 2] = z;
  }
}

// per-step scalars in a fixed order (deterministic), slot bookkeeping
__global__ void k_finalize(DevParams P, const double* fpart, int nfb, int npb, double dt_jext) {
  __shared__ double red[4][32];
  double so = 0, sn = 0, s2 = 0, ke = 0;
  for (int i = threadIdx.x; i < nfb; i += 32) { so += fpart[3 * i]; sn += fpart[3 * i + 1]; s2 += fpart[3 * i + 2]; }
  for (int i = threadIdx.x; i < npb; i += 32) ke += P.ke_partial[i];
  red[0][threadIdx.x] = so; red[1][threadIdx.x] = sn; red[2][threadIdx.x] = s2; red[3][threadIdx.x] = ke;
  __syncwarp();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0, d = 0;
    for (int i = 0; i < 32; ++i) { a += red[0][i]; b += red[1][i]; c += red[2][i]; d += red[3][i]; }
    StepState* st = P.st;
    st->field_energy = c / (8.0 * 3.141592653589793);
    st->vc = -b;
    st->ext_work += dt_jext * 0.5 * (a + b);
    st->kinetic = d;
    const long long n = st->n_slots, app = st->append;
    long long room = (P.cap - n) / 2 * 2;
    if (room < 0) room = 0;
    st->n_slots = n + (app < room ? app : room);
    st->append = 0;
  }
}

// --------------------------------------------------------------------------
// cell sort: histogram, exclusive scan, scatter (removed slots dropped)
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_hist(DevParams P, uint32_t* counts) {
  const long long n = P.st->n_slots;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < n; i0 += (long long)gridDim.x * blockDim.x) {
    const long long i = i0 + threadIdx.x;
    bool valid = i < n;
    int cell = 0;
    if (valid) {
      valid = P.sp[i] != PIC1D_SP_DEAD;
      cell = min((int)(P.pos[i] >> P.F), P.N - 1);
    }
    const unsigned vm = __ballot_sync(full, valid);
    if (valid) {
      const unsigned grp = __match_any_sync(vm, cell);
      if (lane == __ffs(grp) - 1) atomicAdd(counts + cell, (unsigned)__popc(grp));
    }
  }
}

__global__ void __launch_bounds__(1024) k_scan(DevParams P, const uint32_t* counts, long long* offsets) {
  __shared__ long long part[1024];
  const int N = P.N;
  const int per = (N + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(N, lo + per);
  long long s = 0;
  for (int c = lo; c < hi; ++c) s += counts[c];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    long long v = (threadIdx.x >= (unsigned)d) ? part[threadIdx.x - d] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = part[threadIdx.x] - s;
  for (int c = lo; c < hi; ++c) { offsets[c] = run; run += counts[c]; }
  if (threadIdx.x == 1023) { offsets[N] = part[1023]; P.st->sorted_total = part[1023]; }
}

__global__ void __launch_bounds__(256) k_scatter(DevParams P, long long* cursor, uint32_t* pos2, float* u2,
                                                 float* w2, uint8_t* sp2, uint64_t* id2) {
  const long long n = P.st->n_slots;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < n; i0 += (long long)gridDim.x * blockDim.x) {
    const long long i = i0 + threadIdx.x;
    bool valid = i < n;
    uint32_t pos = 0;
    uint8_t sp = 0;
    int cell = 0;
    if (valid) {
      sp = P.sp[i];
      pos = P.pos[i];
      valid = sp != PIC1D_SP_DEAD;
      cell = min((int)(pos >> P.F), P.N - 1);
    }
    const unsigned vm = __ballot_sync(full, valid);
    if (valid) {
      const unsigned grp = __match_any_sync(vm, cell);
      const int leader = __ffs(grp) - 1;
      long long b = 0;
      if (lane == leader)
        b = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(cursor + cell), (unsigned long long)__popc(grp));
      b = __shfl_sync(grp, b, leader);
      const long long dst = b + __popc(grp & lanemask_lt());
      pos2[dst] = pos;
      u2[dst] = P.u[i];
      w2[dst] = P.w[i];
      sp2[dst] = sp;
      id2[dst] = P.id[i];
    }
  }
}

__global__ void k_sort_done(DevParams P) {
  P.st->n_slots = P.st->sorted_total;
  P.st->append = 0;
}

// --------------------------------------------------------------------------
// drag/rate table by FP64 quadrature (one thread per entry)
// --------------------------------------------------------------------------
__device__ __forceinline__ double one_minus_beta_cos(double u, double gam, double m) {
  const double sm = (u >= 0.0) ? m : -m;
  return (1.0 - sm) + sm / (gam * (gam + fabs(u)));
}

__global__ void k_table(int Ng, int Ns, int n_mu, int n_phi, double log10g_max, double theta_T, double pref,
                        const double* xs, const double* bs, const double* mus, const double* gx,
                        const double* gw, int photon_model, float2* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * Ns * Ng) return;
  const int ig = idx % Ng;
  const int js = (idx / Ng) % Ns;
  const int sg = idx / (Ng * Ns);
  const double lg = log10g_max * (double)ig / (double)(Ng - 1);
  const double gam = pow(10.0, lg);
  const double au = sqrt(fmax(0.0, gam * gam - 1.0));
  const double u = sg ? -au : au;
  const double beta = u / gam;
  const double x = xs[js], b = bs[js], mu = mus[js];
  double F, N;
  if (photon_model == PIC1D_PHOTON_RADIAL) {
    const double D = one_minus_beta_cos(u, gam, mu);
    const double eps = b / (gam * D);
    const double y = eps / theta_T;
    const double em = expm1(y);
    // the disk's solid angle pi/x^2 in place of the quadrature
    N = pref * 3.141592653589793 / (x * x) * eps * eps / em / gam;
    F = N * gam * b * (mu - beta) / D;
  } else {
    const double cmax = (x > 1.0) ? sqrt(1.0 - 1.0 / (x * x)) : 0.0;
    const double smu = sqrt(fmax(0.0, 1.0 - mu * mu));
    const double wphi = 2.0 * 3.141592653589793 / n_phi;
    double sN = 0.0, sF = 0.0;
    for (int i = 0; i < n_mu; ++i) {
      const double ca = cmax + (1.0 - cmax) * 0.5 * (gx[i] + 1.0);
      const double wa = (1.0 - cmax) * 0.5 * gw[i];
      const double sa = sqrt(fmax(0.0, 1.0 - ca * ca));
      for (int j = 0; j < n_phi; ++j) {
        const double ph = 3.141592653589793 * (j + 0.5) / n_phi;
        const double mk = ca * mu + sa * cos(ph) * smu;
        const double D = one_minus_beta_cos(u, gam, mk);
        const double eps = b / (gam * D);
        const double dN = wa * wphi * eps * eps / expm1(eps / theta_T);
        sN += dN;
        sF += dN * gam * b * (mk - beta) / D;
      }
    }
    N = pref / gam * sN;
    F = pref / gam * sF;
  }
  double lnN = (N > 0.0) ? log(N) : -700.0;
  if (lnN < -700.0) lnN = -700.0;
  out[idx] = make_float2((float)F, (float)lnN);
}

// --------------------------------------------------------------------------
// standalone deposit and species count (tests and diagnostics)
// --------------------------------------------------------------------------
__global__ void k_deposit(DevParams P, long long n, const long long* p0, const long long* p1, const float* w,
                          const uint8_t* sp, long long* J) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long a = p0[i], b = p1[i];
  if (a < 0 || a > P.top) return;
  b = b < 0 ? 0 : (b > P.top ? P.top : b);
  const long long wq = (long long)P.qs[sp[i] & 3] * __float2ll_rn(w[i] * 4096.0f);
  // no register/window staging here: every cell goes straight to global memory
  if (a == b) return;
  const long long lo = a < b ? a : b, hi = a < b ? b : a;
  const long long sw = (b > a) ? wq : -wq;
  const int c0 = (int)(lo >> P.F), c1 = (int)((hi - 1) >> P.F);
  if (c0 == c1) {
    atomicAdd(reinterpret_cast<unsigned long long*>(J + c0), (unsigned long long)(sw * (hi - lo)));
  } else {
    const long long k = (long long)c1 << P.F;
    atomicAdd(reinterpret_cast<unsigned long long*>(J + c0), (unsigned long long)(sw * (k - lo)));
    atomicAdd(reinterpret_cast<unsigned long long*>(J + c1), (unsigned long long)(sw * (hi - k)));
  }
}

__global__ void k_count_species(DevParams P, unsigned long long* out4) {
  const long long n = P.st->n_slots;
  unsigned c[4] = {0, 0, 0, 0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint8_t s = P.sp[i];
    if (s < 4) ++c[s];
  }
  for (int k = 0; k < 4; ++k) {
    const unsigned v = __reduce_add_sync(0xffffffffu, c[k]);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out4 + k, (unsigned long long)v);
  }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
int push_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<false>, kBlock, 0);
  return nb > 0 ? nb : 1;
}

cudaError_t launch_push(const DevParams& P, int grid, cudaStream_t s) {
  if (P.use_nmax) k_push<true><<<grid, kBlock, 0, s>>>(P);
  else k_push<false><<<grid, kBlock, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_inject(const DevParams& P, double carriers, float sig_e, float sig_i, cudaStream_t s) {
  k_inject<<<1, 256, 0, s>>>(P, carriers, sig_e, sig_i);
  return cudaGetLastError();
}

cudaError_t launch_field(const DevParams& P, double* E64, float* E32, double a, double cJ, double dt_jext,
                         double* fpart, int grid_push, cudaStream_t s) {
  int nfb = (P.N + 255) / 256;
  if (nfb > kMaxFieldBlocks) nfb = kMaxFieldBlocks;
  k_field<<<nfb, 256, 0, s>>>(P, E64, E32, a, cJ, fpart);
  k_finalize<<<1, 32, 0, s>>>(P, fpart, nfb, grid_push, dt_jext);
  return cudaGetLastError();
}

cudaError_t launch_sort(const DevParams& P, uint32_t* counts, long long* offsets, uint32_t* pos2, float* u2,
                        float* w2, uint8_t* sp2, uint64_t* id2, int grid, cudaStream_t s) {
  cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)P.N, s);
  k_hist<<<grid, 256, 0, s>>>(P, counts);
  k_scan<<<1, 1024, 0, s>>>(P, counts, offsets);
  k_scatter<<<grid, 256, 0, s>>>(P, offsets, pos2, u2, w2, sp2, id2);
  k_sort_done<<<1, 1, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_table(int Ng, int Ns, int n_mu, int n_phi, double log10g_max, double theta_T, double pref,
                         const double* xs, const double* bs, const double* mus, const double* gx, const double* gw,
                         int photon_model, float2* out, cudaStream_t s) {
  const int total = 2 * Ns * Ng;
  k_table<<<(total + 127) / 128, 128, 0, s>>>(Ng, Ns, n_mu, n_phi, log10g_max, theta_T, pref, xs, bs, mus, gx, gw,
                                               photon_model, out);
  return cudaGetLastError();
}

cudaError_t launch_deposit(const DevParams& P, long long n, const long long* p0, const long long* p1, const float* w,
                           const uint8_t* sp, long long* J, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_deposit<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, n, p0, p1, w, sp, J);
  return cudaGetLastError();
}

cudaError_t launch_count_species(const DevParams& P, unsigned long long* out4, cudaStream_t s) {
  cudaMemsetAsync(out4, 0, 4 * sizeof(unsigned long long), s);
  k_count_species<<<1184, 256, 0, s>>>(P, out4);
  return cudaGetLastError();
}

}  // namespace pic1d
