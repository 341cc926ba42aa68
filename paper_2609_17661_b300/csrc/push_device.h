// push_device.h -- device functions of the per-particle physics shared by the
// push kernels (kernels.cu, push_stream.cu): the counter-based generator and
// particle ids, the drag laws and the drag half-step of the Strang split, the
// RICS event kinematics, the exact warp sum of int64 values, the launch
// tallies and the 1D charge-conserving path split.
#pragma once
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
// the scattering draw's uniform on the lattice (0, 1] in steps of 2^-24 (exact
// in FP32): a lepton scatters when it is <= p_sc, so a p_sc below 2^-24 can
// never scatter and is not drawn for
__device__ __forceinline__ float unit24_open(uint32_t x) { return (float)((x >> 8) + 1u) * (1.0f / 16777216.0f); }
constexpr float kDrawMin = 0x1p-24f;

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
// id of atmosphere particle `slot` (m = 0: e-, 1: ion) topped up in `cell` at `step`
__device__ __forceinline__ unsigned long long atmo_id(long long step, int cell, long long slot, int m) {
  const unsigned long long a = mix64(((unsigned long long)step << 1) | (unsigned long long)m);
  const unsigned long long b = ((unsigned long long)(uint32_t)cell << 32) | (unsigned long long)(uint32_t)slot;
  return mix64(a ^ b ^ 0xA7305EEDull) | 0x8000000000000000ull;
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
  int j;             // table row in s/L below the particle
  float c;           // fractional position between rows j and j+1
  float x, b, mu;    // r/R*, B/B_QED, cos(radial, +s) interpolated at s
};

__device__ __forceinline__ void site_rows(const DevParams& P, uint32_t pos0, Site& S) {
  const float v = fminf((float)pos0 * P.v_scale, (float)(P.Ns - 1));
  S.j = min((int)v, P.Ns - 2);
  S.c = v - (float)S.j;
}

struct DragVal {
  float F, dF, lnN;  // F^ (per R*), dF^/du, ln N^ (per R_star/c)
};

// Bilinear table lookup in (log10 gamma, s/L).  The device copy of the table
// pairs neighbouring s-rows: tpair[(sg*(Ns-1) + j)*Ng + i] = (F[j][i], lnN[j][i],
// F[j+1][i], lnN[j+1][i]), so one lookup is two adjacent 16-byte loads.
// log10 gamma = log10(2)/2 * log2(1 + u^2): no square root is needed.
__device__ __forceinline__ DragVal table_eval(const DevParams& P, float u, int j, float c, bool want_dF) {
  const float q = fmaf(u, u, 1.0f);                    // gamma^2
  float t = fmaxf(0.5f * __log2f(q) * P.t_scale, 0.0f);
  bool top = false;
  if (t > (float)(P.Ng - 1)) { t = (float)(P.Ng - 1); top = true; }
  const int i = min((int)t, P.Ng - 2);
  const float a = t - (float)i;
  const int sg = (u >= 0.0f) ? 0 : 1;
  const float4* row = P.tpair + ((size_t)(sg * (P.Ns - 1) + j) * P.Ng);
  const float4 A = __ldg(row + i), B = __ldg(row + i + 1);
  const float ac = 1.0f - a, cc = 1.0f - c;
  DragVal d;
  d.F = ac * (cc * A.x + c * A.z) + a * (cc * B.x + c * B.z);
  d.lnN = ac * (cc * A.y + c * A.w) + a * (cc * B.y + c * B.w);
  d.dF = 0.0f;
  if (want_dF && !top) {
    const float dFdt = cc * (B.x - A.x) + c * (B.z - A.z);
    d.dF = dFdt * __fdividef(u, q) * P.dtdu_scale;
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

// TBL: the caller knows the line's law is the table with the limiter on and
// the branch-certainty table built (a push instantiated for such lines);
// otherwise these switches are read from P.
template <bool TBL = false>
__device__ __forceinline__ DragVal drag_eval(const DevParams& P, float u, const Site& S, bool want_dF) {
  if (TBL || P.drag_law == PIC1D_DRAG_TABLE) return table_eval(P, u, S.j, S.c, want_dF);
  return closed_eval(P, u, S, want_dF);
}

// One drag update over dt/2 at fixed s (Sec. 3): limiter test |F| tau_min <
// |u0|, then the implicit midpoint [Eq. implicit] u1 = u0 + (h/2)(F(u0) +
// F(u1)) by Newton's method, or exponential damping toward
// p~ = mu / sqrt(1 - mu^2).  Newton starts at u0, where the residual is
// -h F(u0): its first iterate is the linearised step u0 + h F0 / (1 - h F0'/2)
// (F0' = dF/du at u0, from the same lookup), whose error against the root is
// (h/4)|F''| (h F0)^2, below 1e-8 of u once |h F0| <= 2^-10 |u0|.  Only a
// larger change takes further iterations (up to 4; one that leaves u1
// unchanged is a fixed point and ends them).  With the limiter on, the
// Newton branch is taken only where |h F0| < (h / tau_min) |u0|, far below
// that bound, so one step is the whole update there.
template <bool TBL = false>
__device__ __forceinline__ float drag_half(const DevParams& P, const Site& S, float u0, unsigned& n_lim,
                                           unsigned& n_newt) {
  const float h = P.half_dt;
  const DragVal d0 = drag_eval<TBL>(P, u0, S, true);
  const float F0 = P.drag_k * d0.F;
  const bool newton = (!TBL && !P.limiter_on) || (fabsf(F0) * P.tau_min < fabsf(u0));
  if (newton) {
    ++n_newt;
    const float dG0 = fmaxf(1.0f - 0.5f * h * P.drag_k * d0.dF, 0.5f);
    float u1 = u0 + __fdividef(h * F0, dG0);
    if (fabsf(h * F0) > 0x1p-10f * fabsf(u0)) {
#pragma unroll 1
      for (int it = 0; it < 4; ++it) {
        const DragVal d1 = drag_eval<TBL>(P, u1, S, true);
        const float F1 = P.drag_k * d1.F;
        const float G = u1 - u0 - 0.5f * h * (F0 + F1);
        const float dG = fmaxf(1.0f - 0.5f * h * P.drag_k * d1.dF, 0.5f);
        const float un = u1 - __fdividef(G, dG);
        if (un == u1) break;
        u1 = un;
      }
    }
    return u1;
  }
  ++n_lim;
  const float ut = S.mu * rsqrtf(1.0f - S.mu * S.mu);
  return fmaf(u0 - ut, P.damp, ut);
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
// deposit helpers
// --------------------------------------------------------------------------
// exact int64 sum over the lanes of `grp` (lanes that share a key): three
// 21-bit slices, each summed by one redux (|v| < 2^62 keeps every slice sum
// inside 32 bits), recombined in 64 bits.  Order-independent and exact.
__device__ __forceinline__ long long group_sum64(unsigned grp, long long v) {
  const unsigned lo = (unsigned)(v & 0x1FFFFF);
  const unsigned mid = (unsigned)((v >> 21) & 0x1FFFFF);
  const int hi = (int)(v >> 42);
  const unsigned slo = __reduce_add_sync(grp, lo);
  const unsigned smid = __reduce_add_sync(grp, mid);
  const int shi = (int)__reduce_add_sync(grp, (unsigned)hi);
  return ((long long)shi << 42) + ((long long)smid << 21) + (long long)slo;
}

// --------------------------------------------------------------------------
// the push: one PIC cycle for every particle slot
// --------------------------------------------------------------------------
enum { C_SCAT, C_CLAMP, C_LIM, C_NEWT, C_NONFIN, C_LOSTN, C_LOSTS, C_PAIRS, C_DROP, C_REJ, C_WALL, C_DRAW, C_COUNT };

// Tallies of one push launch.  The frequent ones stay in each thread's
// registers (drag branches, a Kahan-compensated FP32 sum of w m (gamma - 1));
// rare events are counted straight into the block's shared counters, and the
// energy carried out at the walls into a shared sum, so that they hold no
// registers in the particle loop.
struct Tally {
  unsigned* sc;               // the block's counters (C_COUNT, shared memory)
  float* skl;                 // the block's lost kinetic energy (shared memory)
  unsigned n_lim, n_newt, n_draw;   // drag branches and Monte-Carlo draws, in registers
  float ke, ke_c;
};

__device__ __forceinline__ void tally(Tally& T, int k) { atomicAdd(T.sc + k, 1u); }

__device__ __forceinline__ void tally_init(Tally& T, unsigned* sc, float* skl) {
  T.sc = sc;
  T.skl = skl;
  T.n_lim = T.n_newt = T.n_draw = 0;
  T.ke = T.ke_c = 0.0f;
}

// The block's tallies into its line (block-wide; sRed holds one double per
// warp): branch counts and shared counters to the line's counters, kinetic
// energy to *ke_dst (added atomically or stored), lost energy to the line's
// state.  The tallies and shared counters start again from zero.
__device__ inline void flush_tally(const DevParams& P, Tally& T, double* sRed, double* ke_dst, bool ke_atomic) {
  const int t = threadIdx.x, lane = t & 31;
  const unsigned a = __reduce_add_sync(0xffffffffu, T.n_lim), b = __reduce_add_sync(0xffffffffu, T.n_newt);
  const unsigned c = __reduce_add_sync(0xffffffffu, T.n_draw);
  if (lane == 0) {
    if (a) atomicAdd(T.sc + C_LIM, a);
    if (b) atomicAdd(T.sc + C_NEWT, b);
    if (c) atomicAdd(T.sc + C_DRAW, c);
  }
  double ked = (double)T.ke - (double)T.ke_c;
  for (int d = 16; d > 0; d >>= 1) ked += __shfl_down_sync(0xffffffffu, ked, d);
  if (lane == 0) sRed[t >> 5] = ked;
  __syncthreads();
  if (t == 0) {
    double ke = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) ke += sRed[i];
    if (ke_atomic) atomicAdd(ke_dst, ke);
    else *ke_dst = ke;
    if (*T.skl != 0.0f) atomicAdd(&P.st->ke_lost, (double)*T.skl);
    *T.skl = 0.0f;
    Counters* C = P.ctr;
    unsigned long long* dst[C_COUNT] = {&C->scatters, &C->psc_clamped, &C->limiter_branch, &C->newton_branch,
                                        &C->nonfinite, &C->lost_north, &C->lost_south, &C->pairs_created,
                                        &C->pairs_dropped_cap, &C->pairs_rejected_nmax, &C->pairs_lost_wall,
                                        &C->rng_draws};
    for (int k = 0; k < C_COUNT; ++k) {
      if (T.sc[k]) atomicAdd(dst[k], (unsigned long long)T.sc[k]);
      T.sc[k] = 0;
    }
  }
  __syncthreads();
  T.n_lim = T.n_newt = T.n_draw = 0;
  T.ke = T.ke_c = 0.0f;
}

__device__ __forceinline__ void kahan(float& s, float& c, float x) {
  const float y = x - c, t = s + y;
  c = (t - s) - y;
  s = t;
}

// The 1D charge-conserving current of one step (Sec. 3): the signed path length
// inside each cell.  A step is shorter than a cell, so from the start cell
// only the cell itself and one neighbour receive current.  d is the
// displacement in fixed point (clamped at a wall), frac the start position
// inside its cell; sw = q_sign * w_int.
__device__ __forceinline__ void path_split(int d, uint32_t frac, int F, int sw, long long& xm, long long& x0,
                                           long long& xp) {
  const int up = (int)((1u << F) - frac), dn = (int)frac;
  int l0, lm = 0, lp = 0;
  if (d >= 0) { l0 = min(d, up); lp = d - l0; }
  else { l0 = max(d, -dn); lm = d - l0; }
  x0 = (long long)sw * l0;
  xm = (long long)sw * lm;
  xp = (long long)sw * lp;
}

// The same split as the lower cell cl of the (at most) two cells the path
// touches and the signed lengths la, lb inside cl and cl + 1.
__device__ __forceinline__ void path_lengths(int d, uint32_t frac, int F, int cell, int& cl, int& la, int& lb) {
  const bool neg = d < 0;
  const int l0 = neg ? max(d, -(int)frac) : min(d, (int)((1u << F) - frac));
  const int ln = d - l0;
  cl = cell - (neg ? 1 : 0);
  la = neg ? ln : l0;
  lb = neg ? l0 : ln;
}

// A drag half-step (drag_half) that first consults the branch-certainty
// table (table law with the limiter): where the entry of this sign, s-row
// pair and half-octave of gamma^2 is set, the limiter test would choose the
// damping branch for every momentum there (the damping update is
// drag_half's), or the Newton branch with an update too small to change u in
// FP32 (u is returned as it is), so the table lookup is skipped.
template <bool TBL = false>
__device__ __forceinline__ float drag_half_flagged(const DevParams& P, const Site& S, float u0, unsigned& n_lim,
                                                   unsigned& n_newt) {
  if (TBL || P.dflag) {
    const float q = fmaf(u0, u0, 1.0f);
    const unsigned e2 = (__float_as_uint(q) >> kDampShift) - kDampE2Base;
    if (e2 < (unsigned)kDampNE) {
      const int sg = (u0 >= 0.0f) ? 0 : 1;
      const unsigned f = __ldg(P.dflag + ((size_t)(sg * (P.Ns - 1) + S.j) * kDampNE + e2)) & 3u;
      if (f == kDampCertain) {
        ++n_lim;
        const float ut = S.mu * rsqrtf(1.0f - S.mu * S.mu);
        return fmaf(u0 - ut, P.damp, ut);
      }
      if (f == kNewtonStill) {      // drag_half's Newton step would leave u0 as it is
        ++n_newt;
        return u0;
      }
    }
  }
  return drag_half<TBL>(P, S, u0, n_lim, n_newt);
}

// ---------------------------------------------------------------------------
// current registers of a lane: cells B, B+1, B+2, taking every path whose
// lower cell is B or B+1 (a path of one step touches at most two cells)
// ---------------------------------------------------------------------------
struct JWin {
  int B;
  long long A0, A1, A2;
};

__device__ __forceinline__ void jwin_init(JWin& W) {
  W.B = -(1 << 29);
  W.A0 = W.A1 = W.A2 = 0;
}

// this lane's window into J (native 64-bit atomics; exact, order-independent)
__device__ __forceinline__ void jwin_flush_lane(JWin& W, long long* J, int N) {
  const long long a[3] = {W.A0, W.A1, W.A2};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int c = W.B + j;
    if (a[j] != 0 && c >= 0 && c < N) atomicAdd(reinterpret_cast<unsigned long long*>(J + c), (unsigned long long)a[j]);
  }
  W.A0 = W.A1 = W.A2 = 0;
}

// Warp-collective flush of every lane's window: where the windows that hold
// current lie within two neighbouring anchors (the usual case: the warp's
// particles are neighbours in the cell order), each of the four cells they
// cover gets one exact warp sum and one atomic; else every lane adds its own.
__device__ __forceinline__ void jwin_flush_warp(JWin& W, long long* J, int N) {
  const int lane = threadIdx.x & 31;
  const bool act = (W.A0 | W.A1 | W.A2) != 0;
  if (__any_sync(0xffffffffu, act)) {
    const int wmin = __reduce_min_sync(0xffffffffu, act ? W.B : (1 << 30));
    const int o = W.B - wmin;
    if (__all_sync(0xffffffffu, !act || o <= 1)) {
      const bool lo = act && o == 0, hi = act && o == 1;
      const long long v0 = lo ? W.A0 : 0;
      const long long v1 = lo ? W.A1 : (hi ? W.A0 : 0);
      const long long v2 = lo ? W.A2 : (hi ? W.A1 : 0);
      const long long v3 = hi ? W.A2 : 0;
      const long long s0 = group_sum64(0xffffffffu, v0);
      const long long s1 = group_sum64(0xffffffffu, v1);
      const long long s2 = group_sum64(0xffffffffu, v2);
      const long long s3 = group_sum64(0xffffffffu, v3);
      if (lane < 4) {
        const long long v = lane == 0 ? s0 : (lane == 1 ? s1 : (lane == 2 ? s2 : s3));
        const int c = wmin + lane;
        if (v != 0 && c >= 0 && c < N) atomicAdd(reinterpret_cast<unsigned long long*>(J + c), (unsigned long long)v);
      }
      W.A0 = W.A1 = W.A2 = 0;
    } else if (act) {
      jwin_flush_lane(W, J, N);
    }
  }
}

// one path (lower cell cl, lengths la and lb, weight sw = q_sign w_int) into
// the window; a path outside it first flushes the window (this lane's, or
// the whole warp's with WARP) and moves it to the new cell
template <bool WARP>
__device__ __forceinline__ void jwin_add(JWin& W, bool has, int cl, int la, int lb, int sw, long long* J, int N) {
  const bool need = has && (unsigned)(cl - W.B) > 1u;
  if (WARP) {
    if (__any_sync(0xffffffffu, need)) jwin_flush_warp(W, J, N);
  } else if (need) {
    jwin_flush_lane(W, J, N);
  }
  if (need) W.B = (cl > W.B) ? cl - 1 : cl;
  if (has) {
    const bool up = cl != W.B;
    const int L0 = up ? 0 : la, L1 = up ? la : lb, L2 = up ? lb : 0;
    W.A0 += (long long)sw * L0;
    W.A1 += (long long)sw * L1;
    W.A2 += (long long)sw * L2;
  }
}

}  // namespace pic1d
