// kernels.cu -- sm_103a kernels of the per-step particle loop (the default
// push, k_push_stream, is in push_stream.cu).
//
//   k_push     the per-thread pushes (variants of pic1d_set_variant): gather
//              E, Strang-split drag around the Lorentz kick (Sec. 3),
//              Monte-Carlo RICS scattering with recoil and pair creation
//              (Sec. 3, App. A), move, charge-conserving int64 deposit from
//              per-lane current registers, loss flags at the conducting
//              walls, pair append.
//   k_push_sur the push with drag law SURROGATE (the network on tcgen05).
//   k_inject / k_topup   surface supply (RATE) and the atmosphere's top-up.
//   k_field    Ampere with the external current in FP64 (Sec. 3) + totals.
//   k_finalize per-step scalars in a fixed summation order.
//   k_hist / k_scan / k_scatter   periodic cell sort (drops removed slots).
//   k_annih_scan / k_annih_cell   annihilation at n_max after a sort.
//   k_ens_*    the ensemble: many lines per launch.
//   k_table    drag/rate table by FP64 quadrature over the stellar disk
//              (Sec. 2.2, Eq. scatteringNdot and Eq. contdrag).
//
// The per-thread pushes read the particle SoA with PPT-wide loads (a thread
// owns PPT consecutive particles of a tile) and blocks take contiguous chunks
// of tiles, so that cell-sorted particles of one block fall into a narrow
// window of cells.
#include <math.h>

#include "pic1d_internal.h"
#include "push_device.h"
#include "sur_mlp.h"

namespace pic1d {

// Result of pushing one particle.
struct PushOut {
  uint32_t pos;               // new position (clamped inside the line if lost)
  float u;
  bool lost, want_pair, want_dens;
  float child_u;
  unsigned long long pid;     // id (loaded only if a Philox number was drawn)
  long long xm, x0, xp;       // signed current into cells cell-1, cell, cell+1
  int cl, la, lb, sw;         // the same path as (lower cell, lengths in cl and cl+1) and q_sign w_int
  int cD, vD;                 // cell and weight of the lepton density for the pair cap
  int cell;                   // cell at the start of the step
};

// One PIC cycle of one particle (Sec. 3): gather, Strang-split drag, kick,
// Monte-Carlo RICS, move, and the charge-conserving deposit contributions.
// Positions are u32 fixed point; every particle alive at the start of a step
// has pos < top, and a step is shorter than one cell.  ATMO adds gravity
// (inject mode TOPUP), gathered like E.
template <bool NMAX, bool ATMO = false, bool LEAN = false>
__device__ __forceinline__ PushOut push_one(const DevParams& P, uint32_t idx, uint32_t pos0, float u, float w,
                                            int sp, Tally& T) {
  const uint32_t fmask = (1u << P.F) - 1u;
  const uint32_t half = 1u << (P.F - 1);
  PushOut o;
  o.lost = false; o.want_pair = false; o.want_dens = false; o.child_u = 0.0f; o.pid = 0;
  o.xm = 0; o.x0 = 0; o.xp = 0; o.cD = 0; o.vD = 0;
  const bool ion = (sp == PIC1D_SP_ION);
  const bool lep = !ion;
  const float qm = ion ? P.qm[PIC1D_SP_ION] : (sp == PIC1D_SP_POSITRON ? 1.0f : -1.0f);
  const int qs = (sp == PIC1D_SP_ELECTRON || sp == PIC1D_SP_ATMO) ? -1 : 1;
  const float mass = ion ? P.mass[PIC1D_SP_ION] : 1.0f;
  const int cell = (int)(pos0 >> P.F);
  o.cell = cell;
  // 1. gather E linearly between cell centres (constant beyond the end centres)
  float Ep, Gp = 0.0f;
  {
    const uint32_t x = pos0 < half ? 0u : pos0 - half;
    int ig = (int)(x >> P.F);
    float f = (float)(x & fmask) * P.inv2F;
    if (ig > P.N - 2) { ig = P.N - 2; f = 1.0f; }
    const float e0 = __ldg(P.E32 + ig), e1 = __ldg(P.E32 + ig + 1);
    Ep = fmaf(f, e1 - e0, e0);
    if (ATMO) {
      const float g0 = __ldg(P.G32 + ig), g1 = __ldg(P.G32 + ig + 1);
      Gp = fmaf(f, g1 - g0, g0);
    }
  }
  const bool zone = __ldg(P.zone + cell) != 0;
  const bool cont = lep && P.drag_law != PIC1D_DRAG_OFF && (P.rics_mode == PIC1D_RICS_DRAG_PLUS_PAIRS || !zone);
  const bool mc = lep && P.mc_on && P.drag_law != PIC1D_DRAG_OFF && zone;
  Site S;
  if (cont || mc) {
    const float f = (float)(pos0 & fmask) * P.inv2F;
    const float b0 = __ldg(P.nb + cell), b1 = __ldg(P.nb + cell + 1);
    const float m0 = __ldg(P.nmu + cell), m1 = __ldg(P.nmu + cell + 1);
    S.b = fmaf(f, b1 - b0, b0);
    S.mu = fmaf(f, m1 - m0, m0);
    if (P.drag_law == PIC1D_DRAG_CLOSED) {
      const float x0 = __ldg(P.nx + cell), x1 = __ldg(P.nx + cell + 1);
      S.x = fmaf(f, x1 - x0, x0);
    } else {
      S.x = 1.0f;
    }
    site_rows(P, pos0, S);
  }
  // 2-4. Strang split: drag dt/2, Lorentz kick dt, drag dt/2
  if (cont) u = LEAN ? drag_half_flagged(P, S, u, T.n_lim, T.n_newt) : drag_half(P, S, u, T.n_lim, T.n_newt);
  if (ATMO) u = fmaf(fmaf(qm, Ep, Gp / mass), P.dt, u);
  else u = fmaf(qm * Ep, P.dt, u);
  if (cont) u = LEAN ? drag_half_flagged(P, S, u, T.n_lim, T.n_newt) : drag_half(P, S, u, T.n_lim, T.n_newt);
  // 5. Monte-Carlo RICS in the pair zone
  bool make_pair = false;
  float Pg = 0.0f;
  if (mc) {
    const DragVal dv = drag_eval(P, u, S, false);
    float psc = P.drag_k * expf(dv.lnN) * P.dt;
    if (psc > 1.0f) { psc = 1.0f; tally(T, C_CLAMP); }
    if (psc >= kDrawMin) {
      ++T.n_draw;
      o.pid = P.id[idx];
      const uint4 r = philox4x32_10(
          make_uint4((uint32_t)o.pid, (uint32_t)(o.pid >> 32), (uint32_t)P.step, kTagRics), P.key0, P.key1);
      if (unit24_open(r.x) <= psc) {
        tally(T, C_SCAT);
        const float beta = u * rsqrtf(fmaf(u, u, 1.0f));
        const float d = (S.mu > beta) ? 1.0f : -1.0f;
        const float ct = dipole_cos(unit24(r.y));
        float uf, Eg;
        rics_event(S.b, d, u, ct, uf, Eg, Pg);
        if (P.rics_mode == PIC1D_RICS_SPLIT) u = uf;
        if (P.pairs_on && Eg >= P.pair_e_thr) make_pair = true;
      }
    }
  }
  // 6. move: ds = dt u / gamma, rounded to the fixed-point quantum
  const int wint = __float2int_rn(w * 4096.0f);
  const int sw0 = qs * wint;
  if (!isfinite(u)) {
    // removed in place: no current, counted (the step reports PIC1D_ENUMERIC)
    tally(T, C_NONFIN);
    o.u = 0.0f;
    o.pos = pos0;
    o.lost = true;
    o.cl = cell; o.la = 0; o.lb = 0; o.sw = 0;
    return o;
  }
  const float q = fmaf(u, u, 1.0f);
  const float r = rsqrtf(q);                                   // 1 / gamma
  const int dfix = __float2int_rn(P.dt * (u * r) * (float)(1u << P.F));
  const float e = w * mass * __fdividef(u * u * r, 1.0f + r);  // w m (gamma - 1)
  const bool lostN = dfix < 0 && (uint32_t)(-dfix) > pos0;
  const bool lostS = dfix > 0 && (uint32_t)dfix > P.top1 - pos0;
  o.lost = lostN || lostS;
  kahan(T.ke, T.ke_c, o.lost ? 0.0f : e);
  if (o.lost) atomicAdd(T.skl, e);
  // 7. charge-conserving deposit: signed length of the path inside each cell
  uint32_t p1;
  if (!o.lost) {
    p1 = pos0 + (uint32_t)dfix;
    path_split(dfix, pos0 & fmask, P.F, sw0, o.xm, o.x0, o.xp);
    path_lengths(dfix, pos0 & fmask, P.F, cell, o.cl, o.la, o.lb);
    o.sw = sw0;
    o.pos = p1;
    if (NMAX && lep) {
      o.cD = (int)(p1 >> P.F);
      o.vD = wint;
      o.want_dens = __ldg(P.dens_flag + o.cD) != 0;
    }
  } else {
    // leaves through a wall: the path is clamped at the conductor (64-bit: the
    // southern wall sits at top, which may be 2^32)
    tally(T, lostN ? C_LOSTN : C_LOSTS);
    // the path ends at the wall: to node 0 from cell 0, or to node N from cell N-1
    const int d = lostN ? -(int)pos0 : (int)(P.top - (long long)pos0);
    path_split(d, pos0 & fmask, P.F, sw0, o.xm, o.x0, o.xp);
    path_lengths(d, pos0 & fmask, P.F, cell, o.cl, o.la, o.lb);
    o.sw = sw0;
    o.pos = lostN ? 0u : (uint32_t)(P.top - 1);
    if (make_pair) tally(T, C_WALL);     // the parent left the line: no pair
    make_pair = false;
  }
  o.u = u;
  if (make_pair) {
    if (NMAX && P.dens_cur[(int)(o.pos >> P.F)] >= P.nmax_int) {
      tally(T, C_REJ);
    } else {
      o.want_pair = true;
      o.child_u = 0.5f * Pg;
    }
  }
  return o;
}

// The same PIC cycle for a particle in a "fast" cell (no pair zone within two
// cells, not next to a wall): gather, continuous drag for leptons, kick,
// move, deposit.  A particle there cannot leave the line in one step.  It
// must give bit-for-bit what push_one gives for the same particle.
template <bool LEAN = false>
__device__ __forceinline__ void push_fast(const DevParams& P, uint32_t pos0, float u, float w, int sp, Tally& T,
                                          PushOut& o) {
  const uint32_t fmask = (1u << P.F) - 1u;
  const uint32_t half = 1u << (P.F - 1);
  const bool ion = (sp == PIC1D_SP_ION);
  const float qm = ion ? P.qm[PIC1D_SP_ION] : (sp == PIC1D_SP_POSITRON ? 1.0f : -1.0f);
  const int qs = (sp == PIC1D_SP_ELECTRON || sp == PIC1D_SP_ATMO) ? -1 : 1;
  const float mass = ion ? P.mass[PIC1D_SP_ION] : 1.0f;
  const int cell = (int)(pos0 >> P.F);
  o.cell = cell;
  o.lost = false;
  o.want_pair = false;
  o.want_dens = false;
  o.xm = o.x0 = o.xp = 0;
  float Ep;
  {
    const uint32_t x = pos0 - half;          // pos0 >= 2^F here: cell >= 1
    int ig = (int)(x >> P.F);
    float f = (float)(x & fmask) * P.inv2F;
    if (ig > P.N - 2) { ig = P.N - 2; f = 1.0f; }
    const float e0 = __ldg(P.E32 + ig), e1 = __ldg(P.E32 + ig + 1);
    Ep = fmaf(f, e1 - e0, e0);
  }
  if (!ion && P.drag_law != PIC1D_DRAG_OFF) {
    Site S;
    const float f = (float)(pos0 & fmask) * P.inv2F;
    const float m0 = __ldg(P.nmu + cell), m1 = __ldg(P.nmu + cell + 1);
    S.mu = fmaf(f, m1 - m0, m0);
    if (P.drag_law == PIC1D_DRAG_CLOSED) {
      const float b0 = __ldg(P.nb + cell), b1 = __ldg(P.nb + cell + 1);
      const float x0 = __ldg(P.nx + cell), x1 = __ldg(P.nx + cell + 1);
      S.b = fmaf(f, b1 - b0, b0);
      S.x = fmaf(f, x1 - x0, x0);
    } else {
      S.b = 0.0f;
      S.x = 1.0f;
    }
    site_rows(P, pos0, S);
    u = LEAN ? drag_half_flagged(P, S, u, T.n_lim, T.n_newt) : drag_half(P, S, u, T.n_lim, T.n_newt);
    u = fmaf(qm * Ep, P.dt, u);
    u = LEAN ? drag_half_flagged(P, S, u, T.n_lim, T.n_newt) : drag_half(P, S, u, T.n_lim, T.n_newt);
  } else {
    u = fmaf(qm * Ep, P.dt, u);
  }
  if (!isfinite(u)) {
    tally(T, C_NONFIN);
    o.u = 0.0f;
    o.pos = pos0;
    o.lost = true;
    o.cl = cell; o.la = 0; o.lb = 0; o.sw = 0;
    return;
  }
  const float q = fmaf(u, u, 1.0f);
  const float r = rsqrtf(q);
  const int dfix = __float2int_rn(P.dt * (u * r) * (float)(1u << P.F));
  kahan(T.ke, T.ke_c, w * mass * __fdividef(u * u * r, 1.0f + r));
  const uint32_t p1 = pos0 + (uint32_t)dfix;
  o.sw = qs * __float2int_rn(w * 4096.0f);
  path_split(dfix, pos0 & fmask, P.F, o.sw, o.xm, o.x0, o.xp);
  path_lengths(dfix, pos0 & fmask, P.F, cell, o.cl, o.la, o.lb);
  o.pos = p1;
  o.u = u;
}

template <int PPT> struct Vec;
template <> struct Vec<1> { using U = uint32_t; using F = float; using B = uint8_t; };
template <> struct Vec<2> { using U = uint2; using F = float2; using B = uchar2; };

__device__ __forceinline__ void unpack_u(uint32_t v, uint32_t (&a)[1]) { a[0] = v; }
__device__ __forceinline__ void unpack_u(uint2 v, uint32_t (&a)[2]) { a[0] = v.x; a[1] = v.y; }
__device__ __forceinline__ void unpack_f(float v, float (&a)[1]) { a[0] = v; }
__device__ __forceinline__ void unpack_f(float2 v, float (&a)[2]) { a[0] = v.x; a[1] = v.y; }
__device__ __forceinline__ void unpack_b(uint8_t v, uint8_t (&a)[1]) { a[0] = v; }
__device__ __forceinline__ void unpack_b(uchar2 v, uint8_t (&a)[2]) { a[0] = v.x; a[1] = v.y; }
__device__ __forceinline__ uint32_t pack_u(const uint32_t (&a)[1]) { return a[0]; }
__device__ __forceinline__ uint2 pack_u(const uint32_t (&a)[2]) { return make_uint2(a[0], a[1]); }
__device__ __forceinline__ float pack_f(const float (&a)[1]) { return a[0]; }
__device__ __forceinline__ float2 pack_f(const float (&a)[2]) { return make_float2(a[0], a[1]); }

// a lane's current registers (cells c_ref-1, c_ref, c_ref+1) to global memory
// (native 64-bit atomics; exact and order-independent), then cleared
__device__ __forceinline__ void flush_lane(long long (&a)[3], int c_ref, long long* J, int N) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int c = c_ref - 1 + j;
    if (a[j] != 0 && c >= 0 && c < N) atomicAdd(reinterpret_cast<unsigned long long*>(J + c), (unsigned long long)a[j]);
    a[j] = 0;
  }
}

// shared-memory window add; the thread records the window range it touched
// in two registers (lo, hi), reduced once per chunk
__device__ __forceinline__ void win_add(long long* sWin, int win_lo, int& lo, int& hi, long long* g, int N, int cell,
                                        long long v) {
  if (v == 0 || cell < 0 || cell >= N) return;
  const int o = cell - win_lo;
  if (o >= 0 && o < kWindow) {
    atomicAdd(reinterpret_cast<unsigned long long*>(sWin + o), (unsigned long long)v);
    lo = min(lo, o);
    hi = max(hi, o);
  } else {
    atomicAdd(reinterpret_cast<unsigned long long*>(g + cell), (unsigned long long)v);
  }
}

// flush the touched part [s_rng[0], s_rng[1]] of a shared window to global
// memory and clear it
__device__ __forceinline__ void window_drain(long long* sWin, int win_lo, const int* s_rng, long long* g, int N) {
  const int lo = s_rng[0], hi = s_rng[1];
  for (int i = lo + (int)threadIdx.x; i <= hi; i += kBlock) {
    const long long v = sWin[i];
    if (v) {
      const int c = win_lo + i;
      if (c < N) atomicAdd(reinterpret_cast<unsigned long long*>(g + c), (unsigned long long)v);
      sWin[i] = 0;
    }
  }
}

// The per-thread push.  A thread owns PPT consecutive particles per tile (one
// PPT-wide access per SoA array); blocks take chunks of kChunkTiles tiles
// (kBlock * PPT particles each) from a global counter, so that expensive
// regions of the line (pair zones, dense footpoints) are shared by all SMs.
// A lane's current goes into int64 registers for three cells (c_ref-1 ..
// c_ref+1; with LEAN the two-anchor window JWin) that persist across its
// particles and are added to J with 64-bit atomics, by that lane alone, when
// a path falls outside them (exact and order-independent).  The lepton
// density of the pair cap is summed per warp in a warp-uniform pending
// register while the warp's contributions stay in one cell, else through a
// shared-memory cell window anchored at each chunk's first particle and
// drained to global memory at the end of the chunk.  Slot indices are 32-bit
// (capacity < 2^31).  ATMO (inject mode TOPUP): gravity, and the plasma
// weight of each atmosphere cell after the move, summed into P.atmo_w (the
// atmosphere and the two cells around it are never fast cells, so every
// particle that ends a step there goes through push_one).
template <int PPT, int MINB, bool NMAX, bool ATMO = false, bool LEAN = false>
__global__ void __launch_bounds__(kBlock, MINB) k_push(DevParams P) {
  using VU = typename Vec<PPT>::U;
  using VF = typename Vec<PPT>::F;
  using VB = typename Vec<PPT>::B;
  constexpr int TILE = kBlock * PPT;
  __shared__ long long sD[NMAX ? kWindow : 1];
  __shared__ int s_rngD[2];
  __shared__ unsigned s_chunk;
  __shared__ int s_anchor;
  __shared__ unsigned sCtr[C_COUNT];
  __shared__ double sRed[2][kBlock / 32];

  const uint32_t n = (uint32_t)P.st->n_slots;
  const int lane = threadIdx.x & 31;

  __shared__ float sKl;
  if (NMAX)
    for (int i = threadIdx.x; i < kWindow; i += kBlock) sD[i] = 0;
  if (threadIdx.x < C_COUNT) sCtr[threadIdx.x] = 0;
  if (threadIdx.x == 0) sKl = 0.0f;
  if (threadIdx.x == 0) {
    s_rngD[0] = kWindow;
    s_rngD[1] = -1;
    s_chunk = (unsigned)atomicAdd(&P.st->work, 1ull);
  }
  __syncthreads();

  Tally T;
  tally_init(T, sCtr, &sKl);
  long long aJ[3] = {0, 0, 0};
  int c_ref = -4;
  JWin Wn;                       // LEAN: the two-anchor current window
  jwin_init(Wn);
  int dlo = kWindow, dhi = -1;   // density window range this thread touched
  // warp-uniform pending lepton density (pair cap)
  int dcell = -1;
  long long dsum = 0;

  // a chunk is split among the warps: warp w walks its own contiguous eighth
  // of the chunk, 32 * PPT particles per step of its loop, so a lane's
  // consecutive particles are neighbours in the cell order
  constexpr uint32_t CHUNK = (uint32_t)kChunkTiles * TILE;
  constexpr uint32_t WSPAN = CHUNK / (kBlock / 32);
  constexpr uint32_t WSTEP = 32u * PPT;
  const uint32_t nchunks_w = (n + CHUNK - 1) / CHUNK;
  unsigned chunk = s_chunk;
  while (chunk < nchunks_w) {
    if (threadIdx.x == 0) {
      const int c = (int)(P.pos[(size_t)chunk * CHUNK] >> P.F);
      s_anchor = max(0, min(c, P.N - 1) - kWindow / 8);
    }
    __syncthreads();
    const int win_lo = s_anchor;
    const uint32_t wbase = chunk * CHUNK + (threadIdx.x >> 5) * WSPAN + (uint32_t)lane * PPT;
    const uint32_t t1 = WSPAN / WSTEP;

    VU npos{};
    VF nu{}, nw{};
    VB nsp{};
    // loads are guarded: a chunk may run past the last slot by up to a chunk,
    // beyond the arrays' slack (the arrays have >= PPT slots past n)
    if (wbase < n) {
      npos = __ldcs(reinterpret_cast<const VU*>(P.pos + wbase));
      nu = __ldcs(reinterpret_cast<const VF*>(P.u + wbase));
      nw = __ldcs(reinterpret_cast<const VF*>(P.w + wbase));
      nsp = *reinterpret_cast<const VB*>(P.sp + wbase);
    }
    for (uint32_t t = 0; t < t1; ++t) {
      const uint32_t base = wbase + t * WSTEP;
      uint32_t pp[PPT];
      float uu[PPT], ww[PPT];
      uint8_t ss[PPT];
      unpack_u(npos, pp);
      unpack_f(nu, uu);
      unpack_f(nw, ww);
      unpack_b(nsp, ss);
      if (t + 1 < t1 && base + WSTEP < n) {
        const uint32_t b1 = base + WSTEP;
        npos = __ldcs(reinterpret_cast<const VU*>(P.pos + b1));
        nu = __ldcs(reinterpret_cast<const VF*>(P.u + b1));
        nw = __ldcs(reinterpret_cast<const VF*>(P.w + b1));
        nsp = *reinterpret_cast<const VB*>(P.sp + b1);
      }
      bool dirty = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const uint32_t idx = base + k;
        const bool valid = (idx < n) && (ss[k] != PIC1D_SP_DEAD);
        PushOut o;
        // warp-uniform fast path: every lane's particle sits in a cell at least
        // two cells away from any pair zone and from the walls
        const bool fast = !valid || __ldg(P.fast_cell + (pp[k] >> P.F)) != 0;
        if (__all_sync(0xffffffffu, fast)) {
          if (valid) push_fast<LEAN>(P, pp[k], uu[k], ww[k], ss[k] & 3, T, o);
        } else {
          o.want_pair = false;
          o.want_dens = false;
          if (valid) o = push_one<NMAX, ATMO, LEAN>(P, idx, pp[k], uu[k], ww[k], ss[k] & 3, T);
          // plasma weight of the atmosphere cells after the move
          if (ATMO) {
            const bool ma = valid && !o.lost && __ldg(P.atmo_flag + (o.pos >> P.F)) != 0;
            const unsigned am = __ballot_sync(0xffffffffu, ma);
            if (ma) {
              const int ac = (int)(o.pos >> P.F);
              const unsigned grp = __match_any_sync(am, ac);
              const long long sum = group_sum64(grp, (long long)__float2int_rn(ww[k] * 4096.0f));
              if (lane == __ffs(grp) - 1)
                atomicAdd(reinterpret_cast<unsigned long long*>(P.atmo_w + ac), (unsigned long long)sum);
            }
          }
          // lepton density for the pair cap: only cells where a pair can be tested
          if (NMAX) {
            const unsigned md = __ballot_sync(0xffffffffu, o.want_dens);
            if (md) {
              const int c0 = __shfl_sync(0xffffffffu, o.cD, __ffs(md) - 1);
              if (__all_sync(0xffffffffu, !o.want_dens || o.cD == c0)) {
                long long sd = 0;
                if (o.want_dens) sd = group_sum64(md, (long long)o.vD);
                sd = __shfl_sync(0xffffffffu, sd, __ffs(md) - 1);
                if (c0 != dcell) {
                  if (lane == 0 && dcell >= 0) win_add(sD, win_lo, dlo, dhi, P.dens_next, P.N, dcell, dsum);
                  dcell = c0;
                  dsum = 0;
                }
                dsum += sd;
              } else if (o.want_dens) {
                const unsigned grp = __match_any_sync(md, o.cD);
                const long long sum = group_sum64(grp, (long long)o.vD);
                if (lane == __ffs(grp) - 1) win_add(sD, win_lo, dlo, dhi, P.dens_next, P.N, o.cD, sum);
              }
            }
          }
          // pair append, warp-aggregated
          const unsigned m = __ballot_sync(0xffffffffu, o.want_pair);
          if (m) {
            const int leader = __ffs(m) - 1;
            long long slot0 = 0;
            if (lane == leader) slot0 = atomicAdd(reinterpret_cast<unsigned long long*>(&P.st->append),
                                                  (unsigned long long)(2 * __popc(m)));
            slot0 = __shfl_sync(0xffffffffu, slot0, leader);
            if (o.want_pair) {
              const long long dst = (long long)n + slot0 + 2ll * __popc(m & lanemask_lt());
              if (dst + 2 > P.cap) {
                tally(T, C_DROP);
              } else {
                tally(T, C_PAIRS);
#pragma unroll
                for (int mm = 0; mm < 2; ++mm) {
                  P.pos[dst + mm] = o.pos;
                  P.u[dst + mm] = o.child_u;
                  P.w[dst + mm] = ww[k];
                  P.sp[dst + mm] = (mm == 0) ? PIC1D_SP_ELECTRON : PIC1D_SP_POSITRON;
                  P.id[dst + mm] = pair_child_id(o.pid, P.step, mm);
                }
                if (NMAX && __ldg(P.dens_flag + (o.pos >> P.F)))
                  atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + (int)(o.pos >> P.F)),
                            (unsigned long long)(2ll * __float2int_rn(ww[k] * 4096.0f)));
              }
            }
          }
        }
        if (valid) {
          pp[k] = o.pos;
          uu[k] = o.u;
          if (o.lost) { ss[k] = PIC1D_SP_DEAD; dirty = true; }
          // current into the lane's registers for cells c_ref-1 .. c_ref+1; when
          // the lane's start cell changes, the registers go to global memory
          // (LEAN: the window of two anchors, flushed only when a path leaves it)
          if (LEAN) {
            jwin_add<false>(Wn, true, o.cl, o.la, o.lb, o.sw, P.J, P.N);
          } else {
            if (o.cell != c_ref) {
              flush_lane(aJ, c_ref, P.J, P.N);
              c_ref = o.cell;
            }
            aJ[0] += o.xm;
            aJ[1] += o.x0;
            aJ[2] += o.xp;
          }
        }
      }
      // write back (streaming stores: the data is not re-read in this kernel)
      if (base + PPT <= n) {
        __stcs(reinterpret_cast<VU*>(P.pos + base), pack_u(pp));
        __stcs(reinterpret_cast<VF*>(P.u + base), pack_f(uu));
      } else {
#pragma unroll
        for (int k = 0; k < PPT; ++k)
          if (base + k < n) { P.pos[base + k] = pp[k]; P.u[base + k] = uu[k]; }
      }
      if (dirty) {
#pragma unroll
        for (int k = 0; k < PPT; ++k)
          if (base + k < n && ss[k] == PIC1D_SP_DEAD) P.sp[base + k] = PIC1D_SP_DEAD;
      }
    }
    // end of the chunk: everything pending goes to the window, the window's
    // touched range to global memory, and the next chunk is taken
    if (LEAN) jwin_flush_lane(Wn, P.J, P.N);
    else flush_lane(aJ, c_ref, P.J, P.N);
    c_ref = -4;
    if (NMAX) {
      if (lane == 0 && dcell >= 0) win_add(sD, win_lo, dlo, dhi, P.dens_next, P.N, dcell, dsum);
      dcell = -1;
      dsum = 0;
    }
    if (NMAX) {
      // the density window range touched by the block in this chunk
      const int c = __reduce_min_sync(0xffffffffu, dlo), d = __reduce_max_sync(0xffffffffu, dhi);
      if (lane == 0 && d >= 0) { atomicMin(&s_rngD[0], c); atomicMax(&s_rngD[1], d); }
      dlo = kWindow;
      dhi = -1;
    }
    __syncthreads();
    if (NMAX) window_drain(sD, win_lo, s_rngD, P.dens_next, P.N);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_rngD[0] = kWindow;
      s_rngD[1] = -1;
      s_chunk = (unsigned)atomicAdd(&P.st->work, 1ull);
    }
    __syncthreads();
    chunk = s_chunk;
  }

  // counters and energy totals of the block
  flush_tally(P, T, sRed[0], P.ke_partial + blockIdx.x, false);
}

// --------------------------------------------------------------------------
// the push with drag law SURROGATE: the drag and the scattering rate come
// from the learned network, evaluated for the CTA's 128 particles at once on
// the tensor cores (sur_mlp.h).  One particle per thread; tiles of 128 slots
// from the dynamic schedule.  The per-particle physics is push_one's; the
// Newton iterations of the implicit midpoint run in lockstep over the CTA
// (a lane that has converged contributes a dummy row).
// --------------------------------------------------------------------------

// ln N^ along one photon direction mu (the closed form [contdrag] with solid
// angle pi/x^2) in log form, and its derivative in u:
//   ln N = ln(P/x^2) + 2 ln eps - ln gamma - ln(e^y - 1)
__device__ __forceinline__ float sur_lnrad(const DevParams& P, float u, float gam, float x, float b, float mu,
                                           float& dln) {
  const float au = fabsf(u);
  const float sm = (u >= 0.0f) ? mu : -mu;
  const float D = (1.0f - sm) + sm / (gam * (gam + au));     // 1 - beta mu
  const float eps = b / (gam * D), y = eps / P.theta_T;
  const float lnem1 = (y > 20.0f) ? y + log1pf(-__expf(-y)) : logf(expm1f(y));
  const float dlng = u / (gam * gam);
  const float dlnD = (-mu / (gam * gam * gam)) / D;
  const float dlne = -dlng - dlnD;
  dln = (2.0f - y / (-expm1f(-y))) * dlne - dlng;
  return P.sur_lnP - 2.0f * logf(x) + 2.0f * logf(eps) - logf(gam) - lnem1;
}

// F^ (per R_star), dF^/du and ln N^ of the surrogate at u for this thread's
// particle.  Collective: every thread of the CTA calls it; `want` only says
// whether the caller uses the result.  Outside the training box (gamma above
// 10^G, b outside the range of f2) the line's quadrature table stands in (the
// table law's lookup), or the closed form where a line has no table.
__device__ DragVal sur_eval(const DevParams& P, sur::MlpCta& M, float u, const Site& S, float sL, bool want,
                           bool with_dF) {
  const float q = fmaf(u, u, 1.0f);
  const float gam = sqrtf(q);
  float x[4];
  x[0] = 2.0f * (0.5f * __log2f(q) * 0.30102999566f) / P.sur_G - 1.0f;
  x[1] = 2.0f * sL - 1.0f;
  x[2] = (log10f(S.b) - (float)sur::B_MID) / (float)sur::B_HALF;
  x[3] = (u < 0.0f) ? -1.0f : 1.0f;
  const bool inbox = x[0] <= 1.0f && x[2] >= -1.0f && x[2] <= 1.0f;
  if (!want || !inbox) { x[0] = 0.0f; x[1] = 0.0f; x[2] = 0.0f; }
  float y0, y1, g0, g1;
  sur::mlp_tile(M, x, y0, y1, g0, g1, with_dF);
  DragVal d;
  d.F = d.dF = 0.0f;
  d.lnN = -700.0f;
  if (!want) return d;
  if (!inbox) return P.tpair ? table_eval(P, u, S.j, S.c, with_dF) : closed_eval(P, u, S, with_dF);
  float d1, d2;
  const float l1 = sur_lnrad(P, u, gam, S.x, S.b, S.mu, d1);
  const float ths = acosf(fmaxf(-1.0f, fminf(1.0f, S.mu))), am = asinf(fminf(1.0f, 1.0f / S.x));
  const float me = (u >= 0.0f) ? cosf(fminf(3.14159265f, ths + am)) : cosf(fmaxf(0.0f, ths - am));
  const float l2 = sur_lnrad(P, u, gam, S.x, S.b, me, d2);
  const float a1 = -0.105360516f + l1, a2 = -2.302585093f + l2;   // ln 0.9, ln 0.1
  const float mx = fmaxf(a1, a2);
  const float e1 = __expf(a1 - mx), e2 = __expf(a2 - mx);
  const float B = mx + logf(e1 + e2);
  const float dB = (e1 * d1 + e2 * d2) / (e1 + e2);
  const float Bc = fmaxf(B, sur::LT), dBc = (B > sur::LT) ? dB : 0.0f;
  d.lnN = Bc + y1;
  const float N = __expf(d.lnN);
  d.F = gam * S.b * N * y0;
  if (with_dF) {
    const float df0 = 2.0f / P.sur_G * u / (q * 2.302585093f);
    const float dln = dBc + g1 * df0;
    d.dF = S.b * N * ((u / gam) * y0 + gam * y0 * dln + gam * g0 * df0);
  }
  return d;
}

// One drag update over dt/2 (as drag_half) with the surrogate; collective.
__device__ float sur_drag_half(const DevParams& P, sur::MlpCta& M, const Site& S, float sL, float u0, bool act,
                               unsigned& n_lim, unsigned& n_newt) {
  const float h = P.half_dt;
  const float F0 = P.drag_k * sur_eval(P, M, u0, S, sL, act, false).F;
  const bool newton = act && (!P.limiter_on || (fabsf(F0) * P.tau_min < fabsf(u0)));
  float u1 = u0;
  if (act) {
    if (newton) {
      ++n_newt;
      u1 = fmaf(h, F0, u0);
    } else {
      ++n_lim;
      const float ut = S.mu * rsqrtf(1.0f - S.mu * S.mu);
      u1 = fmaf(u0 - ut, P.damp, ut);
    }
  }
  bool going = newton;
  int it = 0;
  while (__syncthreads_or(going)) {
    const DragVal d1 = sur_eval(P, M, u1, S, sL, going, true);
    if (going) {
      const float F1 = P.drag_k * d1.F;
      const float G = u1 - u0 - 0.5f * h * (F0 + F1);
      const float dG = fmaxf(1.0f - 0.5f * h * P.drag_k * d1.dF, 0.5f);
      const float un = u1 - __fdividef(G, dG);
      if (un == u1) {
        going = false;
      } else {
        u1 = un;
        if (++it == 4) going = false;
      }
    }
  }
  return u1;
}

// warp-aggregated exact add of v into g[cell] from the lanes with `mine`
__device__ __forceinline__ void warp_atomic_cell(bool mine, int cell, long long v, long long* g, int N) {
  const unsigned m = __ballot_sync(0xffffffffu, mine);
  if (!mine) return;
  const unsigned grp = __match_any_sync(m, cell);
  const long long sum = group_sum64(grp, v);
  if ((int)(threadIdx.x & 31) == __ffs(grp) - 1 && sum != 0 && cell >= 0 && cell < N)
    atomicAdd(reinterpret_cast<unsigned long long*>(g + cell), (unsigned long long)sum);
}

// One tile of 128 slots of the surrogate push (collective over the CTA):
// slots tile*128 .. tile*128+127 of P's line, n slots in use.
template <bool NMAX>
__device__ void sur_tile(const DevParams& P, sur::MlpCta& M, uint32_t tile, uint32_t n, Tally& T) {
  const int t = threadIdx.x, lane = t & 31;
  const uint32_t fmask = (1u << P.F) - 1u;
  const uint32_t half = 1u << (P.F - 1);
  const uint32_t idx = tile * sur::TM + t;
  uint32_t pos0 = 0;
  float u = 0.0f, w = 0.0f;
  uint8_t spb = PIC1D_SP_DEAD;
  if (idx < n) {
    pos0 = P.pos[idx];
    u = P.u[idx];
    w = P.w[idx];
    spb = P.sp[idx];
  }
  const bool valid = idx < n && spb != PIC1D_SP_DEAD;
  const int sp = spb & 3;
  const bool ion = (sp == PIC1D_SP_ION), lep = !ion;
  const float qm = ion ? P.qm[PIC1D_SP_ION] : (sp == PIC1D_SP_POSITRON ? 1.0f : -1.0f);
  const int qs = (sp == PIC1D_SP_ELECTRON || sp == PIC1D_SP_ATMO) ? -1 : 1;
  const float mass = ion ? P.mass[PIC1D_SP_ION] : 1.0f;
  const int cell = valid ? (int)(pos0 >> P.F) : 0;
  float Ep = 0.0f, Gp = 0.0f;
  Site S;
  S.x = 1.0f; S.b = 1.0f; S.mu = 0.0f; S.j = 0; S.c = 0.0f;
  bool zone = false;
  if (valid) {
    const uint32_t xg = pos0 < half ? 0u : pos0 - half;
    int ig = (int)(xg >> P.F);
    float fg = (float)(xg & fmask) * P.inv2F;
    if (ig > P.N - 2) { ig = P.N - 2; fg = 1.0f; }
    const float e0 = __ldg(P.E32 + ig), e1 = __ldg(P.E32 + ig + 1);
    Ep = fmaf(fg, e1 - e0, e0);
    if (P.G32) {            // the atmosphere's gravity (inject mode TOPUP), gathered like E
      const float g0 = __ldg(P.G32 + ig), g1 = __ldg(P.G32 + ig + 1);
      Gp = fmaf(fg, g1 - g0, g0);
    }
    zone = __ldg(P.zone + cell) != 0;
    const float f = (float)(pos0 & fmask) * P.inv2F;
    S.b = fmaf(f, __ldg(P.nb + cell + 1) - __ldg(P.nb + cell), __ldg(P.nb + cell));
    S.mu = fmaf(f, __ldg(P.nmu + cell + 1) - __ldg(P.nmu + cell), __ldg(P.nmu + cell));
    S.x = fmaf(f, __ldg(P.nx + cell + 1) - __ldg(P.nx + cell), __ldg(P.nx + cell));
    site_rows(P, pos0, S);
  }
  const bool cont = valid && lep && (P.rics_mode == PIC1D_RICS_DRAG_PLUS_PAIRS || !zone);
  const bool mc = valid && lep && P.mc_on && zone;
  const float sL = (float)((double)pos0 / (double)P.top);
  // 2-4. Strang split with the surrogate drag
  u = sur_drag_half(P, M, S, sL, u, cont, T.n_lim, T.n_newt);
  if (valid) u = P.G32 ? fmaf(fmaf(qm, Ep, Gp / mass), P.dt, u) : fmaf(qm * Ep, P.dt, u);
  u = sur_drag_half(P, M, S, sL, u, cont, T.n_lim, T.n_newt);
  // 5. Monte-Carlo RICS in the pair zone
  bool make_pair = false;
  float Pg = 0.0f;
  unsigned long long pid = 0;
  if (__syncthreads_or(mc)) {
    const DragVal dv = sur_eval(P, M, u, S, sL, mc, false);
    if (mc) {
      float psc = P.drag_k * expf(dv.lnN) * P.dt;
      if (psc > 1.0f) { psc = 1.0f; tally(T, C_CLAMP); }
      if (psc >= kDrawMin) {
        ++T.n_draw;
        pid = P.id[idx];
        const uint4 r = philox4x32_10(
            make_uint4((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)P.step, kTagRics), P.key0, P.key1);
        if (unit24_open(r.x) <= psc) {
          tally(T, C_SCAT);
          const float beta = u * rsqrtf(fmaf(u, u, 1.0f));
          const float d = (S.mu > beta) ? 1.0f : -1.0f;
          const float ct = dipole_cos(unit24(r.y));
          float uf, Eg;
          rics_event(S.b, d, u, ct, uf, Eg, Pg);
          if (P.rics_mode == PIC1D_RICS_SPLIT) u = uf;
          if (P.pairs_on && Eg >= P.pair_e_thr) make_pair = true;
        }
      }
    }
  }
  // 6. move, 7. deposit
  long long xm = 0, x0 = 0, xp = 0;
  uint32_t p1 = pos0;
  bool lost = false;
  const int wint = __float2int_rn(w * 4096.0f);
  if (valid) {
    if (!isfinite(u)) {
      tally(T, C_NONFIN);
      u = 0.0f;
      lost = true;
      make_pair = false;
    } else {
      const float q = fmaf(u, u, 1.0f);
      const float r = rsqrtf(q);
      const int dfix = __float2int_rn(P.dt * (u * r) * (float)(1u << P.F));
      const float e = w * mass * __fdividef(u * u * r, 1.0f + r);
      const bool lostN = dfix < 0 && (uint32_t)(-dfix) > pos0;
      const bool lostS = dfix > 0 && (uint32_t)dfix > P.top1 - pos0;
      lost = lostN || lostS;
      kahan(T.ke, T.ke_c, lost ? 0.0f : e);
      if (lost) atomicAdd(T.skl, e);
      if (!lost) {
        p1 = pos0 + (uint32_t)dfix;
        path_split(dfix, pos0 & fmask, P.F, qs * wint, xm, x0, xp);
      } else {
        tally(T, lostN ? C_LOSTN : C_LOSTS);
        const int dd = lostN ? -(int)pos0 : (int)(P.top - (long long)pos0);
        path_split(dd, pos0 & fmask, P.F, qs * wint, xm, x0, xp);
        p1 = lostN ? 0u : (uint32_t)(P.top - 1);
        if (make_pair) tally(T, C_WALL);
        make_pair = false;
      }
    }
  }
  if (make_pair) {
    if (NMAX && P.dens_cur[(int)(p1 >> P.F)] >= P.nmax_int) {
      tally(T, C_REJ);
      make_pair = false;
    }
  }
  warp_atomic_cell(xm != 0, cell - 1, xm, P.J, P.N);
  warp_atomic_cell(x0 != 0, cell, x0, P.J, P.N);
  warp_atomic_cell(xp != 0, cell + 1, xp, P.J, P.N);
  if (NMAX) {
    const int cD = (int)(p1 >> P.F);
    const bool wd = valid && lep && !lost && __ldg(P.dens_flag + cD) != 0;
    warp_atomic_cell(wd, cD, (long long)wint, P.dens_next, P.N);
  }
  if (P.G32) {
    // plasma weight of the atmosphere cells after the move (every species)
    const int ca = (int)(p1 >> P.F);
    const bool wa = valid && !lost && __ldg(P.atmo_flag + ca) != 0;
    warp_atomic_cell(wa, ca, (long long)wint, P.atmo_w, P.N);
  }
  // pair append, warp-aggregated
  const unsigned mp = __ballot_sync(0xffffffffu, make_pair);
  if (mp) {
    const int leader = __ffs(mp) - 1;
    long long slot0 = 0;
    if (lane == leader)
      slot0 = atomicAdd(reinterpret_cast<unsigned long long*>(&P.st->append), (unsigned long long)(2 * __popc(mp)));
    slot0 = __shfl_sync(0xffffffffu, slot0, leader);
    if (make_pair) {
      const long long dst = (long long)n + slot0 + 2ll * __popc(mp & lanemask_lt());
      if (dst + 2 > P.cap) {
        tally(T, C_DROP);
      } else {
        tally(T, C_PAIRS);
        for (int mm = 0; mm < 2; ++mm) {
          P.pos[dst + mm] = p1;
          P.u[dst + mm] = 0.5f * Pg;
          P.w[dst + mm] = w;
          P.sp[dst + mm] = (mm == 0) ? PIC1D_SP_ELECTRON : PIC1D_SP_POSITRON;
          P.id[dst + mm] = pair_child_id(pid, P.step, mm);
        }
        if (NMAX && __ldg(P.dens_flag + (p1 >> P.F)))
          atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + (int)(p1 >> P.F)),
                    (unsigned long long)(2ll * wint));
      }
    }
  }
  if (valid) {
    P.pos[idx] = p1;
    P.u[idx] = u;
    if (lost) P.sp[idx] = PIC1D_SP_DEAD;
  }
}

template <bool NMAX>
__global__ void __launch_bounds__(sur::NT, 4) k_push_sur(DevParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ uint32_t s_taddr;
  __shared__ unsigned s_tile;
  __shared__ unsigned sCtr[C_COUNT];
  __shared__ float sKl;
  __shared__ double sRed[sur::NT / 32];
  sur::MlpCta M;
  sur::mlp_begin(M, smem_raw, bars, &s_taddr, P.sur_img, P.sur_small);
  const int t = threadIdx.x;
  if (t < C_COUNT) sCtr[t] = 0;
  if (t == 0) {
    sKl = 0.0f;
    s_tile = (unsigned)atomicAdd(&P.st->work, 1ull);
  }
  __syncthreads();
  const uint32_t n = (uint32_t)P.st->n_slots;
  const uint32_t ntiles = (n + sur::TM - 1) / sur::TM;
  Tally T;
  tally_init(T, sCtr, &sKl);
  unsigned tile = s_tile;
  while (tile < ntiles) {
    sur_tile<NMAX>(P, M, tile, n, T);
    __syncthreads();
    if (t == 0) s_tile = (unsigned)atomicAdd(&P.st->work, 1ull);
    __syncthreads();
    tile = s_tile;
  }
  flush_tally(P, T, sRed, P.ke_partial + blockIdx.x, false);
  if (t == 0) {
    if (M.passes) atomicAdd(&P.ctr->sur_rows, (unsigned long long)M.passes * sur::TM);
    if (M.passes_t) atomicAdd(&P.ctr->sur_rows_tangent, (unsigned long long)M.passes_t * sur::TM);
  }
  if (!sur::mlp_end(M) && t == 0) atomicOr(P.sur_err, 1u);
}

// --------------------------------------------------------------------------
// ensemble: every phase of a step is one launch for all lines
// --------------------------------------------------------------------------

// a line's record into the block's shared DevParams, with the line's step
// and the pair-cap density buffers of that step
__device__ void ens_load(const EnsLine* L, int line, DevParams& sP) {
  const int* src = reinterpret_cast<const int*>(&L[line].P);
  int* dst = reinterpret_cast<int*>(&sP);
  for (int k = threadIdx.x; k < (int)(sizeof(DevParams) / 4); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long step = sP.st->step;
    sP.step = step;
    sP.dens_cur = L[line].dens[step & 1];
    sP.dens_next = L[line].dens[(step + 1) & 1];
  }
  __syncthreads();
}

// clear every line's current (start of a step)
__global__ void k_ens_clear(EnsArgs A) {
  const int2 it = A.cell_items[blockIdx.x];
  const EnsLine& L = A.lines[it.x];
  const int c = it.y + threadIdx.x;
  if (c < L.P.N) {
    L.P.J[c] = 0;
    if (L.P.atmo_w) L.P.atmo_w[c] = 0;      // the atmosphere's weight sums of the step
  }
}

// the push of every line with the surrogate drag: items (line, tiles) from a
// global queue; the tallies of an item go to its line
__global__ void __launch_bounds__(sur::NT, 4) k_ens_push(EnsArgs A) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ uint32_t s_taddr;
  __shared__ unsigned s_item;
  __shared__ unsigned sCtr[C_COUNT];
  __shared__ float sKl;
  __shared__ double sRed[sur::NT / 32];
  __shared__ __align__(16) DevParams sP;
  sur::MlpCta M;
  sur::mlp_begin(M, smem_raw, bars, &s_taddr, A.sur_img, A.sur_small);
  const int t = threadIdx.x;
  if (t < C_COUNT) sCtr[t] = 0;
  if (t == 0) sKl = 0.0f;
  Tally T;
  tally_init(T, sCtr, &sKl);
  for (;;) {
    if (t == 0) s_item = (unsigned)atomicAdd(A.work, 1ull);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= (unsigned)A.n_push_items) break;
    const int4 it = A.push_items[item];
    ens_load(A.lines, it.x, sP);
    const long long c0 = clock64();
    const uint32_t n = (uint32_t)sP.st->n_slots;
    const unsigned passes0 = M.passes, passes_t0 = M.passes_t;
    for (int k = 0; k < it.z; ++k) {
      const uint32_t tile = (uint32_t)(it.y + k);
      if (tile * sur::TM >= n) break;
      if (sP.use_nmax) sur_tile<true>(sP, M, tile, n, T);
      else sur_tile<false>(sP, M, tile, n, T);
    }
    flush_tally(sP, T, sRed, &A.lines[it.x].acc[3], true);
    if (t == 0) {
      atomicAdd(&A.lines[it.x].cycles, (unsigned long long)(clock64() - c0));
      if (M.passes > passes0) atomicAdd(&sP.ctr->sur_rows, (unsigned long long)(M.passes - passes0) * sur::TM);
      if (M.passes_t > passes_t0)
        atomicAdd(&sP.ctr->sur_rows_tangent, (unsigned long long)(M.passes_t - passes_t0) * sur::TM);
    }
    __syncthreads();
  }
  if (!sur::mlp_end(M) && t == 0) atomicOr(A.sur_err, 1u);
}

// Ampere update of every line (FP64) and the per-line sums of the step
__global__ void __launch_bounds__(256) k_ens_field(EnsArgs A) {
  const int2 it = A.cell_items[blockIdx.x];
  EnsLine& L = A.lines[it.x];
  const int c = it.y + threadIdx.x;
  double so = 0.0, sn = 0.0, s2 = 0.0;
  if (c < L.P.N) {
    const double Eo = L.E64[c];
    const double En = Eo + (L.a - L.cJ * (double)L.P.J[c]);
    L.E64[c] = En;
    L.E32[c] = (float)En;
    if (L.P.use_nmax) L.dens[L.P.st->step & 1][c] = 0;
    if (L.P.jcum) L.P.jcum[c] += L.P.J[c];
    so = Eo;
    sn = En;
    s2 = En * En;
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
    for (int i = 0; i < 8; ++i) { x += red[0][i]; y += red[1][i]; z += red[2][i]; }
    atomicAdd(&L.acc[0], x);
    atomicAdd(&L.acc[1], y);
    atomicAdd(&L.acc[2], z);
  }
}

// per-line scalars of the step and slot bookkeeping (as k_finalize); the
// next step's push queue starts empty
__global__ void k_ens_finalize(EnsArgs A) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l == 0) *A.work = 0;
  if (l >= A.n_lines) return;
  EnsLine& L = A.lines[l];
  StepState* st = L.P.st;
  st->field_energy = L.acc[2] / (8.0 * 3.141592653589793);
  st->vc = -L.acc[1];
  st->ext_work += L.dt_jext * 0.5 * (L.acc[0] + L.acc[1]);
  st->kinetic = L.acc[3];
  const long long n = st->n_slots, app = st->append;
  long long room = (L.P.cap - n) / 2 * 2;
  if (room < 0) room = 0;
  st->n_slots = n + (app < room ? app : room);
  st->append = 0;
  st->step += 1;
  L.acc[0] = L.acc[1] = L.acc[2] = L.acc[3] = 0.0;
  // the line's history (pic1d_ens_record)
  const EnsRec* R = A.rec;
  if (R && R->cap > 0) {
    const int k = R->n[l];
    if (k < R->cap) {
      R->vc[(size_t)l * R->cap + k] = st->vc;
      R->pairs[(size_t)l * R->cap + k] = (long long)L.P.ctr->pairs_created;
      R->n[l] = k + 1;
    }
  }
}

// after a line's sort: its current buffer is the other one
__global__ void k_ens_flip(EnsLine* lines, int line) {
  EnsLine& L = lines[line];
  const int c = L.cur ^ 1;
  L.cur = c;
  L.P.pos = L.pos[c];
  L.P.u = L.u[c];
  L.P.w = L.w[c];
  L.P.sp = L.sp[c];
  L.P.id = L.id[c];
}

// --------------------------------------------------------------------------
// surface supply: neutral e- (atmospheric) + ion pairs at both footpoints
// --------------------------------------------------------------------------
__global__ void k_inject(DevParams P, double carriers, float sig_e, float sig_i) {
  __shared__ long long cnt[2];
  __shared__ long long slot0;
  // the step being taken, from the device (also right inside an ensemble's
  // captured super-steps, where the launch's parameters are fixed)
  const long long step = P.st->step;
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
    const uint4 r = philox4x32_10(make_uint4((uint32_t)slot, (uint32_t)foot, (uint32_t)step, kTagInj), P.key0, P.key1);
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
      P.id[dst + m] = supply_id(step, foot, slot, m);
    }
    if (P.use_nmax)
      atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + (int)(pfix >> P.F)), 4096ull);
    ++ok;
  }
  if (ok) atomicAdd(&P.ctr->injected, 2ull * ok);
  if (drop) atomicAdd(&P.ctr->injected_dropped, 2ull * drop);
}

// --------------------------------------------------------------------------
// atmosphere top-up (TOPUP): one block per atmosphere cell fills the cell's
// deficit (target minus the plasma weight the push summed) with neutral
// e- + ion pairs of weight 1, uniform in the cell, Maxwellian in both
// directions.  The slots of a cell are one contiguous range taken from the
// step's append counter; pair k of a cell draws Philox (k, cell, step, tag).
// --------------------------------------------------------------------------
__global__ void k_topup(DevParams P, const int* cells, const long long* target, float sig_e, float sig_i) {
  __shared__ long long s_slot0;
  const long long step = P.st->step;     // the step being taken (see k_inject)
  const int c = cells[blockIdx.x];
  const long long deficit = target[blockIdx.x] - P.atmo_w[c];
  const long long npair = deficit > 0 ? deficit / (2ll * 4096ll) : 0;
  if (npair == 0) return;                       // the same for every thread of the block
  if (threadIdx.x == 0)
    s_slot0 = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&P.st->append),
                                   (unsigned long long)(2 * npair));
  __syncthreads();
  const long long n = P.st->n_slots;
  unsigned ok = 0, drop = 0;
  for (long long k = threadIdx.x; k < npair; k += blockDim.x) {
    const long long dst = n + s_slot0 + 2 * k;
    if (dst + 2 > P.cap) { ++drop; continue; }
    const uint4 r = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)c, (uint32_t)step, kTagAtmo), P.key0, P.key1);
    const uint32_t q = r.x >> 16;               // 16 fractional bits of the cell
    const uint32_t frac = P.F >= 16 ? (q << (P.F - 16)) : (q >> (16 - P.F));
    const uint32_t pfix = ((uint32_t)c << P.F) + frac;
    const float rad = sqrtf(-2.0f * logf(1.0f - unit24(r.y)));
    const float ang = 6.283185307179586f * unit24(r.z);
    const float ue = sig_e * rad * cosf(ang);
    const float ui = sig_i * rad * sinf(ang);
    for (int m = 0; m < 2; ++m) {
      P.pos[dst + m] = pfix;
      P.u[dst + m] = m == 0 ? ue : ui;
      P.w[dst + m] = 1.0f;
      P.sp[dst + m] = m == 0 ? PIC1D_SP_ATMO : PIC1D_SP_ION;
      P.id[dst + m] = atmo_id(step, c, k, m);
    }
    if (P.use_nmax) atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + c), 4096ull);
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
    if (P.jcum) P.jcum[c] += P.J[c];
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
    st->step += 1;
  }
}

// --------------------------------------------------------------------------
// cell sort: histogram, exclusive scan, scatter (removed slots dropped).
// Key = group * N + cell with group = 2 * (ion) + (u < 0): four runs (leptons
// moving +s, leptons moving -s, ions moving +s, ions moving -s), each in cell
// order.  The particles of one run move nearly together until the next sort,
// so neighbouring slots stay within a cell or two of each other (the push's
// current registers and shared window stay valid) and a warp mostly follows
// one species' code path.
// --------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

// Sort key: four runs (leptons with u >= 0, u < 0, ions with u >= 0, u < 0),
// each in cell order, and inside a cell kSortBands bands of gamma: the octave
// of gamma^2 (the exponent of the FP32 gamma^2 = 1 + u^2), the last band open
// (gamma^2 >= 2^31), so that the lanes of a warp mostly take the same branch
// of the drag update (the limiter test |F| tau_min < |u| depends on |u|) and
// read the same entries of the drag and branch-certainty tables.
__device__ __forceinline__ int sort_key(const DevParams& P, uint32_t pos, uint8_t sp, float u) {
  const int cell = min((int)(pos >> P.F), P.N - 1);
  const int group = (sp == PIC1D_SP_ION ? 2 : 0) + (u < 0.0f ? 1 : 0);
  const int octave2 = (int)(__float_as_uint(fmaf(u, u, 1.0f)) >> 23) - 127;   // floor(log2 gamma^2) >= 0
  const int band = min(octave2, kSortBands - 1);
  return (group * P.N + cell) * kSortBands + band;
}

// Histogram of the sort keys: K slots per thread per tile (256 K consecutive
// slots, slot t0 + k 256 + thread), all loads issued before the first use so
// that enough bytes are in flight to stream at the copy rate.  The slots were
// sorted at the previous sort and the particles moved a few cells since, so
// a warp's 32 consecutive slots hold a few distinct keys (interleaved: the
// particles of one cell and band spread over two or three new cells): one
// atomic per distinct key of the warp (match.any), not one per run.
template <int K>
__global__ void __launch_bounds__(256) k_hist(DevParams P, uint32_t* counts) {
  const long long n = P.st->n_slots;
  const int lane = threadIdx.x & 31;
  const long long tile = 256ll * K;
  for (long long t0 = (long long)blockIdx.x * tile; t0 < n; t0 += (long long)gridDim.x * tile) {
    uint32_t pos[K];
    float u[K];
    uint8_t sp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const long long i = t0 + k * 256 + threadIdx.x;
      const bool in = i < n;
      sp[k] = in ? P.sp[i] : (uint8_t)PIC1D_SP_DEAD;
      pos[k] = in ? P.pos[i] : 0u;
      u[k] = in ? P.u[i] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool valid = sp[k] != PIC1D_SP_DEAD;
      const int key = valid ? sort_key(P, pos[k], sp[k], u[k]) : -1;
      const unsigned grp = __match_any_sync(0xffffffffu, key);
      if (valid && lane == __ffs(grp) - 1 && PIC1D_BOUND(P, key < 4 * kSortBands * P.N, kChkSortKey))
        atomicAdd(counts + key, (unsigned)__popc(grp));
    }
  }
}

// exclusive scan of the block's values (one per thread) in a 1024-thread block
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* warp_tot, long long& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long t = warp_tot[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += y;
    }
    warp_tot[lane] = t;            // inclusive scan of the warp totals
  }
  __syncthreads();
  total = warp_tot[31];
  const long long before = wid ? warp_tot[wid - 1] : 0;
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* counts, int B, long long* bsum) {
  __shared__ long long wt[32];
  const long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < B) s += counts[base + k];
  long long total;
  block_exclusive_scan(s, wt, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(long long* bsum, int nb, DevParams P) {
  __shared__ long long wt[32];
  long long carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int i = b0 + threadIdx.x;
    const long long v = i < nb ? bsum[i] : 0;
    long long total;
    const long long ex = block_exclusive_scan(v, wt, total);
    if (i < nb) bsum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) P.st->sorted_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* counts, int B, const long long* bsum,
                                                              long long* offsets) {
  __shared__ long long wt[32];
  const long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
  uint32_t c[kScanItems];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    c[k] = (base + k < B) ? counts[base + k] : 0u;
    s += c[k];
  }
  long long total;
  long long run = bsum[blockIdx.x] + block_exclusive_scan(s, wt, total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < B) offsets[base + k] = run;
    run += c[k];
  }
}

// Scatter into key order: per tile of 256 K slots, the keys first, then one
// cursor atomic per distinct key of a warp (all K issued before any result
// is used), then the remaining fields, then the stores; the slots of one key
// in a warp land on consecutive destinations.
template <int K>
__global__ void __launch_bounds__(256) k_scatter(DevParams P, long long* cursor, uint32_t* pos2, float* u2,
                                                 float* w2, uint8_t* sp2, uint64_t* id2) {
  const long long n = P.st->n_slots;
  const int lane = threadIdx.x & 31;
  const long long tile = 256ll * K;
  for (long long t0 = (long long)blockIdx.x * tile; t0 < n; t0 += (long long)gridDim.x * tile) {
    uint32_t pos[K];
    float u[K];
    uint8_t sp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const long long i = t0 + k * 256 + threadIdx.x;
      const bool in = i < n;
      sp[k] = in ? P.sp[i] : (uint8_t)PIC1D_SP_DEAD;
      pos[k] = in ? P.pos[i] : 0u;
      u[k] = in ? P.u[i] : 0.0f;
    }
    long long base[K];
    unsigned grp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool valid = sp[k] != PIC1D_SP_DEAD;
      const int key = valid ? sort_key(P, pos[k], sp[k], u[k]) : -1;
      grp[k] = __match_any_sync(0xffffffffu, key);
      base[k] = 0;
      if (valid && lane == __ffs(grp[k]) - 1)
        base[k] = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(cursor + key),
                                       (unsigned long long)__popc(grp[k]));
    }
    float w[K];
    uint64_t id[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const long long i = t0 + k * 256 + threadIdx.x;
      const bool valid = sp[k] != PIC1D_SP_DEAD;
      w[k] = valid ? P.w[i] : 0.0f;
      id[k] = valid ? P.id[i] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const long long b = __shfl_sync(0xffffffffu, base[k], __ffs(grp[k]) - 1);
      const long long dst = b + __popc(grp[k] & lanemask_lt());
      if (sp[k] != PIC1D_SP_DEAD && PIC1D_BOUND(P, dst >= 0 && dst < P.cap, kChkSortDst)) {
        pos2[dst] = pos[k];
        u2[dst] = u[k];
        w2[dst] = w[k];
        sp2[dst] = sp[k];
        id2[dst] = id[k];
      }
    }
  }
}

__global__ void k_sort_done(DevParams P) {
  P.st->n_slots = P.st->sorted_total;
  P.st->append = 0;
}

// --------------------------------------------------------------------------
// annihilation at n_max, right after a sort.  The sort leaves each cell's
// leptons in two contiguous slot ranges (u >= 0 and u < 0, each over the
// cell's gamma bands); `offsets` holds the end of every bin, `counts` its
// size.  k_annih_scan: one warp per cell sums the lepton, positron and
// pair-electron weight and lists the cells above n_max with the weight A each
// species loses.  k_annih_cell: one block per listed cell finds, per species,
// the smallest key theta whose prefix weight (keys <= theta) reaches A by a
// radix select over the key's eight bytes (eight passes over the cell's
// leptons), takes all weight below theta and the rest of A from the particle
// at theta, and moves E at the cell by the current of the removed charge
// carried to the cell's left node.
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long annih_key(unsigned long long id, long long step) {
  return mix64(id ^ mix64((unsigned long long)step ^ 0xA1111A7Eull));
}

__device__ __forceinline__ void lepton_ranges(const DevParams& P, const uint32_t* counts, const long long* offsets,
                                              int c, long long (&a)[2], long long (&b)[2]) {
  for (int g = 0; g < 2; ++g) {
    const int k0 = (g * P.N + c) * kSortBands;
    a[g] = offsets[k0] - (long long)counts[k0];
    b[g] = offsets[k0 + kSortBands - 1];
  }
}

__global__ void k_annih_scan(DevParams P, const uint32_t* counts, const long long* offsets, int* list,
                             long long* amount, unsigned* count) {
  const int c = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= P.N) return;                          // whole warps
  long long a[2], b[2];
  lepton_ranges(P, counts, offsets, c, a, b);
  long long W = 0, Wp = 0, We = 0;
  for (int g = 0; g < 2; ++g) {
    for (long long i = a[g] + lane; i < b[g]; i += 32) {
      const uint8_t sp = P.sp[i];
      const long long w = __float2ll_rn(P.w[i] * 4096.0f);
      W += w;
      if (sp == PIC1D_SP_POSITRON) Wp += w;
      if (sp == PIC1D_SP_ELECTRON) We += w;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    W += __shfl_down_sync(0xffffffffu, W, o);
    Wp += __shfl_down_sync(0xffffffffu, Wp, o);
    We += __shfl_down_sync(0xffffffffu, We, o);
  }
  if (lane == 0 && W > P.nmax_int) {
    long long A = (W - P.nmax_int) / 2;
    A = min(A, min(Wp, We));
    if (A > 0) {
      const unsigned k = atomicAdd(count, 1u);
      list[k] = c;
      amount[k] = A;
    }
  }
}

// block-wide sums of two int64 values (blockDim.x = kAnnThreads); every thread gets them
constexpr int kAnnThreads = 256;
__device__ __forceinline__ void block_sum2(long long& x, long long& y, long long (*sh)[kAnnThreads / 32]) {
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[0][w] = x; sh[1][w] = y; }
  __syncthreads();
  x = 0;
  y = 0;
  for (int k = 0; k < kAnnThreads / 32; ++k) { x += sh[0][k]; y += sh[1][k]; }
  __syncthreads();
}

// inclusive scan of one int64 per thread over a kAnnThreads block (every
// thread of the block calls it; `tot` holds kAnnThreads / 32 values)
__device__ __forceinline__ long long block_incl_scan(long long v, long long* tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) tot[w] = x;
  __syncthreads();
  long long before = 0;
  for (int k = 0; k < w; ++k) before += tot[k];
  __syncthreads();
  return before + x;
}

__global__ void __launch_bounds__(kAnnThreads) k_annih_cell(DevParams P, const uint32_t* counts,
                                                            const long long* offsets, const int* list,
                                                            const long long* amount, const unsigned* count,
                                                            double* E64, float* E32, double cJ) {
  __shared__ long long sh[2][kAnnThreads / 32];
  __shared__ unsigned long long sHist[2][kAnnThreads];   // one byte's 256 bins per species
  __shared__ long long scan_tot[kAnnThreads / 32];
  __shared__ unsigned long long sPfx[2];
  __shared__ long long sWb[2];
  static_assert(kAnnThreads == 256, "one histogram bin per thread");
  const unsigned ncell = *count;
  const uint32_t fmask = (1u << P.F) - 1u;
  // the step just completed, from the device (also right inside an
  // ensemble's captured super-steps, where the launch's parameters are fixed)
  const long long step = P.st->step;
  for (unsigned item = blockIdx.x; item < ncell; item += gridDim.x) {
    const int c = list[item];
    const long long A = amount[item];
    long long a[2], b[2];
    lepton_ranges(P, counts, offsets, c, a, b);
    // theta[s] = the smallest key with sum_{key <= theta, species s} w >= A,
    // found a byte at a time from the top (radix select): pass d sums the
    // weight of the keys that share the bytes found so far by their next
    // byte, and the byte where the running sum reaches A is the next one of
    // theta; sWb then holds the weight of the keys below theta
    if (threadIdx.x < 2) { sPfx[threadIdx.x] = 0ull; sWb[threadIdx.x] = 0; }
    for (int pass = 0; pass < 8; ++pass) {
      const int shift = 56 - 8 * pass;
      sHist[0][threadIdx.x] = 0ull;
      sHist[1][threadIdx.x] = 0ull;
      __syncthreads();
      const unsigned long long pf0 = sPfx[0], pf1 = sPfx[1];
      for (int g = 0; g < 2; ++g)
        for (long long i = a[g] + threadIdx.x; i < b[g]; i += kAnnThreads) {
          const uint8_t sp = P.sp[i];
          if (sp != PIC1D_SP_ELECTRON && sp != PIC1D_SP_POSITRON) continue;
          const int sg = sp == PIC1D_SP_POSITRON ? 1 : 0;
          const unsigned long long key = annih_key(P.id[i], step);
          if (pass > 0 && (key >> (shift + 8)) != (sg ? pf1 : pf0)) continue;
          const unsigned long long w = (unsigned long long)__float2ll_rn(P.w[i] * 4096.0f);
          atomicAdd(&sHist[sg][(key >> shift) & 255ull], w);
        }
      __syncthreads();
      long long nb[2], nw[2];
      bool hit[2];
      for (int sg = 0; sg < 2; ++sg) {
        const long long v = (long long)sHist[sg][threadIdx.x];
        const long long incl = block_incl_scan(v, scan_tot);
        const long long need = A - sWb[sg];
        hit[sg] = incl - v < need && incl >= need;
        nb[sg] = (long long)(((sg ? pf1 : pf0) << 8) | (unsigned long long)threadIdx.x);
        nw[sg] = sWb[sg] + (incl - v);
      }
      __syncthreads();
      for (int sg = 0; sg < 2; ++sg)
        if (hit[sg]) { sPfx[sg] = (unsigned long long)nb[sg]; sWb[sg] = nw[sg]; }
      __syncthreads();
    }
    const unsigned long long th0 = sPfx[0], th1 = sPfx[1];
    const long long B0 = sWb[0], B1 = sWb[1];
    // remove the weight; X = sum q delta frac (fixed point) of the removed charge
    long long X = 0, unused = 0;
    for (int g = 0; g < 2; ++g)
      for (long long i = a[g] + threadIdx.x; i < b[g]; i += kAnnThreads) {
        const uint8_t sp = P.sp[i];
        if (sp != PIC1D_SP_ELECTRON && sp != PIC1D_SP_POSITRON) continue;
        const bool pos = sp == PIC1D_SP_POSITRON;
        const unsigned long long key = annih_key(P.id[i], step);
        const unsigned long long th = pos ? th1 : th0;
        const long long w = __float2ll_rn(P.w[i] * 4096.0f);
        long long d = 0;
        if (key < th) d = w;
        else if (key == th) d = A - (pos ? B1 : B0);
        if (d > 0) {
          const long long wn = w - d;
          if (wn == 0) P.sp[i] = PIC1D_SP_DEAD;
          else P.w[i] = (float)wn * (1.0f / 4096.0f);
          X += (pos ? d : -d) * (long long)(P.pos[i] & fmask);
        }
      }
    block_sum2(X, unused, sh);
    if (threadIdx.x == 0) {
      const double En = E64[c] + cJ * (double)X;
      E64[c] = En;
      E32[c] = (float)En;
      if (P.jcum) P.jcum[c] -= X;           // the carry to the left node is a current -X in cell c
      if (P.use_nmax) P.dens_cur[c] -= 2 * A;
      atomicAdd(&P.ctr->annihilated, (unsigned long long)(2 * A));
    }
    __syncthreads();
  }
}

// device copy of the table with neighbouring s-rows paired (see table_eval)
__global__ void k_pair_table(const float2* t, int Ng, int Ns, float4* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * (Ns - 1) * Ng) return;
  const int i = idx % Ng;
  const int j = (idx / Ng) % (Ns - 1);
  const int sg = idx / (Ng * (Ns - 1));
  const float2 a = t[((size_t)sg * Ns + j) * Ng + i];
  const float2 b = t[((size_t)sg * Ns + j + 1) * Ng + i];
  out[idx] = make_float4(a.x, a.y, b.x, b.y);
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

// integer charge at the N+1 nodes with the CIC shape: a live particle at
// pos = i 2^F + f gives q w_int (2^F - f) to node i and q w_int f to node
// i + 1 (the units of J: charge x 2^F)
__global__ void k_rho(DevParams P, long long* rho) {
  const long long n = P.st->n_slots;
  const long long one = 1ll << P.F;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const uint8_t s = P.sp[k];
    if (s == PIC1D_SP_DEAD) continue;
    const uint32_t x = P.pos[k];
    const int i = min((int)(x >> P.F), P.N - 1);
    const long long f = (long long)x - ((long long)i << P.F);
    const long long q = (long long)P.qs[s & 3] * __float2ll_rn(P.w[k] * 4096.0f);
    atomicAdd(reinterpret_cast<unsigned long long*>(rho + i), (unsigned long long)(q * (one - f)));
    atomicAdd(reinterpret_cast<unsigned long long*>(rho + i + 1), (unsigned long long)(q * f));
  }
}

// live particles per species: 16 species bytes per thread and load, the
// bytes equal to k found four at a time (__vcmpeq4 sets a matching byte to
// 0xff, so a word's popcount is 8 per match); removed slots (255) match none
__global__ void k_count_species(DevParams P, unsigned long long* out4) {
  const long long n = P.st->n_slots;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long nv = n / 16;
  const uint4* sv = reinterpret_cast<const uint4*>(P.sp);
  unsigned c[4] = {0, 0, 0, 0};
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    const uint4 q = __ldcs(sv + v);
    const unsigned wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      unsigned bits = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) bits += __popc(__vcmpeq4(wd[j], 0x01010101u * (unsigned)k));
      c[k] += bits >> 3;
    }
  }
  for (long long i = nv * 16 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
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
// push variants: particles per thread x minimum resident blocks per SM
struct PushVariant {
  int ppt, minb;
  const void* k_plain;
  const void* k_nmax;
  int stream;               // >= 0: shape of the streaming push (push_stream.cu)
};
#define PV(PPT_, MINB_) {PPT_, MINB_, (const void*)k_push<PPT_, MINB_, false>, (const void*)k_push<PPT_, MINB_, true>, -1}
#define PVL(PPT_, MINB_)                                                                  \
  {PPT_, MINB_, (const void*)k_push<PPT_, MINB_, false, false, true>,                     \
   (const void*)k_push<PPT_, MINB_, true, false, true>, -1}
// variant 0 is the streaming push (push_stream.cu: one block of 32 warps per
// SM, lane-flushed current windows, its table-law instantiation on lines with
// the paper's setup; the default); 1-4 this file's per-thread
// push; 5 the per-thread push with the branch-certainty table and the
// two-anchor current window; 6, 7 other shapes of the streaming push (32
// warps with warp-flushed windows, 24 warps)
static const PushVariant kPushVariants[] = {{1, 1, nullptr, nullptr, 0}, PV(1, 4), PV(1, 3), PV(2, 3), PV(2, 4),
                                            PVL(1, 4), {1, 1, nullptr, nullptr, 1}, {1, 1, nullptr, nullptr, 2}};
#undef PV
#undef PVL
// the atmosphere's push (inject mode TOPUP): one particle per thread, whatever the variant
static const void* const kPushAtmo[2] = {(const void*)k_push<1, 4, false, true>, (const void*)k_push<1, 4, true, true>};
static const void* const kPushAtmoLean[2] = {(const void*)k_push<1, 4, false, true, true>,
                                             (const void*)k_push<1, 4, true, true, true>};
constexpr int kNumPushVariants = sizeof(kPushVariants) / sizeof(kPushVariants[0]);

int push_variant_count() { return kNumPushVariants; }
int push_variant_ppt(int v) { return kPushVariants[v].ppt; }
int push_variant_minb(int v) { return kPushVariants[v].minb; }

int push_blocks_per_sm(int v, bool nmax) {
  if (kPushVariants[v].stream >= 0) return 1;
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, nmax ? kPushVariants[v].k_nmax : kPushVariants[v].k_plain,
                                                kBlock, 0);
  return nb > 0 ? nb : 1;
}

cudaError_t launch_push(const DevParams& P, int variant, int grid, cudaStream_t s) {
  const PushVariant& V = kPushVariants[variant];
  if (V.stream >= 0) return launch_push_stream(P, V.stream, grid, s);
  void* args[] = {const_cast<DevParams*>(&P)};
  const bool lean = variant == 5;
  if (P.G32)
    return cudaLaunchKernel((lean ? kPushAtmoLean : kPushAtmo)[P.use_nmax ? 1 : 0], dim3(grid), dim3(kBlock), args, 0,
                            s);
  return cudaLaunchKernel(P.use_nmax ? V.k_nmax : V.k_plain, dim3(grid), dim3(kBlock), args, 0, s);
}

cudaError_t launch_push_sur(const DevParams& P, int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_push_sur<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sur::MF_SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_push_sur<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sur::MF_SMEM);
    // the whole unified L1/shared capacity as shared memory: 4 CTAs per SM
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_push_sur<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_push_sur<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (P.use_nmax) k_push_sur<true><<<grid, sur::NT, sur::MF_SMEM, s>>>(P);
  else k_push_sur<false><<<grid, sur::NT, sur::MF_SMEM, s>>>(P);
  return cudaGetLastError();
}

cudaError_t ens_launch_clear(const EnsArgs& A, cudaStream_t s) {
  if (A.n_cell_items > 0) k_ens_clear<<<A.n_cell_items, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t ens_launch_push(const EnsArgs& A, int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_ens_push, cudaFuncAttributeMaxDynamicSharedMemorySize, sur::MF_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ens_push, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_ens_push<<<grid, sur::NT, sur::MF_SMEM, s>>>(A);
  return cudaGetLastError();
}

cudaError_t ens_launch_field(const EnsArgs& A, cudaStream_t s) {
  if (A.n_cell_items > 0) k_ens_field<<<A.n_cell_items, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t ens_launch_finalize(const EnsArgs& A, cudaStream_t s) {
  k_ens_finalize<<<(A.n_lines + 127) / 128, 128, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t ens_launch_flip(EnsLine* lines, int line, cudaStream_t s) {
  k_ens_flip<<<1, 1, 0, s>>>(lines, line);
  return cudaGetLastError();
}

cudaError_t launch_topup(const DevParams& P, const int* cells, const long long* target, int n_cells, float sig_e,
                         float sig_i, cudaStream_t s) {
  if (n_cells <= 0) return cudaSuccess;
  k_topup<<<n_cells, 128, 0, s>>>(P, cells, target, sig_e, sig_i);
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

int sort_bins(int N) { return 4 * kSortBands * N; }
int scan_blocks(int N) { return (sort_bins(N) + kScanChunk - 1) / kScanChunk; }

constexpr int kHistK = 8;       // slots per thread per tile of the histogram
constexpr int kScatterK = 8;    // and of the scatter

// blocks of 256 threads resident on `sms` SMs (the sort's kernels stride over
// the slots with a grid that fills the GPU once)
template <typename Kern>
int resident_grid(Kern kern, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 4;
  return sms * per_sm;
}

cudaError_t launch_sort(const DevParams& P, uint32_t* counts, long long* offsets, long long* bsum, uint32_t* pos2,
                        float* u2, float* w2, uint8_t* sp2, uint64_t* id2, int sms, cudaStream_t s) {
  static const int hist_per_sm = resident_grid(k_hist<kHistK>, 1);
  static const int scatter_per_sm = resident_grid(k_scatter<kScatterK>, 1);
  const int B = sort_bins(P.N), nb = scan_blocks(P.N);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)B, s);
  if (e != cudaSuccess) return e;
  k_hist<kHistK><<<sms * hist_per_sm, 256, 0, s>>>(P, counts);
  k_scan_reduce<<<nb, kScanThreads, 0, s>>>(counts, B, bsum);
  k_scan_top<<<1, kScanThreads, 0, s>>>(bsum, nb, P);
  k_scan_apply<<<nb, kScanThreads, 0, s>>>(counts, B, bsum, offsets);
  k_scatter<kScatterK><<<sms * scatter_per_sm, 256, 0, s>>>(P, offsets, pos2, u2, w2, sp2, id2);
  k_sort_done<<<1, 1, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_annihilate(const DevParams& P, const uint32_t* counts, const long long* offsets, int* list,
                              long long* amount, unsigned* count, double* E64, float* E32, double cJ, int sms,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const long long threads = 32ll * P.N;
  k_annih_scan<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(P, counts, offsets, list, amount, count);
  k_annih_cell<<<2 * sms, kAnnThreads, 0, s>>>(P, counts, offsets, list, amount, count, E64, E32, cJ);
  return cudaGetLastError();
}

// the library's generator on caller-given counters (pic1d_philox)
__global__ void k_philox(const uint4* ctr, long long n, uint32_t k0, uint32_t k1, uint4* out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = philox4x32_10(ctr[i], k0, k1);
}

cudaError_t launch_philox(const void* ctr, long long n, unsigned long long key, void* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  const int grid = (int)(blocks < 148 * 16 ? blocks : 148 * 16);
  k_philox<<<grid, 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), n, (uint32_t)key, (uint32_t)(key >> 32),
                                reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

cudaError_t launch_pair_table(const float2* t, int Ng, int Ns, float4* out, cudaStream_t s) {
  const int total = 2 * (Ns - 1) * Ng;
  k_pair_table<<<(total + 255) / 256, 256, 0, s>>>(t, Ng, Ns, out);
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

cudaError_t launch_rho(const DevParams& P, long long* rho, int grid, cudaStream_t s) {
  k_rho<<<grid, 256, 0, s>>>(P, rho);
  return cudaGetLastError();
}

// Discrete continuity, exact in the integer units of the deposit: the node
// charge rho_i (CIC, Sec. 3) changes by the currents of the two cells beside
// node i, rho_i - rho_ref_i = Jcum_{i-1} - Jcum_i at every interior node
// (pairs and supply are created neutral, annihilation carries its charge to
// a node as a current).  out2[0] = max |residual|, out2[1] = the first node
// where it is reached (two passes).
__global__ void k_gauss_residual(DevParams P, const long long* rho, const long long* rho_ref,
                                 unsigned long long* out2, int pass) {
  for (int i = 1 + blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    const long long r = rho[i] - rho_ref[i] - (P.jcum[i - 1] - P.jcum[i]);
    const unsigned long long a = (unsigned long long)(r < 0 ? -r : r);
    if (pass == 0) atomicMax(&out2[0], a);
    else if (a == out2[0]) atomicMin(&out2[1], (unsigned long long)i);
  }
}

cudaError_t launch_gauss_residual(const DevParams& P, const long long* rho, const long long* rho_ref,
                                  unsigned long long* out2, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out2, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(out2 + 1, 0xff, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int grid = P.N / 256 + 1 < 1184 ? P.N / 256 + 1 : 1184;
  for (int pass = 0; pass < 2; ++pass) k_gauss_residual<<<grid, 256, 0, s>>>(P, rho, rho_ref, out2, pass);
  return cudaGetLastError();
}

// checking build: the slack [cap, alloc) past each particle array still
// holds its guard pattern (0xA5 bytes; removed-species code in sp)
__global__ void k_guard_check(const uint8_t* const* arrays, const int* widths, int n_arrays, long long cap,
                              long long alloc, unsigned* check) {
  for (int a = 0; a < n_arrays; ++a) {
    const int wbytes = widths[a];
    const uint8_t want = wbytes == 1 ? (uint8_t)PIC1D_SP_DEAD : (uint8_t)0xA5;
    const long long lo = cap * wbytes, hi = alloc * wbytes;
    for (long long i = lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hi;
         i += (long long)gridDim.x * blockDim.x)
      if (arrays[a][i] != want) atomicOr(check, (unsigned)kChkGuard);
  }
}

cudaError_t launch_guard_check(const uint8_t* const* arrays, const int* widths, int n_arrays, long long cap,
                               long long alloc, unsigned* check, cudaStream_t s) {
  k_guard_check<<<64, 256, 0, s>>>(arrays, widths, n_arrays, cap, alloc, check);
  return cudaGetLastError();
}

cudaError_t launch_count_species(const DevParams& P, unsigned long long* out4, cudaStream_t s) {
  cudaMemsetAsync(out4, 0, 4 * sizeof(unsigned long long), s);
  k_count_species<<<1184, 256, 0, s>>>(P, out4);
  return cudaGetLastError();
}

}  // namespace pic1d
