// push_stream.cu -- the streaming push: one PIC cycle (Sec. 3) for every
// particle slot of a line, with the particle arrays staged through shared
// memory by the bulk-copy engine.
//
// One block of NW warps per SM, every warp on its own.  A warp takes ranges
// of kClaim slots from the launch's dynamic queue (so that the expensive
// parts of the line -- pair zones, dense footpoints -- are shared by every
// SM) and streams each range through a ring of kStages shared-memory slices
// of kSlice slots: lane 0 copies a slice's pos, u, w and sp (13 B per slot)
// in with cp.async.bulk, completion on the slice's mbarrier, one slice ahead
// of the one the warp computes, and once the warp has written a slice's new
// pos and u (8 B per slot) in place copies them back out with bulk stores.
// The bytes in flight then do not depend on registers or occupancy, and the
// warp waits on DRAM only if its next slice is late.
//
// Lane l takes slots l, l + 32, ..., l + 224 of a slice, so its particles
// run through the warp's whole range in the cell order.  Per particle it runs
// the gather, the Strang-split drag around the kick, the Monte-Carlo RICS in
// pair zones, the move and the charge-conserving deposit with the FP32
// arithmetic of the per-thread push of kernels.cu, with three changes that
// remove work:
//   * a drag half-step whose limiter test is certain to choose the damping
//     branch (a precomputed per-(sign, s-row pair, half-octave of gamma^2)
//     flag with a 1e-4 margin) skips the table lookup of that test;
//   * a pair-zone lepton whose scattering probability is certainly below
//     the draw's resolution 2^-24 (another bit of the same table) skips its
//     rate: it cannot scatter and takes no draw;
//   * the current goes into three int64 registers for cells B, B+1, B+2 that
//     take every path whose lower cell is B or B+1 (a path of one step spans
//     at most two cells); only when a path falls outside its lane's window is
//     the window flushed: by that lane alone, or by the whole warp as exact
//     warp sums per cell (one 64-bit atomic per cell and warp).
// Lines that run the table law with the limiter and the certainty table,
// split RICS with the Monte-Carlo step and pairs on (the paper's setup) get an
// instantiation in which those switches are constants, so that no particle
// tests them.
// Every wait on an mbarrier is bounded; a warp whose wait gave up records it
// in the line's counters (pic1d_diag then reports PIC1D_ETIMEOUT) and lets
// the copies it issued land before it stops.
#include <climits>

#include "pic1d_internal.h"
#include "push_device.h"
#include "tc05.h"

namespace pic1d {

namespace {

constexpr int kSlice = 256;                      // slots per slice (8 per lane)
constexpr int kStages = 2;                       // slices in a warp's ring
constexpr int kClaim = 1024;                     // slots per range taken from the queue
constexpr int kOffU = 4 * kSlice, kOffW = 8 * kSlice, kOffSp = 12 * kSlice;
constexpr int kSliceBytes = 13 * kSlice;         // pos | u | w | sp
constexpr long long kWaitLimit = 2000000000ll;   // SM clocks, about a second
static_assert(kSliceBytes % 128 == 0 && kClaim % kSlice == 0, "slices stay aligned");

template <int NW>
constexpr int stream_smem() { return NW * kStages * kSliceBytes + 128; }

// ---------------------------------------------------------------------------
// per-particle physics
// ---------------------------------------------------------------------------
struct SOut {
  uint32_t pos;           // new position (clamped inside the line if lost)
  float u;
  bool lost, want_pair, want_dens;
  float child_u;
  unsigned long long pid;
  int cl;                 // lower of the two cells the step's path can touch
  int la, lb;             // signed path length (fixed point) in cells cl and cl + 1
  int sw;                 // q_sign * w_int
  int cD;                 // end cell (pair-cap density)
  bool atmo;              // in or next to the atmosphere: gravity and the weight sums apply
};

// A RICS scattering of this lane's lepton (App. A): recoil in SPLIT mode,
// true when its photon makes a pair.  Out of line: a few lanes in a million
// scatter, and the others should not carry its arithmetic.
template <bool TBL>
__device__ __noinline__ bool rics_scatter(const DevParams& P, const Site& S, uint32_t ry, float& u, float& Pg) {
  const float beta = u * rsqrtf(fmaf(u, u, 1.0f));
  const float d = (S.mu > beta) ? 1.0f : -1.0f;
  const float ct = dipole_cos(unit24(ry));
  float uf, Eg;
  rics_event(S.b, d, u, ct, uf, Eg, Pg);
  if (TBL || P.rics_mode == PIC1D_RICS_SPLIT) u = uf;
  return (TBL || P.pairs_on) && Eg >= P.pair_e_thr;
}

// One PIC cycle of one particle: the arithmetic of push_one (kernels.cu),
// with the flagged drag half-step and the path split into (cl, la, lb).
// TBL: the line is known to run the table law with the limiter and the
// certainty table, split RICS with the Monte-Carlo step and pairs on (the
// switches are then constants of the instantiation instead of tests of P).
template <bool NMAX, bool ATMO, bool TBL>
__device__ __forceinline__ void stream_one(const DevParams& P, uint32_t gidx, uint32_t pos0, float u, float w, int sp,
                                           Tally& T, float& ke, SOut& o) {
  const uint32_t fmask = (1u << P.F) - 1u;
  const uint32_t half = 1u << (P.F - 1);
  o.lost = false; o.want_pair = false; o.want_dens = false; o.child_u = 0.0f; o.pid = 0; o.atmo = false;
  const bool ion = (sp == PIC1D_SP_ION);
  const bool lep = !ion;
  const float qm = ion ? P.qm[PIC1D_SP_ION] : (sp == PIC1D_SP_POSITRON ? 1.0f : -1.0f);
  const int qs = (sp == PIC1D_SP_ELECTRON || sp == PIC1D_SP_ATMO) ? -1 : 1;
  const float mass = ion ? P.mass[PIC1D_SP_ION] : 1.0f;
  const int cell = (int)(pos0 >> P.F);
  const unsigned cf = __ldg(P.cflag + cell);
  // 1. gather E linearly between cell centres (constant beyond the end centres)
  float Ep, Gp = 0.0f;
  {
    const uint32_t x = pos0 < half ? 0u : pos0 - half;
    int ig = (int)(x >> P.F);
    float f = (float)(x & fmask) * P.inv2F;
    if (ig > P.N - 2) { ig = P.N - 2; f = 1.0f; }
    if (!PIC1D_BOUND(P, ig >= 0, kChkGather)) ig = 0;
    const float e0 = __ldg(P.E32 + ig), e1 = __ldg(P.E32 + ig + 1);
    Ep = fmaf(f, e1 - e0, e0);
    // gravity is zero beyond the atmosphere (and gathers as zero there)
    if (ATMO && (cf & CF_ATMO)) {
      const float g0 = __ldg(P.G32 + ig), g1 = __ldg(P.G32 + ig + 1);
      Gp = fmaf(f, g1 - g0, g0);
      o.atmo = true;
    }
  }
  const bool zone = (cf & CF_ZONE) != 0;
  const bool drag_on = TBL || P.drag_law != PIC1D_DRAG_OFF;
  const bool cont = lep && drag_on && ((!TBL && P.rics_mode == PIC1D_RICS_DRAG_PLUS_PAIRS) || !zone);
  const bool mc = lep && (TBL || P.mc_on) && drag_on && zone;
  Site S;
  if (cont || mc) {
    const float f = (float)(pos0 & fmask) * P.inv2F;
    const float2 mm = __ldg(P.nmu2 + cell);
    S.mu = fmaf(f, mm.y - mm.x, mm.x);
    if (mc || (!TBL && P.drag_law == PIC1D_DRAG_CLOSED)) {
      const float b0 = __ldg(P.nb + cell), b1 = __ldg(P.nb + cell + 1);
      S.b = fmaf(f, b1 - b0, b0);
    } else {
      S.b = 0.0f;
    }
    if (!TBL && P.drag_law == PIC1D_DRAG_CLOSED) {
      const float x0 = __ldg(P.nx + cell), x1 = __ldg(P.nx + cell + 1);
      S.x = fmaf(f, x1 - x0, x0);
    } else {
      S.x = 1.0f;
    }
    site_rows(P, pos0, S);
  }
  // 2-4. Strang split: drag dt/2, Lorentz kick dt, drag dt/2
  if (cont) u = drag_half_flagged<TBL>(P, S, u, T.n_lim, T.n_newt);
  // gravity's acceleration only in and next to the atmosphere (elsewhere Gp
  // is zero and both forms give the same u)
  if (ATMO && o.atmo) u = fmaf(fmaf(qm, Ep, Gp / mass), P.dt, u);
  else u = fmaf(qm * Ep, P.dt, u);
  if (cont) u = drag_half_flagged<TBL>(P, S, u, T.n_lim, T.n_newt);
  // 5. Monte-Carlo RICS in the pair zone
  bool make_pair = false;
  float Pg = 0.0f;
  bool nil = false;
  if (mc && (TBL || P.dflag)) {
    // table law: where every node the lookup can read gives p_sc < 2^-24,
    // there is no draw to make and no rate to evaluate
    const float q = fmaf(u, u, 1.0f);
    const unsigned e2 = (__float_as_uint(q) >> kDampShift) - kDampE2Base;
    if (e2 < (unsigned)kDampNE) {
      const int sg = (u >= 0.0f) ? 0 : 1;
      nil = (__ldg(P.dflag + ((size_t)(sg * (P.Ns - 1) + S.j) * kDampNE + e2)) & kRateNil) != 0;
    }
  }
  if (mc && !nil) {
    const DragVal dv = drag_eval<TBL>(P, u, S, false);
    float psc = P.drag_k * expf(dv.lnN) * P.dt;
    if (psc > 1.0f) { psc = 1.0f; tally(T, C_CLAMP); }
    if (psc >= kDrawMin) {
      ++T.n_draw;
      o.pid = P.id[gidx];
      const uint4 r = philox4x32_10(
          make_uint4((uint32_t)o.pid, (uint32_t)(o.pid >> 32), (uint32_t)P.step, kTagRics), P.key0, P.key1);
      if (unit24_open(r.x) <= psc) {
        tally(T, C_SCAT);
        make_pair = rics_scatter<TBL>(P, S, r.y, u, Pg);
      }
    }
  }
  // 6. move: ds = dt u / gamma, rounded to the fixed-point quantum
  const int wint = __float2int_rn(w * 4096.0f);
  o.sw = qs * wint;
  o.cl = cell;
  o.la = 0;
  o.lb = 0;
  o.cD = cell;
  if (!isfinite(u)) {
    // removed in place: no current, counted (the step reports PIC1D_ENUMERIC)
    tally(T, C_NONFIN);
    o.u = 0.0f;
    o.pos = pos0;
    o.lost = true;
    return;
  }
  const float q = fmaf(u, u, 1.0f);
  const float r = rsqrtf(q);                                   // 1 / gamma
  int d = __float2int_rn(P.dt * (u * r) * (float)(1u << P.F));
  const float e = w * mass * __fdividef(u * u * r, 1.0f + r);  // w m (gamma - 1)
  const bool lostN = d < 0 && (uint32_t)(-d) > pos0;
  const bool lostS = d > 0 && (uint32_t)d > P.top1 - pos0;
  o.lost = lostN || lostS;
  if (o.lost) {
    atomicAdd(T.skl, e);
    // leaves through a wall: the path ends at the conductor (node 0 or node N)
    tally(T, lostN ? C_LOSTN : C_LOSTS);
    d = lostN ? -(int)pos0 : (int)(P.top - (long long)pos0);
    o.pos = lostN ? 0u : (uint32_t)(P.top - 1);
    if (make_pair) tally(T, C_WALL);     // the parent left the line: no pair
    make_pair = false;
  } else {
    ke += e;
    o.pos = pos0 + (uint32_t)d;
    if (NMAX && lep && (cf & CF_DENSN)) {
      o.cD = (int)(o.pos >> P.F);
      o.want_dens = PIC1D_BOUND(P, o.cD < P.N, kChkCell) && __ldg(P.dens_flag + o.cD) != 0;
    }
  }
  // 7. charge-conserving deposit: the signed length of the path inside the
  // start cell and inside the neighbour it moves into (a step is shorter
  // than a cell); cl is the lower of the two
  path_lengths(d, pos0 & fmask, P.F, cell, o.cl, o.la, o.lb);
  o.u = u;
  if (make_pair) {
    if (NMAX && P.dens_cur[(int)(o.pos >> P.F)] >= P.nmax_int) {
      tally(T, C_REJ);
    } else {
      o.want_pair = true;
      o.child_u = 0.5f * Pg;
    }
  }
}

// ---------------------------------------------------------------------------
// a warp's slices
// ---------------------------------------------------------------------------
// copy slice (slots base .. base+len-1) into `st`, completion on `bar`
// (whole 16-byte groups: the arrays have slack past the last slot; slots past
// len are read but not used)
__device__ __forceinline__ void slice_load(const DevParams& P, uint8_t* st, uint64_t* bar, uint32_t base,
                                           uint32_t len) {
  const uint32_t b4 = (len * 4u + 15u) & ~15u, b1 = (len + 15u) & ~15u;
  tc::mbar_expect_tx(bar, 3u * b4 + b1);
  tc::bulk_g2s(st, P.pos + base, b4, bar);
  tc::bulk_g2s(st + kOffU, P.u + base, b4, bar);
  tc::bulk_g2s(st + kOffW, P.w + base, b4, bar);
  tc::bulk_g2s(st + kOffSp, P.sp + base, b1, bar);
}

// the slice's new pos and u back to global memory: whole 16-byte groups by
// the bulk engine (one committed group), the last few slots of the line by
// plain stores
__device__ __forceinline__ void slice_store(const DevParams& P, const uint8_t* st, uint32_t base, uint32_t len) {
  const uint32_t len4 = len & ~3u;
  if (len4) {
    tc::bulk_s2g(P.pos + base, st, len4 * 4u);
    tc::bulk_s2g(P.u + base, st + kOffU, len4 * 4u);
  }
  tc::bulk_commit();
  const uint32_t* spos = reinterpret_cast<const uint32_t*>(st);
  const float* su = reinterpret_cast<const float*>(st + kOffU);
  for (uint32_t i = len4; i < len; ++i) {
    P.pos[base + i] = spos[i];
    P.u[base + i] = su[i];
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <int NW, bool WARPFLUSH, bool NMAX, bool ATMO, bool TBL>
__global__ void __launch_bounds__(32 * NW, 1) k_push_stream(DevParams P) {
  extern __shared__ uint8_t s_raw[];
  __shared__ __align__(8) uint64_t s_bar[NW][kStages];
  __shared__ unsigned sCtr[C_COUNT];
  __shared__ float sKl;
  __shared__ unsigned sBad;
  __shared__ double sRed[NW];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(s_raw) + 127) & ~uintptr_t(127)) +
                  (size_t)warp * kStages * kSliceBytes;
  uint64_t* bar = s_bar[warp];
  if (t < C_COUNT) sCtr[t] = 0;
  if (t == 0) { sKl = 0.0f; sBad = 0; }
  if (lane == 0) {
    for (int q = 0; q < kStages; ++q) tc::mbar_init(&bar[q], 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  const uint32_t n = (uint32_t)P.st->n_slots;
  const uint32_t nclaims = (n + kClaim - 1) / kClaim;
  Tally T;
  tally_init(T, sCtr, &sKl);
  double ke64 = 0.0;
  JWin W;
  jwin_init(W);
  // the pair cap's lepton density of this lane: cells Dc and Dc + 1
  int Dc = -(1 << 29);
  long long D0 = 0, D1 = 0;

  // the slice a warp works on: range `claim`, slice `j` of it
  unsigned claim = 0;
  if (lane == 0) claim = (unsigned)atomicAdd(&P.st->work, 1ull);
  claim = __shfl_sync(0xffffffffu, claim, 0);
  int j = 0;
  if (claim < nclaims && lane == 0) {
    const uint32_t base = claim * (uint32_t)kClaim;
    slice_load(P, ring, &bar[0], base, min((uint32_t)kSlice, n - base));
  }
  bool ok = true;
  for (unsigned k = 0; claim < nclaims; ++k) {
    const int s = (int)(k % kStages);
    uint8_t* st = ring + s * kSliceBytes;
    const uint32_t cbase = claim * (uint32_t)kClaim;
    const uint32_t cend = min(cbase + (uint32_t)kClaim, n);
    const uint32_t base = cbase + (uint32_t)j * kSlice;
    const uint32_t len = min((uint32_t)kSlice, cend - base);
    // the next slice: the next one of this range, or the first of a new range
    unsigned nclaim = claim;
    int nj = j + 1;
    if (cbase + (uint32_t)nj * kSlice >= cend) {
      if (lane == 0) nclaim = (unsigned)atomicAdd(&P.st->work, 1ull);
      nclaim = __shfl_sync(0xffffffffu, nclaim, 0);
      nj = 0;
    }
    if (nclaim < nclaims && lane == 0) {
      // its ring slot last held slice k + 1 - kStages, whose store must have
      // finished reading it (every more recent store may still be running)
      tc::bulk_wait_read_le<kStages - 2>();
      const uint32_t nb = nclaim * (uint32_t)kClaim + (uint32_t)nj * kSlice;
      const uint32_t ne = min(nclaim * (uint32_t)kClaim + (uint32_t)kClaim, n);
      slice_load(P, ring + ((k + 1) % kStages) * kSliceBytes, &bar[(k + 1) % kStages], nb,
                 min((uint32_t)kSlice, ne - nb));
    }
    // every lane waits on its own clock: the warp goes on only if all got there
    const bool got = tc::mbar_wait(&bar[s], (k / kStages) & 1, kWaitLimit);
    if (!__all_sync(0xffffffffu, got)) {
      ok = false;
      if (lane == 0) {
        // let the copies of this slice and the next land before the block ends
        tc::mbar_wait(&bar[s], (k / kStages) & 1, kWaitLimit);
        if (nclaim < nclaims) tc::mbar_wait(&bar[(k + 1) % kStages], ((k + 1) / kStages) & 1, kWaitLimit);
      }
      break;
    }
    float ke = 0.0f;
#pragma unroll 1
    for (int i = 0; i < kSlice / 32; ++i) {
      const uint32_t slot = (uint32_t)(i * 32 + lane);
      if (__all_sync(0xffffffffu, slot >= len)) break;
      const uint32_t pos0 = *reinterpret_cast<const uint32_t*>(st + 4 * slot);
      const float u0 = *reinterpret_cast<const float*>(st + kOffU + 4 * slot);
      const float w0 = *reinterpret_cast<const float*>(st + kOffW + 4 * slot);
      const int spk = st[kOffSp + slot];
      const uint32_t gidx = base + slot;
      const bool valid = slot < len && spk != PIC1D_SP_DEAD &&
                         PIC1D_BOUND(P, (pos0 >> P.F) < (uint32_t)P.N, kChkCell) &&
                         PIC1D_BOUND(P, (long long)gidx < P.cap, kChkSlot);
      SOut o;
      o.want_pair = false;
      o.want_dens = false;
      o.lost = false;
      o.atmo = false;
      if (valid) stream_one<NMAX, ATMO, TBL>(P, gidx, pos0, u0, w0, spk & 3, T, ke, o);
      // current
      jwin_add<WARPFLUSH>(W, valid, o.cl, o.la, o.lb, o.sw, P.J, P.N);
      // plasma weight of the atmosphere cells after the move
      if (ATMO) {
        const bool ma = valid && o.atmo && !o.lost && __ldg(P.atmo_flag + (o.pos >> P.F)) != 0;
        const unsigned am = __ballot_sync(0xffffffffu, ma);
        if (ma) {
          const int ac = (int)(o.pos >> P.F);
          const unsigned grp = __match_any_sync(am, ac);
          const long long sum = group_sum64(grp, (long long)__float2int_rn(w0 * 4096.0f));
          if (lane == __ffs(grp) - 1)
            atomicAdd(reinterpret_cast<unsigned long long*>(P.atmo_w + ac), (unsigned long long)sum);
        }
      }
      // lepton density for the pair cap (only cells where a pair can be
      // tested): two registers per lane, to global memory when a lepton ends
      // outside them
      if (NMAX && o.want_dens) {
        const int kd = o.cD - Dc;
        if ((unsigned)kd > 1u) {
          if (D0) atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + Dc), (unsigned long long)D0);
          if (D1) atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + Dc + 1), (unsigned long long)D1);
          D0 = D1 = 0;
          Dc = (o.cD > Dc) ? o.cD - 1 : o.cD;
        }
        const long long vD = (long long)__float2int_rn(w0 * 4096.0f);
        if (o.cD == Dc) D0 += vD;
        else D1 += vD;
      }
      // pair append, warp-aggregated
      const unsigned m = __ballot_sync(0xffffffffu, o.want_pair);
      if (m) {
        const int leader = __ffs(m) - 1;
        long long slot0 = 0;
        if (lane == leader)
          slot0 = atomicAdd(reinterpret_cast<unsigned long long*>(&P.st->append), (unsigned long long)(2 * __popc(m)));
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
              P.w[dst + mm] = w0;
              P.sp[dst + mm] = (mm == 0) ? PIC1D_SP_ELECTRON : PIC1D_SP_POSITRON;
              P.id[dst + mm] = pair_child_id(o.pid, P.step, mm);
            }
            if (NMAX && __ldg(P.dens_flag + (o.pos >> P.F)))
              atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + (int)(o.pos >> P.F)),
                        (unsigned long long)(2ll * __float2int_rn(w0 * 4096.0f)));
          }
        }
      }
      if (valid) {
        *reinterpret_cast<uint32_t*>(st + 4 * slot) = o.pos;
        *reinterpret_cast<float*>(st + kOffU + 4 * slot) = o.u;
        if (o.lost) P.sp[gidx] = PIC1D_SP_DEAD;
      }
    }
    ke64 += (double)ke;
    // the results become visible to the bulk-copy engine, then go back out
    tc::fence_async_smem();
    __syncwarp();
    if (lane == 0) slice_store(P, st, base, len);
    claim = nclaim;
    j = nj;
  }
  if (lane == 0) tc::bulk_wait_all();
  if (!ok && lane == 0) sBad = 1;
  if (WARPFLUSH) jwin_flush_warp(W, P.J, P.N);
  else jwin_flush_lane(W, P.J, P.N);
  if (NMAX) {
    if (D0) atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + Dc), (unsigned long long)D0);
    if (D1) atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_next + Dc + 1), (unsigned long long)D1);
  }

  // ---------------- the block's tallies
  {
    const unsigned a = __reduce_add_sync(0xffffffffu, T.n_lim), b = __reduce_add_sync(0xffffffffu, T.n_newt);
    const unsigned c = __reduce_add_sync(0xffffffffu, T.n_draw);
    if (lane == 0) {
      if (a) atomicAdd(sCtr + C_LIM, a);
      if (b) atomicAdd(sCtr + C_NEWT, b);
      if (c) atomicAdd(sCtr + C_DRAW, c);
    }
    double ked = ke64;
    for (int dd = 16; dd > 0; dd >>= 1) ked += __shfl_down_sync(0xffffffffu, ked, dd);
    if (lane == 0) sRed[warp] = ked;
  }
  __syncthreads();
  if (t == 0) {
    double ke = 0.0;
    for (int i = 0; i < NW; ++i) ke += sRed[i];
    P.ke_partial[blockIdx.x] = ke;
    if (sKl != 0.0f) atomicAdd(&P.st->ke_lost, (double)sKl);
    Counters* Cn = P.ctr;
    unsigned long long* dst[C_COUNT] = {&Cn->scatters, &Cn->psc_clamped, &Cn->limiter_branch, &Cn->newton_branch,
                                        &Cn->nonfinite, &Cn->lost_north, &Cn->lost_south, &Cn->pairs_created,
                                        &Cn->pairs_dropped_cap, &Cn->pairs_rejected_nmax, &Cn->pairs_lost_wall,
                                        &Cn->rng_draws};
    for (int q = 0; q < C_COUNT; ++q)
      if (sCtr[q]) atomicAdd(dst[q], (unsigned long long)sCtr[q]);
    if (sBad) atomicAdd(&Cn->waits_timed_out, 1ull);
  }
}

// The branch-certainty table: entry (sg, j, h) is kDampCertain when for every gamma^2
// in half-octave h (bits of (float)gamma^2 >> 22 = kDampE2Base + h) and every
// s between rows j and j+1, the limiter test |drag_k F| tau_min < |u| of the
// table law is false with a relative margin of 1e-4: the bilinear F there is
// a convex combination of the table nodes it reads (gamma nodes floor(t_lo)
// .. ceil(t_hi) of that half-octave's t range, rows j and j+1), so when
// those nodes share one sign, |F| is at least their smallest magnitude, and
// |u| is at most sqrt(q_hi - 1).  It is kNewtonStill when the test is
// certain to choose the Newton branch there and that branch's update moves u
// by less than a quarter of the FP32 spacing of the smallest |u| of the
// half-octave, so that the half-step returns u unchanged.  Bit kRateNil marks
// the entries where the scattering probability drag_k N dt of every node the
// lookup reads is below the draw's resolution 2^-24 (no lepton there can
// scatter, so the Monte-Carlo step has nothing to evaluate or draw).
__global__ void k_damp_flags(const float4* tpair, int Ng, int Ns, float t_scale, float drag_k, float tau_min, float dt,
                             uint8_t* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * (Ns - 1) * kDampNE) return;
  const int h = idx % kDampNE;
  const int j = (idx / kDampNE) % (Ns - 1);
  const int sg = idx / (kDampNE * (Ns - 1));
  const int e = (int)kDampE2Base + h;                  // (float bits of q) >> kDampShift
  const int ex = (e >> kDampMant) - 127;                // exponent of q
  const double step = 1.0 / (double)(1 << kDampMant);   // the bin's width in units of 2^ex
  const double q_lo = ldexp(1.0 + step * (double)(e & ((1 << kDampMant) - 1)), ex);
  const double q_hi = q_lo + ldexp(step, ex);
  // t = 0.5 log2(q) t_scale in FP32 by the push; a slack of 1e-3 node units
  const double t_lo = fmax(0.5 * log2(q_lo) * (double)t_scale - 1e-3, 0.0);
  const double t_hi = 0.5 * log2(q_hi) * (double)t_scale + 1e-3;
  int i_lo = (int)floor(t_lo), i_hi = (int)ceil(t_hi);
  if (i_lo > Ng - 1) i_lo = Ng - 1;
  if (i_hi > Ng - 1) i_hi = Ng - 1;
  if (i_lo > Ng - 2) i_lo = Ng - 2;                     // the top clamp reads nodes Ng-2 and Ng-1
  const float4* row = tpair + (size_t)(sg * (Ns - 1) + j) * Ng;
  double fmn = INFINITY;
  int pos = 0, neg = 0;
  for (int i = i_lo; i <= i_hi; ++i) {
    const float4 a = row[i];
    const double f0 = (double)a.x, f1 = (double)a.z;
    pos += (f0 > 0.0) + (f1 > 0.0);
    neg += (f0 < 0.0) + (f1 < 0.0);
    fmn = fmin(fmn, fmin(fabs(f0), fabs(f1)));
  }
  double fmx = 0.0, lmx = -INFINITY;
  for (int i = i_lo; i <= i_hi; ++i) {
    const float4 a = row[i];
    fmx = fmax(fmx, fmax(fabs((double)a.x), fabs((double)a.z)));
    lmx = fmax(lmx, fmax((double)a.y, (double)a.w));
  }
  const int nodes = 2 * (i_hi - i_lo + 1);
  const double u_lo = sqrt(fmax(q_lo - 1.0, 0.0)), u_hi = sqrt(fmax(q_hi - 1.0, 0.0));
  const bool one_sign = (pos == nodes) || (neg == nodes);
  const bool damp = one_sign && (double)drag_k * fmn * (double)tau_min >= u_hi * (1.0 + 1e-4) + 1e-30;
  // Newton branch with a change below a quarter of the FP32 spacing at u_lo:
  // |u1 - u0| <= h |F| / (1 - h F'/2) <= 2 h |F| (the denominator is at least
  // 1/2), so u0 + (u1 - u0) rounds to u0
  bool still = false;
  if (!damp && u_lo > 0.0) {
    const double fk = (double)drag_k * fmx * (1.0 + 1e-3);
    const double h = 0.5 * (double)dt;
    const double ulp = ldexp(1.0, ilogb(u_lo) - 23);
    still = fk * (double)tau_min < u_lo * (1.0 - 1e-4) && 2.0 * h * fk <= 0.25 * ulp;
  }
  // the bilinear ln N is a convex combination of the nodes it reads, so p_sc
  // = drag_k exp(ln N) dt is at most that of their largest ln N; a margin of
  // 1e-3 covers the FP32 interpolation and expf
  const bool nil = (double)drag_k * exp(lmx) * (double)dt < 0x1p-24 * (1.0 - 1e-3);
  out[idx] = (uint8_t)((damp ? kDampCertain : (still ? kNewtonStill : 0)) | (nil ? kRateNil : 0));
}

}  // namespace

namespace {

// the lines the TBL instantiations serve: table law with the limiter and
// the certainty table, split RICS, Monte-Carlo and pairs on
bool table_line(const DevParams& P) {
  return P.drag_law == PIC1D_DRAG_TABLE && P.dflag != nullptr && P.limiter_on && P.rics_mode == PIC1D_RICS_SPLIT &&
         P.mc_on && P.pairs_on;
}

template <int NW, bool WF, bool TBL>
cudaError_t launch_shape(const DevParams& P, int grid, cudaStream_t s, bool& attr) {
  const void* ks[4] = {(const void*)k_push_stream<NW, WF, false, false, TBL>,
                       (const void*)k_push_stream<NW, WF, true, false, TBL>,
                       (const void*)k_push_stream<NW, WF, false, true, TBL>,
                       (const void*)k_push_stream<NW, WF, true, true, TBL>};
  if (!attr) {
    for (const void* k : ks) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, stream_smem<NW>());
      if (e != cudaSuccess) return e;
    }
    attr = true;
  }
  const int which = (P.use_nmax ? 1 : 0) + (P.G32 ? 2 : 0);
  void* args[] = {const_cast<DevParams*>(&P)};
  return cudaLaunchKernel(ks[which], dim3(grid), dim3(32 * NW), args, (size_t)stream_smem<NW>(), s);
}

}  // namespace

// shapes of the streaming push: 32 warps with lane-flushed current windows
// (the fastest measured; table-law lines run its TBL instantiation), 32 warps
// with warp-flushed windows, 24 warps with warp-flushed windows
int stream_variant_count() { return 3; }
int stream_variant_ppl(int) { return 1; }

cudaError_t launch_push_stream(const DevParams& P, int shape, int grid, cudaStream_t s) {
  static bool attr[4] = {false, false, false, false};
  switch (shape) {
    case 0:
      if (table_line(P)) return launch_shape<32, false, true>(P, grid, s, attr[3]);
      return launch_shape<32, false, false>(P, grid, s, attr[0]);
    case 1: return launch_shape<32, true, false>(P, grid, s, attr[1]);
    default: return launch_shape<24, true, false>(P, grid, s, attr[2]);
  }
}

// The bounded wait of the push kernels on an mbarrier that nothing
// completes (no copy, no arrive): it gives up after `limit` SM clocks and the
// block records that in the line's counters, like a push block whose copy
// never landed.
__global__ void k_wait_check(Counters* ctr, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
    if (!tc::mbar_wait(&bar, 0, limit)) atomicAdd(&ctr->waits_timed_out, 1ull);
  }
}

cudaError_t launch_wait_check(Counters* ctr, long long limit_clocks, cudaStream_t s) {
  k_wait_check<<<1, 32, 0, s>>>(ctr, limit_clocks);
  return cudaGetLastError();
}

cudaError_t launch_damp_flags(const float4* tpair, int Ng, int Ns, float t_scale, float drag_k, float tau_min,
                              float dt, uint8_t* out, cudaStream_t s) {
  const int total = 2 * (Ns - 1) * kDampNE;
  k_damp_flags<<<(total + 255) / 256, 256, 0, s>>>(tpair, Ng, Ns, t_scale, drag_k, tau_min, dt, out);
  return cudaGetLastError();
}

}  // namespace pic1d
