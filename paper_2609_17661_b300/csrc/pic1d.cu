// pic1d.cu -- host side of the C ABI declared in include/pic1d.h.
//
// Builds the dipole field-line tables of App. B.2 in FP64 on the host (arc
// length in closed form, theta(s) by Newton), the drag/rate table by FP64
// quadrature on the device, owns all device memory of a context and issues
// the per-step kernels of kernels.cu on the caller's stream.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "pic1d_internal.h"
#include "push_device.h"

namespace {
// an NVTX range over a host scope (free when no tool is attached)
struct Nvtx {
  explicit Nvtx(const char* name) { nvtxRangePushA(name); }
  ~Nvtx() { nvtxRangePop(); }
  Nvtx(const Nvtx&) = delete;
  Nvtx& operator=(const Nvtx&) = delete;
};
}  // namespace

using namespace pic1d;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kRe = 2.8179403262e-13;       // classical electron radius, cm (CODATA 2018)
constexpr double kLbar = 3.8615926796e-11;     // reduced Compton wavelength, cm
constexpr double kMeKeV = 510.99895;           // m_e c^2, keV

// arc length of r = r_eq sin^2(theta) from the northern footpoint, in R*:
// the antiderivative of sin(t) sqrt(1 + 3 cos^2 t) is -A(cos t) with
// A(c) = c sqrt(1+3c^2)/2 + asinh(sqrt(3) c)/(2 sqrt(3)).
double arc_A(double c) { return 0.5 * c * std::sqrt(1.0 + 3.0 * c * c) + std::asinh(std::sqrt(3.0) * c) / (2.0 * std::sqrt(3.0)); }

struct Line {
  double r_eq, th0, c0, L;
  explicit Line(double r) : r_eq(r) {
    th0 = std::asin(std::sqrt(1.0 / r));
    c0 = std::cos(th0);
    L = 2.0 * r * arc_A(c0);
  }
  double s_of(double th) const { return r_eq * (arc_A(c0) - arc_A(std::cos(th))); }
  double ds(double th) const {
    const double c = std::cos(th);
    return r_eq * std::sin(th) * std::sqrt(1.0 + 3.0 * c * c);
  }
  // theta(s), s in R*; Newton from a guess, guarded by a bracket
  double theta_of(double s, double guess) const {
    double lo = th0, hi = kPi - th0;
    double th = std::min(std::max(guess, lo), hi);
    for (int it = 0; it < 60; ++it) {
      const double f = s_of(th) - s;
      if (f > 0) hi = th; else lo = th;
      const double d = ds(th);
      double nt = (d > 0) ? th - f / d : 0.5 * (lo + hi);
      if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
      if (std::fabs(nt - th) < 1e-15) { th = nt; break; }
      th = nt;
    }
    return th;
  }
};

void field_at(const pic1d_params& p, double th, double& x, double& b, double& mu) {
  const double c = std::cos(th), sn = std::sin(th);
  x = p.r_eq * sn * sn;
  const double root = std::sqrt(1.0 + 3.0 * c * c);
  b = p.b_star * root / (x * x * x);
  if (p.b_convention == 1) b *= 0.5;
  mu = 2.0 * c / root;
}

// Gauss-Legendre nodes/weights on [-1, 1]: Newton on P_n from Chebyshev guesses
void legendre_nodes(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// default push variant: PIC1D_PUSH_VARIANT (index) if set, else the
// streaming push (variant 0, the fastest measured on the 1e9-particle line)
int default_push_variant() {
  const char* e = std::getenv("PIC1D_PUSH_VARIANT");
  if (e) {
    const int v = std::atoi(e);
    if (v >= 0 && v < push_variant_count()) return v;
  }
  return 0;
}

int fbits_of(int n) {
  int b = 0;
  while ((1 << b) < n) ++b;
  return 32 - b;
}

}  // namespace

namespace {
constexpr int kSurPushPerSm = 4;     // CTAs per SM of the surrogate push (52 KB shared, 128 TMEM columns each)
}

struct pic1d_ctx {
  pic1d_params p{};
  cudaStream_t s = nullptr;
  int N = 0, F = 0;
  double L_R = 0, R_cells = 0, q_p = 0, j_ext = 0, tau_min = 0, dt = 0;
  long long cap = 0;     // logical capacity (slots)
  long long alloc = 0;   // allocated slots per buffer
  int cur = 0;
  uint32_t* pos[2] = {nullptr, nullptr};
  float* u[2] = {nullptr, nullptr};
  float* w[2] = {nullptr, nullptr};
  uint8_t* sp[2] = {nullptr, nullptr};
  uint64_t* id[2] = {nullptr, nullptr};
  double* E64 = nullptr;
  float* E32 = nullptr;
  long long* J = nullptr;
  long long* dens[2] = {nullptr, nullptr};
  float *nb = nullptr, *nmu = nullptr, *nx = nullptr;
  uint8_t* zone = nullptr;
  uint8_t* dens_flag = nullptr;
  uint8_t* fast_cell = nullptr;
  // atmosphere (inject mode TOPUP)
  float* G32 = nullptr;             // gravity along s per unit mass at cell centres
  uint8_t* atmo_flag = nullptr;     // cells of the atmosphere
  long long* atmo_w = nullptr;      // plasma weight per cell after the push (w_int)
  int* atmo_cells = nullptr;        // the atmosphere's cells
  long long* atmo_target = nullptr; // their target weights (w_int)
  int n_atmo = 0;
  // annihilation at n_max (annihilate_every > 0)
  int* ann_list = nullptr;          // cells that annihilate in a pass
  long long* ann_amount = nullptr;  // weight each species loses there (w_int)
  unsigned* ann_count = nullptr;
  float2* table = nullptr;
  float4* tpair = nullptr;
  Counters* ctr = nullptr;
  StepState* st = nullptr;
  double* ke_partial = nullptr;
  double* field_partial = nullptr;
  uint32_t* counts = nullptr;
  long long* offsets = nullptr;
  long long* bsum = nullptr;
  unsigned long long* spc = nullptr;
  int push_grid = 0;      // grid of the current push variant
  int push_variant = 0;   // index into the push variants (particles per thread x occupancy)
  uint8_t* cflag = nullptr;   // cell flags of the streaming push
  float2* nmu2 = nullptr;     // mu at both nodes of each cell
  uint8_t* dflag = nullptr;   // branch-certainty table of the table law (damping, Newton, rate)
  int sms = 0;
  long long step = 0;
  std::string err;
  // push timing (pic1d_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev;      // pairs (start, stop) per timed launch
  std::vector<long long> ev_slots;  // slots read by each timed launch (filled at diag)
  long long* slot_log = nullptr;    // device copy of n_slots at each timed launch
  long long slot_log_cap = 0;
  long long timed = 0;
  double timed_ms = 0.0;
  long long timed_slots = 0;
  // learned surrogate (allocated on first use)
  bool sur_on = false;
  SurBufs sur{};
  int sur_t = 0;                 // Adam steps taken since the parameters were set
  double* sur_gx = nullptr;      // Gauss-Legendre nodes of the sample quadrature
  double* sur_gw = nullptr;
  float* sur_grad = nullptr;
  float* sur_loss = nullptr;     // loss sum of a gradient call
  long long* rho = nullptr;      // node charge of pic1d_get_rho (allocated on first use)
  // discrete continuity check (pic1d_gauss_mark): the cumulative current of
  // every cell (always kept, added by the field update) and the node charge
  // when the mark was taken
  long long* jcum = nullptr;
  long long* rho_ref = nullptr;
  // checking build: the failed-bounds word, and the guard test's array table
  unsigned* check = nullptr;
  const uint8_t** guard_arrays = nullptr;
  int* guard_widths = nullptr;
  unsigned long long* gauss_out = nullptr;
  bool gauss_on = false;
};

namespace {

int fail(pic1d_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(pic1d_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? PIC1D_ENOMEM : PIC1D_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                             \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

// Device memory of contexts and ensembles comes from one process-wide
// allocator: cudaMalloc/cudaFree, or the caller's hooks (pic1d_set_allocator).
// The hooks may change only while no context or ensemble is alive, so every
// buffer is freed by the allocator that made it.
pic1d_alloc_fn g_alloc = nullptr;
pic1d_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;
std::atomic<long long> g_live{0};

cudaError_t raw_alloc(void** p, size_t bytes) {
  if (!g_alloc) return cudaMalloc(p, bytes);
  *p = g_alloc(bytes, g_alloc_user);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

void dfree(void* p) {
  if (!p) return;
  if (g_free) g_free(p, g_alloc_user);
  else cudaFree(p);
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return raw_alloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
}

void free_particles(pic1d_ctx* c) {
  for (int b = 0; b < 2; ++b) {
    dfree(c->pos[b]); dfree(c->u[b]); dfree(c->w[b]); dfree(c->sp[b]); dfree(c->id[b]);
    c->pos[b] = nullptr; c->u[b] = nullptr; c->w[b] = nullptr; c->sp[b] = nullptr; c->id[b] = nullptr;
  }
}

int alloc_particles(pic1d_ctx* c, long long want) {
  // whole tiles plus one tile of slack for the 128-bit loads past the end;
  // the logical capacity is exactly what was asked for
  const long long cap = (want + kTile - 1) / kTile * kTile + kTile;
  free_particles(c);
  for (int b = 0; b < 2; ++b) {
    CK(dalloc(&c->pos[b], cap), "alloc pos");
    CK(dalloc(&c->u[b], cap), "alloc u");
    CK(dalloc(&c->w[b], cap), "alloc w");
    CK(dalloc(&c->sp[b], cap), "alloc sp");
    CK(dalloc(&c->id[b], cap), "alloc id");
    CK(cudaMemsetAsync(c->sp[b], PIC1D_SP_DEAD, cap, c->s), "memset sp");
  }
  c->cap = want;
  c->alloc = cap;
#ifdef PIC1D_CHECK
  // the slack past the capacity: a guard pattern the step must leave alone
  // (sp's slack already holds the removed-species code)
  for (int b = 0; b < 2; ++b) {
    CK(cudaMemsetAsync(c->pos[b] + want, 0xA5, (size_t)(cap - want) * sizeof(uint32_t), c->s), "guard");
    CK(cudaMemsetAsync(c->u[b] + want, 0xA5, (size_t)(cap - want) * sizeof(float), c->s), "guard");
    CK(cudaMemsetAsync(c->w[b] + want, 0xA5, (size_t)(cap - want) * sizeof(float), c->s), "guard");
    CK(cudaMemsetAsync(c->id[b] + want, 0xA5, (size_t)(cap - want) * sizeof(uint64_t), c->s), "guard");
  }
  if (!c->guard_arrays) CK(dalloc(&c->guard_arrays, 10), "guard");
  if (!c->guard_widths) CK(dalloc(&c->guard_widths, 10), "guard");
  const uint8_t* arrays[10];
  int widths[10];
  for (int b = 0; b < 2; ++b) {
    arrays[5 * b + 0] = reinterpret_cast<const uint8_t*>(c->pos[b]); widths[5 * b + 0] = 4;
    arrays[5 * b + 1] = reinterpret_cast<const uint8_t*>(c->u[b]); widths[5 * b + 1] = 4;
    arrays[5 * b + 2] = reinterpret_cast<const uint8_t*>(c->w[b]); widths[5 * b + 2] = 4;
    arrays[5 * b + 3] = c->sp[b]; widths[5 * b + 3] = 1;
    arrays[5 * b + 4] = reinterpret_cast<const uint8_t*>(c->id[b]); widths[5 * b + 4] = 8;
  }
  CK(cudaMemcpyAsync(c->guard_arrays, arrays, sizeof(arrays), cudaMemcpyHostToDevice, c->s), "guard");
  CK(cudaMemcpyAsync(c->guard_widths, widths, sizeof(widths), cudaMemcpyHostToDevice, c->s), "guard");
  CK(cudaStreamSynchronize(c->s), "guard");
#endif
  return PIC1D_OK;
}

DevParams dev_params(pic1d_ctx* c) {
  const pic1d_params& p = c->p;
  DevParams P{};
  P.N = c->N;
  P.F = c->F;
  P.top = (long long)c->N << c->F;
  P.top1 = (uint32_t)(P.top - 1);
  P.inv2F = std::ldexp(1.0f, -c->F);
  P.dt = (float)c->dt;
  P.half_dt = (float)(0.5 * c->dt);
  const float qm[4] = {-1.0f, 1.0f, (float)(1.0 / p.mass_ratio), -1.0f};
  const int qs[4] = {-1, 1, 1, -1};
  const float ms[4] = {1.0f, 1.0f, (float)p.mass_ratio, 1.0f};
  for (int k = 0; k < 4; ++k) { P.qm[k] = qm[k]; P.qs[k] = qs[k]; P.mass[k] = ms[k]; }
  P.drag_law = p.drag_law;
  P.rics_mode = p.rics_mode;
  P.mc_on = p.mc_on;
  P.pairs_on = p.pairs_on;
  P.limiter_on = c->tau_min > 0.0;
  P.use_nmax = p.n_max_ppc > 0.0;
  P.drag_k = (float)(p.drag_scale / c->R_cells);
  P.tau_min = (float)c->tau_min;
  P.damp = c->tau_min > 0.0 ? (float)std::exp(-c->dt / (2.0 * c->tau_min)) : 1.0f;
  P.pair_e_thr = (float)p.pair_energy_threshold;
  P.nmax_int = P.use_nmax ? (long long)std::floor(p.n_max_ppc * 4096.0) : 0;
  P.Ng = p.table_n_gamma;
  P.Ns = p.table_n_s;
  const double dg = p.table_log10g_max / (p.table_n_gamma - 1);
  P.t_scale = (float)(std::log10(2.0) / dg);
  P.dtdu_scale = (float)(1.0 / (std::log(10.0) * dg));
  P.v_scale = (float)((double)(p.table_n_s - 1) / ((double)P.top));
  const double th = p.kT_keV / kMeKeV;
  P.theta_T = (float)th;
  P.closedK = (float)(kRe * p.r_star_cm / (kLbar * kLbar) * th * th * th / 4.0);
  P.closedN = (float)(kRe * p.r_star_cm / (kLbar * kLbar) / 4.0);
  P.key0 = (uint32_t)p.seed;
  P.key1 = (uint32_t)(p.seed >> 32);
  P.step = c->step;
  const int b = c->cur;
  P.pos = c->pos[b]; P.u = c->u[b]; P.w = c->w[b]; P.sp = c->sp[b]; P.id = c->id[b];
  P.E32 = c->E32;
  P.J = c->J;
  P.tpair = c->tpair;
  P.nb = c->nb; P.nmu = c->nmu; P.nx = c->nx;
  P.nmu2 = c->nmu2;
  P.zone = c->zone;
  P.dens_flag = c->dens_flag;
  P.fast_cell = c->fast_cell;
  P.cflag = c->cflag;
  P.dflag = c->dflag;
  P.G32 = c->G32;
  P.atmo_flag = c->atmo_flag;
  P.atmo_w = c->atmo_w;
  P.jcum = c->jcum;
  P.check = c->check;
  P.dens_cur = c->dens[c->step & 1];
  P.dens_next = c->dens[(c->step + 1) & 1];
  P.cap = c->cap;
  P.ctr = c->ctr;
  P.st = c->st;
  P.ke_partial = c->ke_partial;
  P.sur_img = c->sur.img;
  P.sur_small = c->sur.small;
  P.sur_G = (float)p.table_log10g_max;
  P.sur_lnP = (float)std::log(kRe * p.r_star_cm / (4.0 * kLbar * kLbar));
  P.sur_err = c->sur.err;
  return P;
}

int validate(const pic1d_params* p, std::string& why) {
  auto bad = [&](const char* m) { why = m; return PIC1D_EINVAL; };
  if (!p) return bad("params is NULL");
  if (!(p->r_eq > 1.0)) return bad("r_eq must exceed 1 (the line must leave the star)");
  if (p->n_cells < 8 || p->n_cells > (1 << 24)) return bad("n_cells must be in [8, 2^24]");
  if (!(p->cfl > 0.0 && p->cfl < 1.0)) return bad("cfl must be in (0, 1)");
  if (p->ppc_e < 0 || p->ppc_p < 0 || p->ppc_i < 0 || p->ppc_e > 4096)
    return bad("ppc_e, ppc_p, ppc_i must be in [0, 4096]");
  if (p->ppc_e > 0) {
    if (p->ppc_p + p->ppc_i != p->ppc_e) return bad("the initial load needs ppc_p + ppc_i = ppc_e (neutral nodes)");
    if (!(p->init_multiplicity > 1.0)) return bad("init_multiplicity must exceed 1 (drift beta = 1/M)");
    if (!(p->u_sigma >= 0.0)) return bad("u_sigma must be >= 0");
    if ((long long)p->n_cells * 2 * p->ppc_e >= (1ll << 31)) return bad("the initial load exceeds 2^31 particles");
  }
  if (!(p->b_star > 0.0)) return bad("b_star must be positive");
  if (p->b_convention != 0 && p->b_convention != 1) return bad("b_convention must be 0 or 1");
  if (!(p->kT_keV > 0.0)) return bad("kT_keV must be positive");
  if (p->photon_model != PIC1D_PHOTON_RADIAL && p->photon_model != PIC1D_PHOTON_DISK) return bad("bad photon_model");
  if (p->drag_law < PIC1D_DRAG_OFF || p->drag_law > PIC1D_DRAG_SURROGATE) return bad("bad drag_law");
  if (p->drag_law == PIC1D_DRAG_TABLE && (p->table_n_gamma < 2 || p->table_n_s < 2 || p->table_n_gamma > 65536 ||
                                          p->table_n_s > 65536 || !(p->table_log10g_max > 0.0)))
    return bad("bad table shape");
  if (p->photon_model == PIC1D_PHOTON_DISK && (p->quad_n_mu < 1 || p->quad_n_mu > 256 || p->quad_n_phi < 1))
    return bad("bad quadrature node counts");
  if (p->rics_mode != PIC1D_RICS_SPLIT && p->rics_mode != PIC1D_RICS_DRAG_PLUS_PAIRS) return bad("bad rics_mode");
  if (!(p->cells_per_skin_depth > 0.0) || !(p->n0_ppc > 0.0) || !(p->j_psi >= 0.0)) return bad("bad plasma scales");
  if (!(p->mass_ratio > 0.0)) return bad("mass_ratio must be positive");
  if (p->inject_mode != PIC1D_INJECT_NONE && p->inject_mode != PIC1D_INJECT_RATE &&
      p->inject_mode != PIC1D_INJECT_TOPUP)
    return bad("bad inject_mode");
  if (p->inject_mode == PIC1D_INJECT_TOPUP) {
    if (!(p->atmo_a0 > 0.0) || !(p->atmo_h > 0.0) || !(p->atmo_ncut > 0.0) || !(p->inject_T >= 0.0))
      return bad("TOPUP needs atmo_a0, atmo_h, atmo_ncut > 0 and inject_T >= 0");
  }
  if (p->annihilate_every < 0) return bad("annihilate_every must be >= 0");
  if (p->annihilate_every > 0 && !(p->n_max_ppc > 0.0)) return bad("annihilation needs n_max_ppc > 0");
  if (p->sort_every < 1) return bad("sort_every must be >= 1");
  if (p->capacity < 0 || p->capacity > PIC1D_MAX_SLOTS) return bad("capacity must be in [0, PIC1D_MAX_SLOTS]");
  if ((long long)p->n_cells * ((long long)p->ppc_e + p->ppc_p + p->ppc_i) > PIC1D_MAX_SLOTS)
    return bad("the initial load exceeds PIC1D_MAX_SLOTS particles");
  if (!(p->r_star_cm > 0.0)) return bad("r_star_cm must be positive");
  return PIC1D_OK;
}

int build_tables(pic1d_ctx* c) {
  const pic1d_params& p = c->p;
  const int N = c->N;
  Line line(p.r_eq);
  c->L_R = line.L;
  c->R_cells = N / line.L;
  std::vector<float> hb(N + 1), hmu(N + 1), hx(N + 1);
  std::vector<uint8_t> hz(N), ha(N, 0);
  std::vector<float> hg(N, 0.0f);
  std::vector<int> acells;
  std::vector<long long> atarget;
  const bool topup = p.inject_mode == PIC1D_INJECT_TOPUP;
  double guess = line.th0;
  for (int k = 0; k <= N; ++k) {
    const double th = line.theta_of(line.L * (double)k / N, guess);
    guess = th;
    double x, b, mu;
    field_at(p, th, x, b, mu);
    hb[k] = (float)b; hmu[k] = (float)mu; hx[k] = (float)x;
  }
  guess = line.th0;
  for (int cc = 0; cc < N; ++cc) {
    const double th = line.theta_of(line.L * (cc + 0.5) / N, guess);
    guess = th;
    double x, b, mu;
    field_at(p, th, x, b, mu);
    hz[cc] = (b > p.b_pair_threshold) ? 1 : 0;
    if (topup) {
      // Eq. densprofile with r - R_star in cells; hydrostatic gravity -T/h along r
      const double n_rel = p.atmo_a0 * std::exp(-(x - 1.0) * c->R_cells / p.atmo_h);
      if (n_rel >= p.atmo_ncut) {
        ha[cc] = 1;
        hg[cc] = (float)(-(p.inject_T / p.atmo_h) * mu);
        acells.push_back(cc);
        atarget.push_back((long long)std::floor(n_rel * p.n0_ppc * 4096.0));
      }
    }
  }
  CK(dalloc(&c->nb, N + 1), "alloc nodes");
  CK(dalloc(&c->nmu, N + 1), "alloc nodes");
  CK(dalloc(&c->nx, N + 1), "alloc nodes");
  CK(dalloc(&c->zone, N), "alloc zone");
  std::vector<uint8_t> hf(N);
  for (int cc = 0; cc < N; ++cc)
    hf[cc] = hz[cc] | (cc > 0 ? hz[cc - 1] : 0) | (cc + 1 < N ? hz[cc + 1] : 0);
  CK(dalloc(&c->dens_flag, N), "alloc zone");
  CK(cudaMemcpyAsync(c->dens_flag, hf.data(), N, cudaMemcpyHostToDevice, c->s), "copy zone");
  // fast cells: no zone or atmosphere cell within two cells, not an end cell
  std::vector<uint8_t> hq(N);
  for (int cc = 0; cc < N; ++cc) {
    bool ok = cc >= 1 && cc <= N - 2;
    for (int d = -2; d <= 2 && ok; ++d) {
      const int k = cc + d;
      if (k >= 0 && k < N && (hz[k] || ha[k])) ok = false;
    }
    hq[cc] = ok ? 1 : 0;
  }
  if (topup) {
    c->n_atmo = (int)acells.size();
    CK(dalloc(&c->G32, N), "alloc atmosphere");
    CK(dalloc(&c->atmo_flag, N), "alloc atmosphere");
    CK(dalloc(&c->atmo_w, N), "alloc atmosphere");
    CK(dalloc(&c->atmo_cells, std::max<size_t>(acells.size(), 1)), "alloc atmosphere");
    CK(dalloc(&c->atmo_target, std::max<size_t>(atarget.size(), 1)), "alloc atmosphere");
    CK(cudaMemcpyAsync(c->G32, hg.data(), N * sizeof(float), cudaMemcpyHostToDevice, c->s), "copy atmosphere");
    CK(cudaMemcpyAsync(c->atmo_flag, ha.data(), N, cudaMemcpyHostToDevice, c->s), "copy atmosphere");
    if (!acells.empty()) {
      CK(cudaMemcpyAsync(c->atmo_cells, acells.data(), acells.size() * sizeof(int), cudaMemcpyHostToDevice, c->s),
         "copy atmosphere");
      CK(cudaMemcpyAsync(c->atmo_target, atarget.data(), atarget.size() * sizeof(long long),
                         cudaMemcpyHostToDevice, c->s),
         "copy atmosphere");
    }
    CK(cudaStreamSynchronize(c->s), "copy atmosphere");
  }
  CK(dalloc(&c->fast_cell, N), "alloc zone");
  CK(cudaMemcpyAsync(c->fast_cell, hq.data(), N, cudaMemcpyHostToDevice, c->s), "copy zone");
  // cell flags of the streaming push
  std::vector<uint8_t> hc(N);
  for (int cc = 0; cc < N; ++cc)
    hc[cc] = (uint8_t)((hz[cc] ? CF_ZONE : 0) | ((cc == 0 || cc == N - 1) ? CF_WALL : 0) |
                       ((hf[cc] || (cc > 0 && hf[cc - 1]) || (cc + 1 < N && hf[cc + 1])) ? CF_DENSN : 0) |
                       ((ha[cc] || (cc > 0 && ha[cc - 1]) || (cc + 1 < N && ha[cc + 1])) ? CF_ATMO : 0));
  CK(dalloc(&c->cflag, N), "alloc zone");
  CK(cudaMemcpyAsync(c->cflag, hc.data(), N, cudaMemcpyHostToDevice, c->s), "copy zone");
  std::vector<float2> hm2(N);
  for (int cc = 0; cc < N; ++cc) hm2[cc] = make_float2(hmu[cc], hmu[cc + 1]);
  CK(dalloc(&c->nmu2, N), "alloc nodes");
  CK(cudaMemcpyAsync(c->nmu2, hm2.data(), N * sizeof(float2), cudaMemcpyHostToDevice, c->s), "copy nodes");
  CK(cudaStreamSynchronize(c->s), "copy nodes");
  CK(cudaStreamSynchronize(c->s), "copy zone");
  CK(cudaMemcpyAsync(c->nb, hb.data(), (N + 1) * sizeof(float), cudaMemcpyHostToDevice, c->s), "copy nodes");
  CK(cudaMemcpyAsync(c->nmu, hmu.data(), (N + 1) * sizeof(float), cudaMemcpyHostToDevice, c->s), "copy nodes");
  CK(cudaMemcpyAsync(c->nx, hx.data(), (N + 1) * sizeof(float), cudaMemcpyHostToDevice, c->s), "copy nodes");
  CK(cudaMemcpyAsync(c->zone, hz.data(), N, cudaMemcpyHostToDevice, c->s), "copy zone");
  CK(cudaStreamSynchronize(c->s), "sync nodes");

  // the table law's table; a SURROGATE line keeps one as the network's
  // fallback outside its training box
  if (p.drag_law == PIC1D_DRAG_TABLE || p.drag_law == PIC1D_DRAG_SURROGATE) {
    const int Ns = p.table_n_s, Ng = p.table_n_gamma;
    std::vector<double> xs(Ns), bs(Ns), ms(Ns);
    guess = line.th0;
    for (int j = 0; j < Ns; ++j) {
      const double th = line.theta_of(line.L * (double)j / (Ns - 1), guess);
      guess = th;
      field_at(p, th, xs[j], bs[j], ms[j]);
    }
    std::vector<double> gx, gw;
    legendre_nodes(std::max(1, p.quad_n_mu), gx, gw);
    // the quadrature's inputs, freed on every way out
    double *dxs = nullptr, *dbs = nullptr, *dms = nullptr, *dgx = nullptr, *dgw = nullptr;
    auto table_build = [&]() -> int {
      CK(dalloc(&dxs, Ns), "alloc quad");
      CK(dalloc(&dbs, Ns), "alloc quad");
      CK(dalloc(&dms, Ns), "alloc quad");
      CK(dalloc(&dgx, gx.size()), "alloc quad");
      CK(dalloc(&dgw, gw.size()), "alloc quad");
      CK(cudaMemcpyAsync(dxs, xs.data(), Ns * sizeof(double), cudaMemcpyHostToDevice, c->s), "copy quad");
      CK(cudaMemcpyAsync(dbs, bs.data(), Ns * sizeof(double), cudaMemcpyHostToDevice, c->s), "copy quad");
      CK(cudaMemcpyAsync(dms, ms.data(), Ns * sizeof(double), cudaMemcpyHostToDevice, c->s), "copy quad");
      CK(cudaMemcpyAsync(dgx, gx.data(), gx.size() * sizeof(double), cudaMemcpyHostToDevice, c->s), "copy quad");
      CK(cudaMemcpyAsync(dgw, gw.data(), gw.size() * sizeof(double), cudaMemcpyHostToDevice, c->s), "copy quad");
      CK(dalloc(&c->table, (size_t)2 * Ns * Ng), "alloc table");
      const double pref = kRe * p.r_star_cm / (4.0 * kPi * kLbar * kLbar);
      CK(launch_table(Ng, Ns, p.quad_n_mu, p.quad_n_phi, p.table_log10g_max, p.kT_keV / kMeKeV, pref, dxs, dbs,
                      dms, dgx, dgw, p.photon_model, c->table, c->s),
         "table kernel");
      CK(dalloc(&c->tpair, (size_t)2 * (Ns - 1) * Ng), "alloc table");
      CK(launch_pair_table(c->table, Ng, Ns, c->tpair, c->s), "pair table");
      if (p.drag_law == PIC1D_DRAG_TABLE) {
        // where the limiter test is certain (the push skips its lookup), and
        // where no lepton can scatter (the Monte-Carlo step skips its rate)
        const DevParams Q = dev_params(c);
        CK(dalloc(&c->dflag, (size_t)2 * (Ns - 1) * kDampNE), "alloc damping flags");
        CK(launch_damp_flags(c->tpair, Ng, Ns, Q.t_scale, Q.drag_k, Q.tau_min, Q.dt, c->dflag, c->s),
           "damping flags");
      }
      CK(cudaStreamSynchronize(c->s), "table sync");
      return PIC1D_OK;
    };
    const int rc = table_build();
    if (rc != PIC1D_OK) cudaStreamSynchronize(c->s);
    dfree(dxs); dfree(dbs); dfree(dms); dfree(dgx); dfree(dgw);
    if (rc != PIC1D_OK) return rc;
  }
  return PIC1D_OK;
}

int do_sort(pic1d_ctx* c) {
  Nvtx range("sort");
  DevParams P = dev_params(c);
  const int o = 1 - c->cur;
  CK(launch_sort(P, c->counts, c->offsets, c->bsum, c->pos[o], c->u[o], c->w[o], c->sp[o], c->id[o], c->sms,
                 c->s),
     "sort");
  c->cur = o;
  return PIC1D_OK;
}

// The initial plasma of Sec. 3 (pic1d_params' recipe): thread (c, k) writes
// electron k of cell c and the positron or ion on its position.  Positions in
// integer arithmetic from word 0 of Philox(c, k, 0, INIT); Gaussians by
// Box-Muller on words 1 and 2 of Philox(c, k, m, INIT).
__global__ void k_init_load(DevParams P, int ppc_e, int ppc_p, int ppc_i, float u_d, float sigma) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)P.N * ppc_e) return;
  const int c = (int)(t / ppc_e), k = (int)(t % ppc_e);
  const long long ne = (long long)P.N * ppc_e, np = (long long)P.N * ppc_p;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)k, 0u, kTagInit), P.key0, P.key1);
  const unsigned long long A = ((unsigned long long)k << 24) + (unsigned long long)(r.x >> 8);
  const unsigned long long frac = P.F >= 24 ? (A << (P.F - 24)) / (unsigned long long)ppc_e
                                            : A / ((unsigned long long)ppc_e << (24 - P.F));
  const uint32_t pos = (uint32_t)(((unsigned long long)c << P.F) + frac);
#pragma unroll 1
  for (int m = 0; m < 3; ++m) {
    long long slot;
    if (m == 0) slot = (long long)c * ppc_e + k;
    else if (m == 1 && k < ppc_p) slot = ne + (long long)c * ppc_p + k;
    else if (m == 2 && k >= ppc_p) slot = ne + np + (long long)c * ppc_i + (k - ppc_p);
    else continue;
    const uint4 q = m == 0 ? r : philox4x32_10(make_uint4((uint32_t)c, (uint32_t)k, (uint32_t)m, kTagInit), P.key0,
                                              P.key1);
    const float U1 = (float)((q.y >> 8) + 1u) * (1.0f / 16777216.0f);
    const float U2 = (float)(q.z >> 8) * (1.0f / 16777216.0f);
    const float g = sqrtf(-2.0f * logf(U1)) * cospif(2.0f * U2);
    const float drift = m == 0 ? -u_d : (m == 1 ? u_d : 0.0f);
    P.pos[slot] = pos;
    P.u[slot] = fmaf(sigma, g, drift);
    P.w[slot] = 1.0f;
    P.sp[slot] = m == 0 ? PIC1D_SP_ELECTRON : (m == 1 ? PIC1D_SP_POSITRON : PIC1D_SP_ION);
    P.id[slot] = (unsigned long long)slot;
  }
}

// Check a freshly loaded state (species in range, positions on the line) and
// accumulate the integer lepton weight of every cell that the pair cap reads.
// Leptons of one warp that share a cell (the usual case for states stored in
// cell order) add their weights in registers first and issue one atomic.
__global__ void k_load(DevParams P, long long n, long long top, int want_density, unsigned long long* bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  const bool in = i < n;
  const uint8_t s = in ? P.sp[i] : (uint8_t)PIC1D_SP_DEAD;
  const uint32_t x = in ? P.pos[i] : 0u;
  const bool badp = in && ((s > 3 && s != PIC1D_SP_DEAD) || (long long)x >= top);
  const unsigned bm = __ballot_sync(0xffffffffu, badp);
  if (bm && lane == 0) atomicAdd(bad, (unsigned long long)__popc(bm));
  if (!want_density) return;
  const bool lep = in && !badp && s != PIC1D_SP_DEAD && s != PIC1D_SP_ION;
  const int cell = lep ? min((int)(x >> P.F), P.N - 1) : -1;
  long long v = lep ? __float2ll_rn(P.w[i] * 4096.0f) : 0;
  const unsigned lm = __ballot_sync(0xffffffffu, lep);
  if (!lm) return;
  const int c0 = __shfl_sync(0xffffffffu, cell, __ffs(lm) - 1);
  if (__all_sync(0xffffffffu, !lep || cell == c0)) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_cur + c0), (unsigned long long)v);
  } else if (lep) {
    atomicAdd(reinterpret_cast<unsigned long long*>(P.dens_cur + cell), (unsigned long long)v);
  }
}

// pic1d_init's initial plasma: the particles, then the state a set_state of
// them leaves (step 0, E = 0, the pair cap's density)
int initial_load(pic1d_ctx* c) {
  const pic1d_params& p = c->p;
  const long long n = (long long)c->N * (p.ppc_e + p.ppc_p + p.ppc_i);
  const double beta_d = 1.0 / p.init_multiplicity;
  const double u_d = beta_d / std::sqrt(1.0 - beta_d * beta_d);
  c->cur = 0;
  DevParams P = dev_params(c);
  const long long threads = (long long)c->N * p.ppc_e;
  k_init_load<<<(unsigned)((threads + 255) / 256), 256, 0, c->s>>>(P, p.ppc_e, p.ppc_p, p.ppc_i, (float)u_d,
                                                                   (float)p.u_sigma);
  CK(cudaGetLastError(), "initial load");
  StepState st{};
  st.n_slots = n;
  CK(cudaMemcpyAsync(c->st, &st, sizeof(st), cudaMemcpyHostToDevice, c->s), "initial load");
  CK(cudaMemsetAsync(c->dens[0], 0, c->N * sizeof(long long), c->s), "initial load");
  CK(cudaMemsetAsync(c->dens[1], 0, c->N * sizeof(long long), c->s), "initial load");
  CK(cudaMemsetAsync(c->spc, 0, sizeof(unsigned long long), c->s), "initial load");
  const long long top = (long long)c->N << c->F;
  k_load<<<(unsigned)((n + 255) / 256), 256, 0, c->s>>>(P, n, top, p.n_max_ppc > 0.0 ? 1 : 0, c->spc);
  CK(cudaGetLastError(), "initial load");
  CK(cudaStreamSynchronize(c->s), "initial load");
  return PIC1D_OK;
}

// record the start event of one timed push launch and log the slot count it reads
int timing_begin(pic1d_ctx* c) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a), "timing");
  CK(cudaEventCreate(&b), "timing");
  c->ev.push_back(a);
  c->ev.push_back(b);
  const long long k = (long long)c->ev.size() / 2 - 1;
  if (k >= c->slot_log_cap) {
    long long ncap = std::max<long long>(1024, 2 * c->slot_log_cap);
    long long* nl = nullptr;
    CK(dalloc(&nl, ncap), "timing");
    if (c->slot_log) {
      CK(cudaMemcpyAsync(nl, c->slot_log, c->slot_log_cap * sizeof(long long), cudaMemcpyDeviceToDevice, c->s), "timing");
      CK(cudaStreamSynchronize(c->s), "timing");
      dfree(c->slot_log);
    }
    c->slot_log = nl;
    c->slot_log_cap = ncap;
  }
  CK(cudaMemcpyAsync(c->slot_log + k, &c->st->n_slots, sizeof(long long), cudaMemcpyDeviceToDevice, c->s), "timing");
  CK(cudaEventRecord(a, c->s), "timing");
  return PIC1D_OK;
}

// fold the recorded events into the totals (stream already synchronised)
int timing_collect(pic1d_ctx* c) {
  const long long k = (long long)c->ev.size() / 2;
  if (k == 0) return PIC1D_OK;
  std::vector<long long> slots(k);
  CK(cudaMemcpy(slots.data(), c->slot_log, k * sizeof(long long), cudaMemcpyDeviceToHost), "timing");
  for (long long i = 0; i < k; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]), "timing");
    c->timed_ms += ms;
    c->timed_slots += slots[i];
    c->timed += 1;
    cudaEventDestroy(c->ev[2 * i]);
    cudaEventDestroy(c->ev[2 * i + 1]);
  }
  c->ev.clear();
  return PIC1D_OK;
}

}  // namespace

extern "C" {

int pic1d_init(const pic1d_params* p, pic1d_ctx** out) {
  if (!out) return PIC1D_EINVAL;
  *out = nullptr;
  std::string why;
  if (validate(p, why) != PIC1D_OK) {
    std::fprintf(stderr, "pic1d_init: %s\n", why.c_str());
    return PIC1D_EINVAL;
  }
  pic1d_ctx* c = new pic1d_ctx();
  g_live.fetch_add(1);
  c->p = *p;
  c->s = reinterpret_cast<cudaStream_t>(p->cuda_stream);
  c->N = p->n_cells;
  c->F = fbits_of(p->n_cells);
  c->dt = p->cfl;
  const double n0 = p->n0_ppc;
  c->q_p = 1.0 / (4.0 * kPi * p->cells_per_skin_depth * p->cells_per_skin_depth * n0);
  c->j_ext = p->j_psi * n0 * c->q_p;
  c->tau_min = (p->eta_min > 0.0 && p->j_psi > 0.0) ? p->eta_min * std::sqrt(p->j_psi) * p->cells_per_skin_depth : 0.0;
  int rc = build_tables(c);
  const int N = c->N;
  if (rc == PIC1D_OK) {
    cudaError_t e = cudaSuccess;
    auto chain = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chain(dalloc(&c->E64, N));
    chain(dalloc(&c->E32, N));
    chain(dalloc(&c->J, N));
    chain(dalloc(&c->jcum, N));
#ifdef PIC1D_CHECK
    chain(dalloc(&c->check, 1));
    if (e == cudaSuccess) chain(cudaMemsetAsync(c->check, 0, sizeof(unsigned), c->s));
#endif
    chain(dalloc(&c->dens[0], N));
    chain(dalloc(&c->dens[1], N));
    chain(dalloc(&c->ctr, 1));
    chain(dalloc(&c->st, 1));
    chain(dalloc(&c->field_partial, 3 * kMaxFieldBlocks));
    chain(dalloc(&c->counts, sort_bins(N)));
    chain(dalloc(&c->offsets, sort_bins(N) + 1));
    chain(dalloc(&c->bsum, scan_blocks(N)));
    chain(dalloc(&c->spc, 4));
    if (p->annihilate_every > 0) {
      chain(dalloc(&c->ann_list, N));
      chain(dalloc(&c->ann_amount, N));
      chain(dalloc(&c->ann_count, 1));
    }
    int dev = 0, sms = 0;
    chain(cudaGetDevice(&dev));
    chain(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    c->sms = std::max(1, sms);
    chain(dalloc(&c->ke_partial, c->sms * 8));     // at most 8 blocks of 256 threads per SM
    c->push_variant = default_push_variant();
    c->push_grid = c->sms * push_blocks_per_sm(c->push_variant, p->n_max_ppc > 0.0);
    if (e == cudaSuccess) {
      chain(cudaMemsetAsync(c->E64, 0, N * sizeof(double), c->s));
      chain(cudaMemsetAsync(c->E32, 0, N * sizeof(float), c->s));
      chain(cudaMemsetAsync(c->J, 0, N * sizeof(long long), c->s));
      chain(cudaMemsetAsync(c->jcum, 0, N * sizeof(long long), c->s));
      chain(cudaMemsetAsync(c->dens[0], 0, N * sizeof(long long), c->s));
      chain(cudaMemsetAsync(c->dens[1], 0, N * sizeof(long long), c->s));
      chain(cudaMemsetAsync(c->ctr, 0, sizeof(Counters), c->s));
      chain(cudaMemsetAsync(c->st, 0, sizeof(StepState), c->s));
      chain(cudaMemsetAsync(c->ke_partial, 0, c->sms * 8 * sizeof(double), c->s));
    }
    if (e != cudaSuccess) rc = cuda_fail(c, e, "init");
  }
  if (rc == PIC1D_OK) {
    const long long n_load = (long long)p->n_cells * (p->ppc_e + p->ppc_p + p->ppc_i);
    const long long want = p->capacity > 0 ? std::max<long long>(p->capacity, n_load)
                                           : std::min<long long>(n_load > 0 ? 2 * n_load + 4 * kTile : 4 * kTile,
                                                                 PIC1D_MAX_SLOTS);
    rc = alloc_particles(c, want);
  }
  if (rc == PIC1D_OK && p->ppc_e > 0) rc = initial_load(c);
  if (rc == PIC1D_OK) {
    cudaError_t e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "init sync");
  }
  if (rc != PIC1D_OK) {
    std::fprintf(stderr, "pic1d_init: %s\n", c->err.c_str());
    pic1d_free(c);
    return rc;
  }
  *out = c;
  return PIC1D_OK;
}

int pic1d_set_state(pic1d_ctx* c, int64_t n, const uint32_t* pos, const float* u, const float* w,
                    const uint8_t* sp, const uint64_t* id, const double* E, int64_t step, int mem) {
  if (!c) return PIC1D_EINVAL;
  if (n < 0 || (n > 0 && (!pos || !u || !w || !sp || !id)) || (mem != 0 && mem != 1) || step < 0)
    return fail(c, PIC1D_EINVAL, "set_state: bad arguments");
  const long long top = (long long)c->N << c->F;
  if (n > PIC1D_MAX_SLOTS) return fail(c, PIC1D_EINVAL, "set_state: more than PIC1D_MAX_SLOTS particles");
  const long long want = c->p.capacity > 0 ? std::max<long long>(c->p.capacity, n)
                                           : std::min<long long>(2 * n + 4 * kTile, PIC1D_MAX_SLOTS);
  if (n > c->cap || (c->p.capacity == 0 && c->cap < want)) {
    int rc = alloc_particles(c, want);
    if (rc != PIC1D_OK) return rc;
  }
  c->cur = 0;
  const cudaMemcpyKind k = mem ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n > 0) {
    CK(cudaMemcpyAsync(c->pos[0], pos, n * sizeof(uint32_t), k, c->s), "set_state pos");
    CK(cudaMemcpyAsync(c->u[0], u, n * sizeof(float), k, c->s), "set_state u");
    CK(cudaMemcpyAsync(c->w[0], w, n * sizeof(float), k, c->s), "set_state w");
    CK(cudaMemcpyAsync(c->sp[0], sp, n * sizeof(uint8_t), k, c->s), "set_state sp");
    CK(cudaMemcpyAsync(c->id[0], id, n * sizeof(uint64_t), k, c->s), "set_state id");
  }
  CK(cudaMemsetAsync(c->sp[0] + n, PIC1D_SP_DEAD, (size_t)(c->alloc - n), c->s), "set_state tail");
  if (E) {
    std::vector<float> e32;
    CK(cudaMemcpyAsync(c->E64, E, c->N * sizeof(double), k, c->s), "set_state E");
    std::vector<double> h(c->N);
    if (mem == 0) std::memcpy(h.data(), E, c->N * sizeof(double));
    else CK(cudaMemcpyAsync(h.data(), E, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->s), "set_state E");
    CK(cudaStreamSynchronize(c->s), "set_state E");
    e32.resize(c->N);
    for (int i = 0; i < c->N; ++i) e32[i] = (float)h[i];
    CK(cudaMemcpyAsync(c->E32, e32.data(), c->N * sizeof(float), cudaMemcpyHostToDevice, c->s), "set_state E32");
    CK(cudaStreamSynchronize(c->s), "set_state E32");
  } else {
    CK(cudaMemsetAsync(c->E64, 0, c->N * sizeof(double), c->s), "set_state E");
    CK(cudaMemsetAsync(c->E32, 0, c->N * sizeof(float), c->s), "set_state E");
  }
  CK(cudaMemsetAsync(c->J, 0, c->N * sizeof(long long), c->s), "set_state J");
  c->gauss_on = false;                   // a new state: the continuity mark no longer applies
  c->step = step;
  StepState st{};
  st.n_slots = n;
  st.step = step;
  CK(cudaMemcpyAsync(c->st, &st, sizeof(st), cudaMemcpyHostToDevice, c->s), "set_state st");
  CK(cudaMemsetAsync(c->dens[0], 0, c->N * sizeof(long long), c->s), "set_state dens");
  CK(cudaMemsetAsync(c->dens[1], 0, c->N * sizeof(long long), c->s), "set_state dens");
  if (n > 0) {
    // validation of the copied state, fused with the pair-cap density
    unsigned long long* bad = c->spc;
    CK(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), c->s), "set_state validate");
    DevParams P = dev_params(c);
    k_load<<<(unsigned)((n + 255) / 256), 256, 0, c->s>>>(P, n, top, c->p.n_max_ppc > 0.0 ? 1 : 0, bad);
    CK(cudaGetLastError(), "set_state validate");
    unsigned long long hb = 0;
    CK(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, c->s), "set_state validate");
    CK(cudaStreamSynchronize(c->s), "set_state validate");
    if (hb) {
      // leave an empty line rather than a half-loaded one
      StepState empty{};
      CK(cudaMemcpyAsync(c->st, &empty, sizeof(empty), cudaMemcpyHostToDevice, c->s), "set_state reset");
      CK(cudaMemsetAsync(c->sp[0], PIC1D_SP_DEAD, (size_t)c->alloc, c->s), "set_state reset");
      CK(cudaMemsetAsync(c->dens[0], 0, c->N * sizeof(long long), c->s), "set_state reset");
      CK(cudaMemsetAsync(c->dens[1], 0, c->N * sizeof(long long), c->s), "set_state reset");
      CK(cudaStreamSynchronize(c->s), "set_state reset");
      return fail(c, PIC1D_EINVAL, "set_state: " + std::to_string(hb) + " particles with bad species or position "
                                   "(the line is left empty)");
    }
  }
  CK(cudaStreamSynchronize(c->s), "set_state sync");
  return PIC1D_OK;
}

int pic1d_step(pic1d_ctx* c, int n_steps) {
  if (!c) return PIC1D_EINVAL;
  Nvtx range("pic1d_step");
  if (n_steps < 0) return fail(c, PIC1D_EINVAL, "step: n_steps < 0");
  const pic1d_params& p = c->p;
  const double four_pi = 4.0 * kPi;
  const double a = four_pi * c->dt * c->j_ext;
  const double cJ = four_pi * c->q_p * std::ldexp(1.0, -c->F - kWBits);
  const double dt_jext = c->dt * c->j_ext;
  const double carriers = p.j_psi * p.n0_ppc * c->dt;     // j_ext dt / q_p carriers of weight 1
  const float sig_e = (float)std::sqrt(p.inject_T), sig_i = (float)std::sqrt(p.inject_T / p.mass_ratio);
  const bool sur_law = p.drag_law == PIC1D_DRAG_SURROGATE;
  if (sur_law && !c->sur_on) return fail(c, PIC1D_EINVAL, "step: drag law SURROGATE without a network (set or train it)");
  for (int k = 0; k < n_steps; ++k) {
    DevParams P = dev_params(c);
    CK(cudaMemsetAsync(c->J, 0, c->N * sizeof(long long), c->s), "clear J");
    CK(cudaMemsetAsync(&c->st->work, 0, sizeof(unsigned long long), c->s), "clear schedule");
    if (c->atmo_w) CK(cudaMemsetAsync(c->atmo_w, 0, c->N * sizeof(long long), c->s), "clear atmosphere");
    if (c->timing) {
      int rc = timing_begin(c);
      if (rc != PIC1D_OK) return rc;
    }
    int grid = c->push_grid;
    {
      Nvtx push_range("push");
      if (sur_law) {
        grid = c->sms * kSurPushPerSm;
        CK(launch_push_sur(P, grid, c->s), "push");
      } else {
        CK(launch_push(P, c->push_variant, c->push_grid, c->s), "push");
      }
    }
    if (c->timing) CK(cudaEventRecord(c->ev.back(), c->s), "timing");
    if (p.inject_mode == PIC1D_INJECT_RATE) CK(launch_inject(P, carriers, sig_e, sig_i, c->s), "inject");
    if (p.inject_mode == PIC1D_INJECT_TOPUP)
      CK(launch_topup(P, c->atmo_cells, c->atmo_target, c->n_atmo, sig_e, sig_i, c->s), "top-up");
    {
      Nvtx field_range("field");
      CK(launch_field(P, c->E64, c->E32, a, cJ, dt_jext, c->field_partial, grid, c->s), "field");
    }
    c->step += 1;
    const bool ann = p.annihilate_every > 0 && c->step % p.annihilate_every == 0;
    if (c->step % p.sort_every == 0 || ann) {
      int rc = do_sort(c);
      if (rc != PIC1D_OK) return rc;
    }
    if (ann) {
      Nvtx ann_range("annihilate");
      const DevParams Q = dev_params(c);     // the sorted buffer, the step just finished
      CK(launch_annihilate(Q, c->counts, c->offsets, c->ann_list, c->ann_amount, c->ann_count, c->E64, c->E32, cJ,
                           c->sms, c->s),
         "annihilate");
    }
#ifdef PIC1D_CHECK
    // checking build: the slack past the particle arrays is intact
    if (c->guard_arrays)
      CK(launch_guard_check(c->guard_arrays, c->guard_widths, 10, c->cap, c->alloc, c->check, c->s), "guard check");
#endif
  }
  return PIC1D_OK;
}

int pic1d_sort(pic1d_ctx* c) {
  if (!c) return PIC1D_EINVAL;
  return do_sort(c);
}

int64_t pic1d_slots(pic1d_ctx* c) {
  if (!c) return -1;
  StepState st{};
  if (cudaMemcpyAsync(&st, c->st, sizeof(st), cudaMemcpyDeviceToHost, c->s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(c->s) != cudaSuccess) return -1;
  return st.n_slots;
}

int pic1d_diag(pic1d_ctx* c, pic1d_diag_t* out) {
  if (!c || !out) return PIC1D_EINVAL;
  std::memset(out, 0, sizeof(*out));
  DevParams P = dev_params(c);
  CK(launch_count_species(P, c->spc, c->s), "diag count");
  Counters C{};
  StepState st{};
  unsigned long long spc[4];
  CK(cudaMemcpyAsync(&C, c->ctr, sizeof(C), cudaMemcpyDeviceToHost, c->s), "diag");
  CK(cudaMemcpyAsync(&st, c->st, sizeof(st), cudaMemcpyDeviceToHost, c->s), "diag");
  CK(cudaMemcpyAsync(spc, c->spc, sizeof(spc), cudaMemcpyDeviceToHost, c->s), "diag");
  CK(cudaStreamSynchronize(c->s), "diag sync");
  out->step = c->step;
  out->n_slots = st.n_slots;
  for (int k = 0; k < 4; ++k) out->n_alive[k] = (int64_t)spc[k];
  out->pairs_created = C.pairs_created;
  out->pairs_dropped_cap = C.pairs_dropped_cap;
  out->pairs_rejected_nmax = C.pairs_rejected_nmax;
  out->pairs_lost_wall = C.pairs_lost_wall;
  out->lost_north = C.lost_north;
  out->lost_south = C.lost_south;
  out->injected = C.injected;
  out->injected_dropped = C.injected_dropped;
  out->scatters = C.scatters;
  out->psc_clamped = C.psc_clamped;
  out->limiter_branch = C.limiter_branch;
  out->newton_branch = C.newton_branch;
  out->nonfinite = C.nonfinite;
  out->rng_draws = C.rng_draws;
  out->annihilated = (int64_t)C.annihilated;
  out->sur_rows = C.sur_rows;
  out->sur_rows_tangent = C.sur_rows_tangent;
  {
    int rc = timing_collect(c);
    if (rc != PIC1D_OK) return rc;
  }
  out->push_launches = c->timed;
  out->push_ms = c->timed_ms;
  out->push_slots = c->timed_slots;
  out->field_energy = st.field_energy;
  out->kinetic_energy = st.kinetic * c->q_p;
  out->ext_work = st.ext_work;
  out->vc = st.vc;
  out->ke_lost = st.ke_lost * c->q_p;
  out->q_p = c->q_p;
  out->j_ext = c->j_ext;
  out->dt = c->dt;
  out->tau_min = c->tau_min;
  out->R_cells = c->R_cells;
  out->L_Rstar = c->L_R;
  out->fbits = c->F;
  out->push_variant = c->push_variant;
  out->gauss_marked = c->gauss_on ? 1 : 0;
  out->gauss_residual_max = -1;
  out->gauss_residual_node = -1;
  if (c->gauss_on) {
    CK(cudaMemsetAsync(c->rho, 0, sizeof(long long) * (c->N + 1), c->s), "diag continuity");
    CK(launch_rho(P, c->rho, c->sms * 8, c->s), "diag continuity");
    CK(launch_gauss_residual(P, c->rho, c->rho_ref, c->gauss_out, c->s), "diag continuity");
    unsigned long long g[2];
    CK(cudaMemcpyAsync(g, c->gauss_out, sizeof(g), cudaMemcpyDeviceToHost, c->s), "diag continuity");
    CK(cudaStreamSynchronize(c->s), "diag continuity");
    out->gauss_residual_max = (int64_t)g[0];
    out->gauss_residual_node = g[1] == ~0ull ? -1 : (int64_t)g[1];
  }
  int status = PIC1D_OK;
#ifdef PIC1D_CHECK
  if (c->check) {
    unsigned chk = 0;
    CK(cudaMemcpy(&chk, c->check, sizeof(chk), cudaMemcpyDeviceToHost), "diag check");
    if (chk) {
      char msg[160];
      std::snprintf(msg, sizeof(msg), "checking build: failed bounds 0x%x (1 cell, 2 slot, 4 gather, 8 sort "
                                      "destination, 16 sort key, 32 guard past the particle arrays)", chk);
      c->err = msg;
      out->status = PIC1D_ECHECK;
      return PIC1D_ECHECK;
    }
  }
#endif
  if (C.waits_timed_out) {
    // reported once: the count restarts, the context stays usable
    CK(cudaMemsetAsync(&c->ctr->waits_timed_out, 0, sizeof(unsigned long long), c->s), "diag");
    CK(cudaStreamSynchronize(c->s), "diag sync");
    c->err = "a push block's bounded wait on a bulk copy gave up (" + std::to_string(C.waits_timed_out) +
             " blocks)";
    out->status = PIC1D_ETIMEOUT;
    return PIC1D_ETIMEOUT;
  }
  if (C.nonfinite) status = PIC1D_ENUMERIC;
  else if (C.pairs_dropped_cap || C.injected_dropped) status = PIC1D_WCAPACITY;
  out->status = status;
  if (status == PIC1D_ENUMERIC) c->err = "a step met a non-finite momentum";
  return status;
}

int pic1d_get_fields(pic1d_ctx* c, double* E, int64_t* J, int mem) {
  if (!c || (mem != 0 && mem != 1)) return PIC1D_EINVAL;
  const cudaMemcpyKind k = mem ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (E) CK(cudaMemcpyAsync(E, c->E64, c->N * sizeof(double), k, c->s), "get E");
  if (J) CK(cudaMemcpyAsync(J, c->J, c->N * sizeof(long long), k, c->s), "get J");
  CK(cudaStreamSynchronize(c->s), "get_fields sync");
  return PIC1D_OK;
}

int pic1d_get_particles(pic1d_ctx* c, int64_t n, uint32_t* pos, float* u, float* w, uint8_t* sp, uint64_t* id,
                        int mem) {
  if (!c || n < 0 || (mem != 0 && mem != 1)) return PIC1D_EINVAL;
  const int64_t have = pic1d_slots(c);
  if (have < 0) return fail(c, PIC1D_ECUDA, "get_particles: slot count");
  if (n > have) return fail(c, PIC1D_EINVAL, "get_particles: n exceeds the used slots");
  const cudaMemcpyKind k = mem ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const int b = c->cur;
  if (n > 0) {
    if (pos) CK(cudaMemcpyAsync(pos, c->pos[b], n * sizeof(uint32_t), k, c->s), "get pos");
    if (u) CK(cudaMemcpyAsync(u, c->u[b], n * sizeof(float), k, c->s), "get u");
    if (w) CK(cudaMemcpyAsync(w, c->w[b], n * sizeof(float), k, c->s), "get w");
    if (sp) CK(cudaMemcpyAsync(sp, c->sp[b], n * sizeof(uint8_t), k, c->s), "get sp");
    if (id) CK(cudaMemcpyAsync(id, c->id[b], n * sizeof(uint64_t), k, c->s), "get id");
  }
  CK(cudaStreamSynchronize(c->s), "get_particles sync");
  return PIC1D_OK;
}

int pic1d_get_table(pic1d_ctx* c, float* out) {
  if (!c || !out) return PIC1D_EINVAL;
  if (!c->table) return fail(c, PIC1D_EINVAL, "get_table: drag_law is not TABLE");
  const size_t n = (size_t)2 * c->p.table_n_s * c->p.table_n_gamma;
  CK(cudaMemcpyAsync(out, c->table, n * sizeof(float2), cudaMemcpyDeviceToHost, c->s), "get table");
  CK(cudaStreamSynchronize(c->s), "get table sync");
  return PIC1D_OK;
}

int pic1d_deposit(pic1d_ctx* c, int64_t n, const int64_t* pos0, const int64_t* pos1, const float* w,
                  const uint8_t* sp, int64_t* J) {
  if (!c || n < 0 || (n > 0 && (!pos0 || !pos1 || !w || !sp || !J))) return PIC1D_EINVAL;
  DevParams P = dev_params(c);
  CK(launch_deposit(P, n, reinterpret_cast<const long long*>(pos0), reinterpret_cast<const long long*>(pos1), w, sp,
                    reinterpret_cast<long long*>(J), c->s),
     "deposit");
  CK(cudaStreamSynchronize(c->s), "deposit sync");
  return PIC1D_OK;
}

int pic1d_check_wait(pic1d_ctx* c, int64_t limit_clocks) {
  if (!c || limit_clocks < 1 || limit_clocks > (int64_t)4000000000ll) return PIC1D_EINVAL;
  CK(launch_wait_check(c->ctr, (long long)limit_clocks, c->s), "check wait");
  CK(cudaStreamSynchronize(c->s), "check wait");
  return PIC1D_OK;
}

int pic1d_set_variant(pic1d_ctx* c, int variant) {
  if (!c) return PIC1D_EINVAL;
  if (variant < 0 || variant >= push_variant_count()) return fail(c, PIC1D_EINVAL, "set_variant: no such variant");
  c->push_variant = variant;
  c->push_grid = c->sms * push_blocks_per_sm(variant, c->p.n_max_ppc > 0.0);
  return PIC1D_OK;
}

int pic1d_variant_info(int variant, int* particles_per_thread, int* min_blocks_per_sm) {
  if (variant < 0 || variant >= push_variant_count()) return PIC1D_EINVAL;
  if (particles_per_thread) *particles_per_thread = push_variant_ppt(variant);
  if (min_blocks_per_sm) *min_blocks_per_sm = push_variant_minb(variant);
  return push_variant_count();
}

int pic1d_timing(pic1d_ctx* c, int on) {
  if (!c) return PIC1D_EINVAL;
  CK(cudaStreamSynchronize(c->s), "timing sync");
  int rc = timing_collect(c);
  if (rc != PIC1D_OK) return rc;
  c->timing = on != 0;
  c->timed = 0;
  c->timed_ms = 0.0;
  c->timed_slots = 0;
  return PIC1D_OK;
}

// ------------------------------------------------------------- surrogate
namespace {

constexpr int kSurMaxTiles = 512;   // rows per gradient launch: 512 x 128

int sur_ensure(pic1d_ctx* c) {
  if (c->sur_on) return PIC1D_OK;
  SurBufs& B = c->sur;
  B.max_tiles = kSurMaxTiles;
  CK(dalloc(&B.master, W_N_PARAMS), "surrogate alloc");
  CK(dalloc(&B.m, W_N_PARAMS), "surrogate alloc");
  CK(dalloc(&B.v, W_N_PARAMS), "surrogate alloc");
  CK(dalloc(&B.img, 32768), "surrogate alloc");
  CK(dalloc(&B.small, 580), "surrogate alloc");
  CK(dalloc(&B.part, (size_t)kSurMaxTiles * W_N_PARAMS), "surrogate alloc");
  CK(dalloc(&B.loss_part, kSurMaxTiles), "surrogate alloc");
  CK(dalloc(&B.err, 1), "surrogate alloc");
  CK(dalloc(&c->sur_grad, W_N_PARAMS), "surrogate alloc");
  CK(dalloc(&c->sur_loss, 1), "surrogate alloc");
  CK(cudaMemsetAsync(B.master, 0, W_N_PARAMS * sizeof(float), c->s), "surrogate init");
  CK(cudaMemsetAsync(B.m, 0, W_N_PARAMS * sizeof(float), c->s), "surrogate init");
  CK(cudaMemsetAsync(B.v, 0, W_N_PARAMS * sizeof(float), c->s), "surrogate init");
  CK(cudaMemsetAsync(B.img, 0, 32768, c->s), "surrogate init");
  CK(cudaMemsetAsync(B.small, 0, 580 * sizeof(float), c->s), "surrogate init");
  CK(cudaMemsetAsync(B.err, 0, sizeof(unsigned), c->s), "surrogate init");
  std::vector<double> gx, gw;
  legendre_nodes(std::max(1, c->p.quad_n_mu), gx, gw);
  CK(dalloc(&c->sur_gx, gx.size()), "surrogate alloc");
  CK(dalloc(&c->sur_gw, gw.size()), "surrogate alloc");
  CK(cudaMemcpyAsync(c->sur_gx, gx.data(), gx.size() * sizeof(double), cudaMemcpyHostToDevice, c->s), "surrogate");
  CK(cudaMemcpyAsync(c->sur_gw, gw.data(), gw.size() * sizeof(double), cudaMemcpyHostToDevice, c->s), "surrogate");
  CK(cudaStreamSynchronize(c->s), "surrogate init");
  c->sur_on = true;
  return PIC1D_OK;
}

SurPhys sur_phys(const pic1d_ctx* c) {
  SurPhys Q;
  Q.theta_T = c->p.kT_keV / kMeKeV;
  Q.pref = kRe * c->p.r_star_cm / (4.0 * kPi * kLbar * kLbar);
  Q.log10g_max = c->p.table_log10g_max;
  Q.b_star = c->p.b_star;
  Q.b_convention = c->p.b_convention;
  Q.photon_model = c->p.photon_model;
  Q.n_mu = std::max(1, c->p.quad_n_mu);
  Q.n_phi = std::max(1, c->p.quad_n_phi);
  Q.gx = c->sur_gx;
  Q.gw = c->sur_gw;
  return Q;
}

// the error flag of the surrogate's kernels (bounded waits that gave up)
int sur_check(pic1d_ctx* c) {
  unsigned h = 0;
  CK(cudaMemcpyAsync(&h, c->sur.err, sizeof(h), cudaMemcpyDeviceToHost, c->s), "surrogate status");
  CK(cudaStreamSynchronize(c->s), "surrogate status");
  if (h) return fail(c, PIC1D_ETIMEOUT, "surrogate: a wait for the tensor cores gave up");
  return PIC1D_OK;
}

}  // namespace

int pic1d_sur_set_params(pic1d_ctx* c, const float* theta) {
  if (!c || !theta) return fail(c, PIC1D_EINVAL, "sur_set_params: NULL argument");
  int rc = sur_ensure(c);
  if (rc != PIC1D_OK) return rc;
  CK(cudaMemcpyAsync(c->sur.master, theta, W_N_PARAMS * sizeof(float), cudaMemcpyHostToDevice, c->s), "sur_set_params");
  CK(cudaMemsetAsync(c->sur.m, 0, W_N_PARAMS * sizeof(float), c->s), "sur_set_params");
  CK(cudaMemsetAsync(c->sur.v, 0, W_N_PARAMS * sizeof(float), c->s), "sur_set_params");
  CK(sur_launch_update(c->sur, 0, 2, 0.0f, 1, nullptr, nullptr, c->s), "sur_set_params");
  CK(cudaStreamSynchronize(c->s), "sur_set_params");
  c->sur_t = 0;
  return PIC1D_OK;
}

int pic1d_sur_get_params(pic1d_ctx* c, float* theta) {
  if (!c || !theta) return fail(c, PIC1D_EINVAL, "sur_get_params: NULL argument");
  int rc = sur_ensure(c);
  if (rc != PIC1D_OK) return rc;
  CK(cudaMemcpyAsync(theta, c->sur.master, W_N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, c->s), "sur_get_params");
  CK(cudaStreamSynchronize(c->s), "sur_get_params");
  return PIC1D_OK;
}

int pic1d_sur_samples(pic1d_ctx* c, uint64_t seed, uint64_t start, int64_t n, double r_lo, double r_hi,
                      float* out_dev) {
  if (!c) return PIC1D_EINVAL;
  if (n < 0 || (n > 0 && !out_dev) || !(r_lo >= 1.0) || !(r_hi >= r_lo))
    return fail(c, PIC1D_EINVAL, "sur_samples: bad arguments (need n >= 0, 1 <= r_lo <= r_hi)");
  int rc = sur_ensure(c);
  if (rc != PIC1D_OK) return rc;
  CK(sur_launch_samples(sur_phys(c), seed, start, n, r_lo, r_hi, out_dev, c->s), "sur_samples");
  CK(cudaStreamSynchronize(c->s), "sur_samples");
  return PIC1D_OK;
}

int pic1d_sur_grad(pic1d_ctx* c, const float* samples_dev, int64_t n, float* grad_host, double* loss_host) {
  if (!c) return PIC1D_EINVAL;
  if (!samples_dev || !grad_host || n < 1 || n > (int64_t)kSurMaxTiles * 128)
    return fail(c, PIC1D_EINVAL, "sur_grad: bad arguments (1 <= n <= 65536)");
  int rc = sur_ensure(c);
  if (rc != PIC1D_OK) return rc;
  const int tiles = (int)((n + 127) / 128);
  float* loss_d = c->sur_loss;
  CK(sur_launch_train(c->sur, samples_dev, n, 1, 0, 0, (int)n, c->s), "sur_grad");
  CK(sur_launch_update(c->sur, tiles, 0, 0.0f, 1, c->sur_grad, loss_d, c->s), "sur_grad");
  float hl = 0.0f;
  CK(cudaMemcpyAsync(grad_host, c->sur_grad, W_N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, c->s), "sur_grad");
  CK(cudaMemcpyAsync(&hl, loss_d, sizeof(float), cudaMemcpyDeviceToHost, c->s), "sur_grad");
  CK(cudaStreamSynchronize(c->s), "sur_grad");
  if (loss_host) *loss_host = (double)hl / (double)n;
  return sur_check(c);
}

int pic1d_sur_train_steps(pic1d_ctx* c, const float* samples_dev, int64_t n, int32_t batch, int32_t steps,
                          double lr) {
  if (!c) return PIC1D_EINVAL;
  if (!samples_dev || n < 1 || batch < 1 || batch > kSurMaxTiles * 128 || steps < 0 || !(lr > 0.0))
    return fail(c, PIC1D_EINVAL, "sur_train_steps: bad arguments");
  int rc = sur_ensure(c);
  if (rc != PIC1D_OK) return rc;
  const int tiles = (batch + 127) / 128;
  for (int k = 0; k < steps; ++k) {
    CK(sur_launch_train(c->sur, samples_dev, n, 1, 0, (long long)k * batch, batch, c->s), "sur_train_steps");
    CK(sur_launch_update(c->sur, tiles, 1, (float)lr, ++c->sur_t, nullptr, nullptr, c->s), "sur_train_steps");
  }
  CK(cudaStreamSynchronize(c->s), "sur_train_steps");
  return sur_check(c);
}

int pic1d_sur_infer(pic1d_ctx* c, const float* feat_dev, int32_t stride, int64_t n, float* out_dev) {
  if (!c) return PIC1D_EINVAL;
  if (n < 0 || stride < 4 || (n > 0 && (!feat_dev || !out_dev)))
    return fail(c, PIC1D_EINVAL, "sur_infer: bad arguments");
  int rc = sur_ensure(c);
  if (rc != PIC1D_OK) return rc;
  CK(sur_launch_infer(c->sur, feat_dev, stride, n, out_dev, c->sms, c->s), "sur_infer");
  CK(cudaStreamSynchronize(c->s), "sur_infer");
  return sur_check(c);
}

int pic1d_train_surrogate(pic1d_ctx* c, const pic1d_train_cfg* cfg, pic1d_train_report* rep) {
  if (!c) return PIC1D_EINVAL;
  Nvtx range("pic1d_train_surrogate");
  if (!cfg || !rep || cfg->n_samples < cfg->batch || cfg->batch < 128 || cfg->batch % 128 != 0 ||
      cfg->batch > kSurMaxTiles * 128 || cfg->epochs < 0 || !(cfg->lr > 0.0) || !(cfg->r_lo >= 1.0) ||
      !(cfg->r_hi >= cfg->r_lo) || cfg->n_val < 0)
    return fail(c, PIC1D_EINVAL, "train_surrogate: bad configuration");
  int rc = sur_ensure(c);
  if (rc != PIC1D_OK) return rc;
  *rep = pic1d_train_report{};
  const long long n = cfg->n_samples, nv = cfg->n_val;
  const int tiles = cfg->batch / 128;
  const long long per_epoch = n / cfg->batch;
  const long long steps = per_epoch * cfg->epochs;
  float *rec = nullptr, *vrec = nullptr, *vy = nullptr, *verr = nullptr, *losses = nullptr;
  cudaEvent_t e0, e1, e2, e3;
  CK(cudaEventCreate(&e0), "train");
  CK(cudaEventCreate(&e1), "train");
  CK(cudaEventCreate(&e2), "train");
  CK(cudaEventCreate(&e3), "train");
  auto cleanup = [&]() {
    dfree(rec); dfree(vrec); dfree(vy); dfree(verr); dfree(losses);
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2); cudaEventDestroy(e3);
  };
  cudaError_t e = dalloc(&rec, (size_t)n * kSurRecord);
  if (e == cudaSuccess && nv > 0) e = dalloc(&vrec, (size_t)nv * kSurRecord);
  if (e == cudaSuccess && nv > 0) e = dalloc(&vy, (size_t)nv * 4);
  if (e == cudaSuccess && nv > 0) e = dalloc(&verr, (size_t)nv * 2);
  if (e == cudaSuccess && steps > 0) e = dalloc(&losses, (size_t)steps);
  if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "train_surrogate alloc"); }
  const SurPhys Q = sur_phys(c);
  e = cudaEventRecord(e0, c->s);
  if (e == cudaSuccess) e = sur_launch_samples(Q, cfg->seed, 0, n, cfg->r_lo, cfg->r_hi, rec, c->s);
  if (e == cudaSuccess && nv > 0) e = sur_launch_samples(Q, cfg->val_seed, 0, nv, cfg->r_lo, cfg->r_hi, vrec, c->s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->s);
  // epochs: batches drawn through an affine permutation i -> (a i + c) mod n
  // with a coprime to n, fresh per epoch
  std::mt19937_64 rng(cfg->seed ^ 0x5EEDull);
  for (int ep = 0; ep < cfg->epochs && e == cudaSuccess; ++ep) {
    unsigned long long a = (rng() % (unsigned long long)n) | 1ull, cc = rng() % (unsigned long long)n;
    while (std::gcd(a, (unsigned long long)n) != 1ull) a += 2;
    a %= (unsigned long long)n;
    if (a == 0) a = 1;
    for (long long k = 0; k < per_epoch && e == cudaSuccess; ++k) {
      const long long step = (long long)ep * per_epoch + k;
      double lr = cfg->lr;
      if (cfg->lr_final > 0.0 && steps > 1)
        lr = cfg->lr_final + 0.5 * (cfg->lr - cfg->lr_final) * (1.0 + std::cos(kPi * (double)step / (double)(steps - 1)));
      e = sur_launch_train(c->sur, rec, n, a, cc, k * cfg->batch, cfg->batch, c->s);
      if (e == cudaSuccess)
        e = sur_launch_update(c->sur, tiles, 1, (float)lr, ++c->sur_t, nullptr, losses + step, c->s);
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(e2, c->s);
  if (e == cudaSuccess && nv > 0) e = sur_launch_infer(c->sur, vrec, kSurRecord, nv, vy, c->sms, c->s);
  if (e == cudaSuccess && nv > 0) e = sur_launch_val(vrec, vy, nv, verr, c->s);
  if (e == cudaSuccess) e = cudaEventRecord(e3, c->s);
  std::vector<float> herr((size_t)nv * 2), hl(2, 0.0f);
  if (e == cudaSuccess && nv > 0)
    e = cudaMemcpyAsync(herr.data(), verr, (size_t)nv * 2 * sizeof(float), cudaMemcpyDeviceToHost, c->s);
  if (e == cudaSuccess && steps > 0) e = cudaMemcpyAsync(&hl[0], losses, sizeof(float), cudaMemcpyDeviceToHost, c->s);
  if (e == cudaSuccess && steps > 0)
    e = cudaMemcpyAsync(&hl[1], losses + steps - 1, sizeof(float), cudaMemcpyDeviceToHost, c->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
  if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "train_surrogate"); }
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1); rep->samples_ms = ms;
  cudaEventElapsedTime(&ms, e1, e2); rep->train_ms = ms;
  cudaEventElapsedTime(&ms, e2, e3); rep->val_ms = ms;
  cleanup();
  rep->steps = steps;
  rep->n_samples = n;
  rep->n_val = nv;
  rep->loss_first = hl[0] / cfg->batch;
  rep->loss_last = hl[1] / cfg->batch;
  std::vector<float> de, le;
  for (long long i = 0; i < nv; ++i)
    if (herr[2 * i] >= 0.0f) { de.push_back(herr[2 * i]); le.push_back(herr[2 * i + 1]); }
  rep->val_count = (int64_t)de.size();
  auto pct = [](std::vector<float>& v, double q) -> double {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1)));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
  };
  rep->drag_err_median = pct(de, 0.5);
  rep->drag_err_p99 = pct(de, 0.99);
  rep->drag_err_max = de.empty() ? 0.0 : *std::max_element(de.begin(), de.end());
  rep->lnN_err_median = pct(le, 0.5);
  rep->lnN_err_p99 = pct(le, 0.99);
  rep->lnN_err_max = le.empty() ? 0.0 : *std::max_element(le.begin(), le.end());
  return sur_check(c);
}

// ------------------------------------------------------------- checkpoints
}  // extern "C"

namespace {

const char kCkptMagic[8] = {'P', 'I', 'C', '1', 'D', 'C', 'K', '1'};
constexpr uint32_t kCkptVersion = 3;

// The parameters as they must agree between a checkpoint and the context
// that loads it, field by field (the struct's padding is not part of it; the
// stream and the capacity may differ): doubles by their bit patterns,
// integers by value.
std::vector<uint64_t> ckpt_params(const pic1d_params& p) {
  auto d = [](double x) { uint64_t u; std::memcpy(&u, &x, 8); return u; };
  return {d(p.r_eq), (uint64_t)p.n_cells, d(p.cfl), d(p.b_star), (uint64_t)p.b_convention, d(p.kT_keV),
          (uint64_t)p.photon_model, (uint64_t)p.drag_law, d(p.drag_scale), (uint64_t)p.table_n_gamma,
          (uint64_t)p.table_n_s, d(p.table_log10g_max), (uint64_t)p.quad_n_mu, (uint64_t)p.quad_n_phi,
          d(p.eta_min), (uint64_t)p.rics_mode, (uint64_t)p.mc_on, d(p.cells_per_skin_depth), d(p.j_psi),
          d(p.n0_ppc), d(p.mass_ratio), (uint64_t)p.inject_mode, d(p.inject_T), d(p.atmo_a0), d(p.atmo_h),
          d(p.atmo_ncut), (uint64_t)p.pairs_on,
          d(p.b_pair_threshold), d(p.pair_energy_threshold), d(p.n_max_ppc), (uint64_t)p.annihilate_every, p.seed,
          d(p.r_star_cm),
          (uint64_t)p.sort_every};
}

struct File {
  FILE* f = nullptr;
  explicit File(FILE* x) : f(x) {}
  ~File() { if (f) std::fclose(f); }
  bool put(const void* p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
  bool get(void* p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
};

// device array -> file (through a host buffer)
template <typename T>
bool put_dev(pic1d_ctx* c, File& F, const T* d, long long n) {
  std::vector<T> h((size_t)n);
  if (n > 0 && cudaMemcpyAsync(h.data(), d, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, c->s) != cudaSuccess)
    return false;
  if (cudaStreamSynchronize(c->s) != cudaSuccess) return false;
  return F.put(h.data(), sizeof(T) * (size_t)n);
}

template <typename T>
bool get_dev(pic1d_ctx* c, File& F, T* d, long long n) {
  std::vector<T> h((size_t)n);
  if (!F.get(h.data(), sizeof(T) * (size_t)n)) return false;
  if (n > 0 && cudaMemcpyAsync(d, h.data(), sizeof(T) * (size_t)n, cudaMemcpyHostToDevice, c->s) != cudaSuccess)
    return false;
  return cudaStreamSynchronize(c->s) == cudaSuccess;
}

}  // namespace

extern "C" {

int pic1d_save(pic1d_ctx* c, const char* path) {
  if (!c || !path) return fail(c, PIC1D_EINVAL, "save: NULL argument");
  CK(cudaStreamSynchronize(c->s), "save");
  StepState st{};
  Counters ctr{};
  CK(cudaMemcpy(&st, c->st, sizeof(st), cudaMemcpyDeviceToHost), "save");
  CK(cudaMemcpy(&ctr, c->ctr, sizeof(ctr), cudaMemcpyDeviceToHost), "save");
  File F(std::fopen(path, "wb"));
  if (!F.f) return fail(c, PIC1D_EINVAL, std::string("save: cannot open ") + path);
  const std::vector<uint64_t> q = ckpt_params(c->p);
  const uint32_t ver = kCkptVersion, nq = (uint32_t)q.size();
  const long long step = c->step, n = st.n_slots;
  const int N = c->N, b = c->cur;
  bool ok = F.put(kCkptMagic, 8) && F.put(&ver, 4) && F.put(&nq, 4) && F.put(q.data(), 8 * q.size()) &&
            F.put(&step, 8) && F.put(&n, 8) && F.put(&N, 4);
  ok = ok && put_dev(c, F, c->pos[b], n) && put_dev(c, F, c->u[b], n) && put_dev(c, F, c->w[b], n) &&
       put_dev(c, F, c->sp[b], n) && put_dev(c, F, c->id[b], n);
  ok = ok && put_dev(c, F, c->E64, N) && put_dev(c, F, c->J, N);
  // the pair-cap density of this step, then of the next
  ok = ok && put_dev(c, F, c->dens[step & 1], N) && put_dev(c, F, c->dens[(step + 1) & 1], N);
  ok = ok && F.put(&ctr, sizeof(ctr)) && F.put(&st, sizeof(st));
  const int32_t sur = c->sur_on ? 1 : 0;
  ok = ok && F.put(&sur, 4);
  if (ok && sur) {
    const int32_t t = c->sur_t;
    ok = F.put(&t, 4) && put_dev(c, F, c->sur.master, W_N_PARAMS) && put_dev(c, F, c->sur.m, W_N_PARAMS) &&
         put_dev(c, F, c->sur.v, W_N_PARAMS);
  }
  if (!ok) return fail(c, PIC1D_ECUDA, std::string("save: write to ") + path + " failed");
  return PIC1D_OK;
}

int pic1d_load(pic1d_ctx* c, const char* path) {
  if (!c || !path) return fail(c, PIC1D_EINVAL, "load: NULL argument");
  File F(std::fopen(path, "rb"));
  if (!F.f) return fail(c, PIC1D_EINVAL, std::string("load: cannot open ") + path);
  char magic[8];
  uint32_t ver = 0, nq = 0;
  const std::vector<uint64_t> mine = ckpt_params(c->p);
  std::vector<uint64_t> q(mine.size());
  if (!F.get(magic, 8) || std::memcmp(magic, kCkptMagic, 8) != 0 || !F.get(&ver, 4) || ver != kCkptVersion ||
      !F.get(&nq, 4) || nq != mine.size() || !F.get(q.data(), 8 * q.size()))
    return fail(c, PIC1D_EINVAL, std::string("load: ") + path + " is not a checkpoint of this library version");
  if (q != mine) return fail(c, PIC1D_EINVAL, "load: the checkpoint was written with other parameters");
  long long step = 0, n = 0;
  int N = 0;
  if (!F.get(&step, 8) || !F.get(&n, 8) || !F.get(&N, 4) || N != c->N || n < 0 || step < 0)
    return fail(c, PIC1D_EINVAL, "load: bad checkpoint header");
  if (c->p.capacity > 0 && n > c->p.capacity) return fail(c, PIC1D_EINVAL, "load: more slots than the capacity");
  if (n > PIC1D_MAX_SLOTS) return fail(c, PIC1D_EINVAL, "load: more than PIC1D_MAX_SLOTS particles");
  if (n > c->cap) {
    const int rc = alloc_particles(c, c->p.capacity > 0 ? c->p.capacity
                                                      : std::min<long long>(2 * n + 4 * kTile, PIC1D_MAX_SLOTS));
    if (rc != PIC1D_OK) return rc;
  }
  CK(cudaStreamSynchronize(c->s), "load");
  c->cur = 0;
  bool ok = get_dev(c, F, c->pos[0], n) && get_dev(c, F, c->u[0], n) && get_dev(c, F, c->w[0], n) &&
            get_dev(c, F, c->sp[0], n) && get_dev(c, F, c->id[0], n);
  ok = ok && cudaMemsetAsync(c->sp[0] + n, PIC1D_SP_DEAD, (size_t)(c->alloc - n), c->s) == cudaSuccess;
  std::vector<double> E((size_t)N);
  ok = ok && F.get(E.data(), sizeof(double) * (size_t)N);
  std::vector<float> E32((size_t)N);
  for (int i = 0; i < N; ++i) E32[i] = (float)E[i];
  ok = ok && cudaMemcpy(c->E64, E.data(), sizeof(double) * N, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->E32, E32.data(), sizeof(float) * N, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && get_dev(c, F, c->J, N) && get_dev(c, F, c->dens[step & 1], N) &&
       get_dev(c, F, c->dens[(step + 1) & 1], N);
  Counters ctr{};
  StepState st{};
  ok = ok && F.get(&ctr, sizeof(ctr)) && F.get(&st, sizeof(st));
  int32_t sur = 0;
  ok = ok && F.get(&sur, 4);
  if (!ok) return fail(c, PIC1D_EINVAL, std::string("load: ") + path + " is truncated or unreadable");
  st.n_slots = n;
  st.append = 0;
  st.work = 0;
  st.step = step;
  CK(cudaMemcpy(c->ctr, &ctr, sizeof(ctr), cudaMemcpyHostToDevice), "load");
  CK(cudaMemcpy(c->st, &st, sizeof(st), cudaMemcpyHostToDevice), "load");
  c->step = step;
  c->gauss_on = false;
  if (sur) {
    int rc = sur_ensure(c);
    if (rc != PIC1D_OK) return rc;
    int32_t t = 0;
    ok = F.get(&t, 4) && get_dev(c, F, c->sur.master, W_N_PARAMS) && get_dev(c, F, c->sur.m, W_N_PARAMS) &&
         get_dev(c, F, c->sur.v, W_N_PARAMS);
    if (!ok) return fail(c, PIC1D_EINVAL, std::string("load: ") + path + " is truncated (network)");
    CK(sur_launch_update(c->sur, 0, 2, 0.0f, 1, nullptr, nullptr, c->s), "load");
    CK(cudaStreamSynchronize(c->s), "load");
    c->sur_t = t;
  }
  return PIC1D_OK;
}

// ------------------------------------------------------------- ensemble
}  // extern "C"

namespace {
constexpr int kEnsSuper = 80;               // steps per captured graph
const int kEnsCadences[3] = {10, 20, 40};   // sort cadences (each divides kEnsSuper / 2)
const int kEnsChunks[3] = {1, 4, 16};       // tiles of 128 slots per push item
}  // namespace

struct pic1d_ens {
  int n = 0;
  std::vector<pic1d_ctx*> lines;
  cudaStream_t s = nullptr;
  int sms = 0;
  EnsLine* dlines = nullptr;
  int4* push_items = nullptr;
  int n_push_items = 0;
  int2* cell_items = nullptr;
  int n_cell_items = 0;
  unsigned long long* work = nullptr;
  std::vector<int> chunk, cadence;
  cudaGraphExec_t graph = nullptr;
  std::vector<long long> graph_phase;       // per line: step mod kEnsSuper at capture
  std::vector<int> graph_cur;               // per line: buffer at capture
  bool schedule_dirty = true;
  std::string err;
  // autotuner bookkeeping (eager steps)
  bool time_sorts = false;
  std::vector<double> sort_ms;
  std::vector<int> sort_count;
  // per-step history (pic1d_ens_record)
  EnsRec* drec = nullptr;           // descriptor read by the finalize kernel
  EnsRec rec{};                     // host copy of it
  std::vector<long long> rec_base;  // pairs_created of each line when the record was armed
};

namespace {

int ens_fail(pic1d_ens* e, int code, const std::string& msg) {
  if (e) e->err = msg;
  return code;
}

#define ECK(call, where)                                                                        \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return ens_fail(e, e_ == cudaErrorMemoryAllocation ? PIC1D_ENOMEM : PIC1D_ECUDA,          \
                      std::string(where) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

EnsLine ens_record(pic1d_ctx* c, pic1d_ctx* net) {
  EnsLine L{};
  L.P = dev_params(c);
  L.P.sur_img = net->sur.img;
  L.P.sur_small = net->sur.small;
  L.P.sur_err = net->sur.err;
  for (int b = 0; b < 2; ++b) {
    L.pos[b] = c->pos[b]; L.u[b] = c->u[b]; L.w[b] = c->w[b]; L.sp[b] = c->sp[b]; L.id[b] = c->id[b];
    L.dens[b] = c->dens[b];
  }
  L.E64 = c->E64;
  L.E32 = c->E32;
  L.a = 4.0 * kPi * c->dt * c->j_ext;
  L.cJ = 4.0 * kPi * c->q_p * std::ldexp(1.0, -c->F - kWBits);
  L.dt_jext = c->dt * c->j_ext;
  L.cur = c->cur;
  return L;
}

// upload the line records (the host contexts are the source of truth between calls)
int ens_sync_records(pic1d_ens* e) {
  std::vector<EnsLine> h(e->n);
  for (int l = 0; l < e->n; ++l) h[l] = ens_record(e->lines[l], e->lines[0]);
  ECK(cudaMemcpyAsync(e->dlines, h.data(), sizeof(EnsLine) * e->n, cudaMemcpyHostToDevice, e->s), "ensemble records");
  ECK(cudaStreamSynchronize(e->s), "ensemble records");
  return PIC1D_OK;
}

// push items: each line's capacity in items of chunk[l] tiles, largest lines first
int ens_build_items(pic1d_ens* e) {
  std::vector<int> order(e->n);
  for (int l = 0; l < e->n; ++l) order[l] = l;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return e->lines[a]->cap > e->lines[b]->cap; });
  std::vector<int4> items;
  for (int l : order) {
    const long long tiles = (e->lines[l]->cap + 127) / 128;
    for (long long t0 = 0; t0 < tiles; t0 += e->chunk[l])
      items.push_back(make_int4(l, (int)t0, (int)std::min<long long>(e->chunk[l], tiles - t0), 0));
  }
  std::vector<int2> cells;
  for (int l = 0; l < e->n; ++l)
    for (int c0 = 0; c0 < e->lines[l]->N; c0 += 256) cells.push_back(make_int2(l, c0));
  dfree(e->push_items);
  dfree(e->cell_items);
  e->push_items = nullptr;
  e->cell_items = nullptr;
  ECK(raw_alloc(reinterpret_cast<void**>(&e->push_items), sizeof(int4) * std::max<size_t>(1, items.size())), "ensemble items");
  ECK(raw_alloc(reinterpret_cast<void**>(&e->cell_items), sizeof(int2) * std::max<size_t>(1, cells.size())), "ensemble items");
  ECK(cudaMemcpyAsync(e->push_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, e->s),
      "ensemble items");
  ECK(cudaMemcpyAsync(e->cell_items, cells.data(), sizeof(int2) * cells.size(), cudaMemcpyHostToDevice, e->s),
      "ensemble items");
  ECK(cudaStreamSynchronize(e->s), "ensemble items");
  e->n_push_items = (int)items.size();
  e->n_cell_items = (int)cells.size();
  return PIC1D_OK;
}

EnsArgs ens_args(pic1d_ens* e) {
  EnsArgs A;
  A.lines = e->dlines;
  A.n_lines = e->n;
  A.push_items = e->push_items;
  A.n_push_items = e->n_push_items;
  A.cell_items = e->cell_items;
  A.n_cell_items = e->n_cell_items;
  A.work = e->work;
  A.sur_img = e->lines[0]->sur.img;
  A.sur_small = e->lines[0]->sur.small;
  A.sur_err = e->lines[0]->sur.err;
  A.rec = e->drec;
  return A;
}

// a line's kernel parameters for buffer `cur` at step `step` (the ensemble
// enqueues steps ahead of the line's own bookkeeping)
DevParams line_params(pic1d_ctx* c, int cur, long long step) {
  const int keep_cur = c->cur;
  const long long keep_step = c->step;
  c->cur = cur;
  c->step = step;
  const DevParams P = dev_params(c);
  c->cur = keep_cur;
  c->step = keep_step;
  return P;
}

// sorts a line takes at the end of step k: its cadence, and annihilation's
bool ens_sorts_at(const pic1d_ens* e, int l, long long k) {
  const int ae = e->lines[l]->p.annihilate_every;
  return k % e->cadence[l] == 0 || (ae > 0 && k % ae == 0);
}

// enqueue k steps of every line on the stream; cur/step give each line's
// buffer and step at the start and are advanced as the steps would
int ens_enqueue(pic1d_ens* e, int k, std::vector<int>& cur, std::vector<long long>& step) {
  const EnsArgs A = ens_args(e);
  std::vector<cudaEvent_t> evs;
  std::vector<int> ev_line;
  for (int i = 0; i < k; ++i) {
    ECK(ens_launch_clear(A, e->s), "ensemble clear");
    ECK(ens_launch_push(A, e->sms * kSurPushPerSm, e->s), "ensemble push");
    // the surface supply of the lines that have one (Sec. 3, App. B.1)
    for (int l = 0; l < e->n; ++l) {
      pic1d_ctx* c = e->lines[l];
      const pic1d_params& p = c->p;
      if (p.inject_mode == PIC1D_INJECT_NONE) continue;
      const DevParams P = line_params(c, cur[l], step[l]);
      const float sig_e = (float)std::sqrt(p.inject_T), sig_i = (float)std::sqrt(p.inject_T / p.mass_ratio);
      if (p.inject_mode == PIC1D_INJECT_RATE)
        ECK(launch_inject(P, p.j_psi * p.n0_ppc * c->dt, sig_e, sig_i, e->s), "ensemble supply");
      else
        ECK(launch_topup(P, c->atmo_cells, c->atmo_target, c->n_atmo, sig_e, sig_i, e->s), "ensemble top-up");
    }
    ECK(ens_launch_field(A, e->s), "ensemble field");
    ECK(ens_launch_finalize(A, e->s), "ensemble finalize");
    for (int l = 0; l < e->n; ++l) {
      step[l] += 1;
      if (!ens_sorts_at(e, l, step[l])) continue;
      pic1d_ctx* c = e->lines[l];
      DevParams P = line_params(c, cur[l], step[l]);
      const int o = 1 - cur[l];
      cudaEvent_t a = nullptr, b = nullptr;
      if (e->time_sorts) {
        ECK(cudaEventCreate(&a), "ensemble timing");
        ECK(cudaEventCreate(&b), "ensemble timing");
        ECK(cudaEventRecord(a, e->s), "ensemble timing");
      }
      ECK(launch_sort(P, c->counts, c->offsets, c->bsum, c->pos[o], c->u[o], c->w[o], c->sp[o], c->id[o],
                      c->sms, e->s),
          "ensemble sort");
      ECK(ens_launch_flip(e->dlines, l, e->s), "ensemble sort");
      if (e->time_sorts) {
        ECK(cudaEventRecord(b, e->s), "ensemble timing");
        evs.push_back(a);
        evs.push_back(b);
        ev_line.push_back(l);
        e->sort_count[l] += 1;
      }
      cur[l] = o;
      const int ae = c->p.annihilate_every;
      if (ae > 0 && step[l] % ae == 0) {
        // annihilation at n_max on the sorted buffer (Sec. 3)
        const DevParams Q = line_params(c, cur[l], step[l]);
        const double cJ = 4.0 * kPi * c->q_p * std::ldexp(1.0, -c->F - kWBits);
        ECK(launch_annihilate(Q, c->counts, c->offsets, c->ann_list, c->ann_amount, c->ann_count, c->E64, c->E32,
                              cJ, c->sms, e->s),
            "ensemble annihilation");
      }
    }
  }
  if (!evs.empty()) {
    ECK(cudaStreamSynchronize(e->s), "ensemble timing");
    for (size_t j = 0; j < ev_line.size(); ++j) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, evs[2 * j], evs[2 * j + 1]);
      e->sort_ms[ev_line[j]] += ms;
    }
    for (cudaEvent_t x : evs) cudaEventDestroy(x);
  }
  return PIC1D_OK;
}

void ens_apply(pic1d_ens* e, const std::vector<int>& cur, const std::vector<long long>& step) {
  for (int l = 0; l < e->n; ++l) {
    e->lines[l]->cur = cur[l];
    e->lines[l]->step = step[l];
  }
}

}  // namespace

extern "C" {

int pic1d_ens_init(const pic1d_params* params, int32_t n_lines, pic1d_ens** out) {
  if (!out) return PIC1D_EINVAL;
  *out = nullptr;
  if (!params || n_lines < 1) return PIC1D_EINVAL;
  for (int l = 0; l < n_lines; ++l) {
    if (params[l].drag_law != PIC1D_DRAG_SURROGATE || params[l].cuda_stream != params[0].cuda_stream ||
        (params[l].annihilate_every > 0 && kEnsSuper % params[l].annihilate_every != 0)) {
      std::fprintf(stderr, "pic1d_ens_init: line %d: the ensemble runs drag law SURROGATE, one stream for all "
                           "lines, and an annihilation cadence that divides %d\n", l, kEnsSuper);
      return PIC1D_EINVAL;
    }
  }
  pic1d_ens* e = new pic1d_ens();
  e->n = n_lines;
  e->lines.assign(n_lines, nullptr);
  for (int l = 0; l < n_lines; ++l) {
    const int rc = pic1d_init(&params[l], &e->lines[l]);
    if (rc != PIC1D_OK) {
      std::fprintf(stderr, "pic1d_ens_init: line %d failed (%d)\n", l, rc);
      pic1d_ens_free(e);
      return rc;
    }
  }
  // one non-blocking stream of the ensemble's own for every line (a stream
  // that can be captured into a graph)
  if (cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking) != cudaSuccess) {
    e->s = nullptr;
    pic1d_ens_free(e);
    return PIC1D_ECUDA;
  }
  for (pic1d_ctx* c : e->lines) {
    if (c->s) cudaStreamSynchronize(c->s);
    c->s = e->s;
  }
  e->sms = e->lines[0]->sms;
  e->chunk.assign(n_lines, 4);
  e->cadence.assign(n_lines, 20);
  for (int l = 0; l < n_lines; ++l) {
    int best = kEnsCadences[0];
    for (int cd : kEnsCadences)
      if (std::abs(cd - params[l].sort_every) < std::abs(best - params[l].sort_every)) best = cd;
    e->cadence[l] = best;
  }
  e->sort_ms.assign(n_lines, 0.0);
  e->sort_count.assign(n_lines, 0);
  int rc = sur_ensure(e->lines[0]);
  cudaError_t ce = cudaSuccess;
  if (rc == PIC1D_OK) ce = raw_alloc(reinterpret_cast<void**>(&e->dlines), sizeof(EnsLine) * n_lines);
  if (rc == PIC1D_OK && ce == cudaSuccess) ce = raw_alloc(reinterpret_cast<void**>(&e->work), sizeof(unsigned long long));
  if (rc == PIC1D_OK && ce == cudaSuccess) ce = cudaMemsetAsync(e->work, 0, sizeof(unsigned long long), e->s);
  if (rc == PIC1D_OK && ce == cudaSuccess) ce = raw_alloc(reinterpret_cast<void**>(&e->drec), sizeof(EnsRec));
  if (rc == PIC1D_OK && ce == cudaSuccess) ce = cudaMemsetAsync(e->drec, 0, sizeof(EnsRec), e->s);
  if (rc == PIC1D_OK && ce != cudaSuccess) rc = PIC1D_ECUDA;
  if (rc == PIC1D_OK) rc = ens_build_items(e);
  if (rc != PIC1D_OK) {
    pic1d_ens_free(e);
    return rc;
  }
  *out = e;
  return PIC1D_OK;
}

pic1d_ctx* pic1d_ens_line(pic1d_ens* e, int32_t line) {
  if (!e || line < 0 || line >= e->n) return nullptr;
  return e->lines[line];
}

int pic1d_ens_set_schedule(pic1d_ens* e, const int32_t* chunk_tiles, const int32_t* sort_every) {
  if (!e) return PIC1D_EINVAL;
  for (int l = 0; l < e->n; ++l) {
    if (chunk_tiles && chunk_tiles[l] < 1) return ens_fail(e, PIC1D_EINVAL, "set_schedule: chunk_tiles < 1");
    if (sort_every && std::find(std::begin(kEnsCadences), std::end(kEnsCadences), sort_every[l]) ==
                          std::end(kEnsCadences))
      return ens_fail(e, PIC1D_EINVAL, "set_schedule: sort_every must be 10, 20 or 40");
  }
  for (int l = 0; l < e->n; ++l) {
    if (chunk_tiles) e->chunk[l] = chunk_tiles[l];
    if (sort_every) e->cadence[l] = sort_every[l];
  }
  e->schedule_dirty = true;
  return ens_build_items(e);
}

int pic1d_ens_get_schedule(pic1d_ens* e, int32_t* chunk_tiles, int32_t* sort_every) {
  if (!e) return PIC1D_EINVAL;
  for (int l = 0; l < e->n; ++l) {
    if (chunk_tiles) chunk_tiles[l] = e->chunk[l];
    if (sort_every) sort_every[l] = e->cadence[l];
  }
  return PIC1D_OK;
}

int pic1d_ens_step(pic1d_ens* e, int n_steps) {
  if (!e) return PIC1D_EINVAL;
  Nvtx range("pic1d_ens_step");
  if (n_steps < 0) return ens_fail(e, PIC1D_EINVAL, "ens_step: n_steps < 0");
  if (!e->lines[0]->sur_on) return ens_fail(e, PIC1D_EINVAL, "ens_step: no network (set or train it on line 0)");
  int rc = ens_sync_records(e);
  if (rc != PIC1D_OK) return rc;
  std::vector<int> cur(e->n);
  std::vector<long long> step(e->n);
  for (int l = 0; l < e->n; ++l) { cur[l] = e->lines[l]->cur; step[l] = e->lines[l]->step; }
  while (n_steps >= kEnsSuper) {
    // a captured super-step replays exactly when every line starts from the
    // buffer and the step phase it had at capture
    bool match = e->graph && !e->schedule_dirty;
    for (int l = 0; l < e->n && match; ++l)
      match = e->graph_cur[l] == cur[l] && e->graph_phase[l] == step[l] % kEnsSuper;
    if (!match) {
      if (e->graph) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
      std::vector<int> c2 = cur;
      std::vector<long long> s2 = step;
      cudaGraph_t g = nullptr;
      ECK(cudaStreamBeginCapture(e->s, cudaStreamCaptureModeThreadLocal), "ensemble capture");
      rc = ens_enqueue(e, kEnsSuper, c2, s2);
      cudaError_t ce = cudaStreamEndCapture(e->s, &g);
      if (rc != PIC1D_OK) { if (g) cudaGraphDestroy(g); return rc; }
      ECK(ce, "ensemble capture");
      ce = cudaGraphInstantiate(&e->graph, g, 0);
      cudaGraphDestroy(g);
      ECK(ce, "ensemble graph");
      e->graph_cur = cur;
      e->graph_phase.resize(e->n);
      for (int l = 0; l < e->n; ++l) e->graph_phase[l] = step[l] % kEnsSuper;
      e->schedule_dirty = false;
    }
    ECK(cudaGraphLaunch(e->graph, e->s), "ensemble graph launch");
    for (int l = 0; l < e->n; ++l) {
      long long sorts = 0;
      for (long long k = step[l] + 1; k <= step[l] + kEnsSuper; ++k) sorts += ens_sorts_at(e, l, k);
      if (sorts & 1) cur[l] ^= 1;
      step[l] += kEnsSuper;
    }
    n_steps -= kEnsSuper;
  }
  if (n_steps > 0) {
    rc = ens_enqueue(e, n_steps, cur, step);
    if (rc != PIC1D_OK) return rc;
  }
  ens_apply(e, cur, step);
  return PIC1D_OK;
}

int pic1d_ens_tune(pic1d_ens* e, int32_t trial_steps, int32_t* chunk_out, int32_t* cadence_out, double* cost_ms) {
  if (!e) return PIC1D_EINVAL;
  if (trial_steps < 1) return ens_fail(e, PIC1D_EINVAL, "ens_tune: trial_steps < 1");
  if (!e->lines[0]->sur_on) return ens_fail(e, PIC1D_EINVAL, "ens_tune: no network (set or train it on line 0)");
  int clock_khz = 0;
  ECK(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, 0), "ens_tune");
  const int nc = 3, nk = 3;
  std::vector<double> cost((size_t)e->n * nc * nk, 0.0);
  const std::vector<int> chunk0 = e->chunk, cad0 = e->cadence;
  for (int ci = 0; ci < nc; ++ci) {
    for (int ki = 0; ki < nk; ++ki) {
      for (int l = 0; l < e->n; ++l) { e->chunk[l] = kEnsChunks[ci]; e->cadence[l] = kEnsCadences[ki]; }
      int rc = ens_build_items(e);
      if (rc != PIC1D_OK) return rc;
      rc = ens_sync_records(e);
      if (rc != PIC1D_OK) return rc;
      std::vector<int> cur(e->n);
      std::vector<long long> step(e->n);
      for (int l = 0; l < e->n; ++l) { cur[l] = e->lines[l]->cur; step[l] = e->lines[l]->step; }
      // a trial long enough to hold at least one sort of every line
      const int steps = std::max<int>(trial_steps, kEnsCadences[ki]);
      std::fill(e->sort_ms.begin(), e->sort_ms.end(), 0.0);
      std::fill(e->sort_count.begin(), e->sort_count.end(), 0);
      e->time_sorts = true;
      rc = ens_enqueue(e, steps, cur, step);
      e->time_sorts = false;
      if (rc != PIC1D_OK) return rc;
      ECK(cudaStreamSynchronize(e->s), "ens_tune");
      std::vector<EnsLine> h(e->n);
      ECK(cudaMemcpy(h.data(), e->dlines, sizeof(EnsLine) * e->n, cudaMemcpyDeviceToHost), "ens_tune");
      ens_apply(e, cur, step);
      for (int l = 0; l < e->n; ++l) {
        const double push_ms = (double)h[l].cycles / (double)clock_khz / steps;   // SM-clock ms per step
        const double sort_ms = e->sort_count[l] ? e->sort_ms[l] / e->sort_count[l] : 0.0;
        cost[((size_t)l * nc + ci) * nk + ki] = push_ms + sort_ms / kEnsCadences[ki];
      }
    }
  }
  for (int l = 0; l < e->n; ++l) {
    int bc = 0, bk = 0;
    for (int ci = 0; ci < nc; ++ci)
      for (int ki = 0; ki < nk; ++ki)
        if (cost[((size_t)l * nc + ci) * nk + ki] < cost[((size_t)l * nc + bc) * nk + bk]) { bc = ci; bk = ki; }
    e->chunk[l] = kEnsChunks[bc];
    e->cadence[l] = kEnsCadences[bk];
    if (chunk_out) chunk_out[l] = e->chunk[l];
    if (cadence_out) cadence_out[l] = e->cadence[l];
    if (cost_ms) cost_ms[l] = cost[((size_t)l * nc + bc) * nk + bk];
  }
  (void)chunk0;
  (void)cad0;
  e->schedule_dirty = true;
  return ens_build_items(e);
}

void* pic1d_ens_stream(pic1d_ens* e) { return e ? reinterpret_cast<void*>(e->s) : nullptr; }

const char* pic1d_ens_last_error(const pic1d_ens* e) {
  if (!e) return "no ensemble";
  return e->err.c_str();
}

int pic1d_ens_record(pic1d_ens* e, int32_t capacity) {
  if (!e) return PIC1D_EINVAL;
  if (capacity < 0) return ens_fail(e, PIC1D_EINVAL, "record: capacity < 0");
  ECK(cudaStreamSynchronize(e->s), "record");
  // the finalize kernel stops recording before the old buffers go (a failed
  // allocation below then leaves the record off, not pointing at freed memory)
  const EnsRec off{};
  ECK(cudaMemcpyAsync(e->drec, &off, sizeof(EnsRec), cudaMemcpyHostToDevice, e->s), "record");
  ECK(cudaStreamSynchronize(e->s), "record");
  dfree(e->rec.vc);
  dfree(e->rec.pairs);
  dfree(e->rec.n);
  e->rec = EnsRec{};
  if (capacity > 0) {
    const size_t m = (size_t)e->n * (size_t)capacity;
    ECK(raw_alloc(reinterpret_cast<void**>(&e->rec.vc), m * sizeof(double)), "record");
    ECK(raw_alloc(reinterpret_cast<void**>(&e->rec.pairs), m * sizeof(long long)), "record");
    ECK(raw_alloc(reinterpret_cast<void**>(&e->rec.n), (size_t)e->n * sizeof(int)), "record");
    ECK(cudaMemsetAsync(e->rec.n, 0, (size_t)e->n * sizeof(int), e->s), "record");
    e->rec.cap = capacity;
  }
  e->rec_base.assign(e->n, 0);
  for (int l = 0; l < e->n; ++l) {
    Counters C{};
    ECK(cudaMemcpyAsync(&C, e->lines[l]->ctr, sizeof(C), cudaMemcpyDeviceToHost, e->s), "record");
    ECK(cudaStreamSynchronize(e->s), "record");
    e->rec_base[l] = (long long)C.pairs_created;
  }
  ECK(cudaMemcpyAsync(e->drec, &e->rec, sizeof(EnsRec), cudaMemcpyHostToDevice, e->s), "record");
  ECK(cudaStreamSynchronize(e->s), "record");
  return PIC1D_OK;
}

int pic1d_ens_history(pic1d_ens* e, int32_t line, int32_t window, double* vc, int64_t* pairs, double* pair_rate,
                      int32_t* n_out) {
  if (!e || !n_out) return PIC1D_EINVAL;
  if (line < 0 || line >= e->n) return ens_fail(e, PIC1D_EINVAL, "history: no such line");
  if (window < 1 && pair_rate) return ens_fail(e, PIC1D_EINVAL, "history: window < 1");
  *n_out = 0;
  if (e->rec.cap == 0) return PIC1D_OK;
  int n = 0;
  ECK(cudaStreamSynchronize(e->s), "history");
  ECK(cudaMemcpy(&n, e->rec.n + line, sizeof(int), cudaMemcpyDeviceToHost), "history");
  n = std::min(n, e->rec.cap);
  std::vector<double> hv(n);
  std::vector<long long> hp(n);
  const size_t off = (size_t)line * (size_t)e->rec.cap;
  if (n > 0) {
    ECK(cudaMemcpy(hv.data(), e->rec.vc + off, n * sizeof(double), cudaMemcpyDeviceToHost), "history");
    ECK(cudaMemcpy(hp.data(), e->rec.pairs + off, n * sizeof(long long), cudaMemcpyDeviceToHost), "history");
  }
  for (int k = 0; k < n; ++k) hp[k] -= e->rec_base[line];
  if (vc) std::copy(hv.begin(), hv.end(), vc);
  if (pairs) for (int k = 0; k < n; ++k) pairs[k] = hp[k];
  if (pair_rate) {
    // pairs created per unit time over the last `window` steps (fewer at the start)
    const double dt = e->lines[line]->dt;
    for (int k = 0; k < n; ++k) {
      const int w = std::min(k + 1, (int)window);
      const long long before = (k >= window) ? hp[k - window] : 0;
      pair_rate[k] = (double)(hp[k] - before) / (w * dt);
    }
  }
  *n_out = n;
  return PIC1D_OK;
}

void pic1d_ens_free(pic1d_ens* e) {
  if (!e) return;
  if (e->s) cudaStreamSynchronize(e->s);
  if (e->graph) cudaGraphExecDestroy(e->graph);
  dfree(e->dlines);
  dfree(e->push_items);
  dfree(e->cell_items);
  dfree(e->work);
  dfree(e->drec);
  dfree(e->rec.vc);
  dfree(e->rec.pairs);
  dfree(e->rec.n);
  for (pic1d_ctx* c : e->lines) pic1d_free(c);
  if (e->s) cudaStreamDestroy(e->s);
  delete e;
}

int pic1d_tp_map(const pic1d_params* p, const double* r_eq, int32_t n, double gamma0, double dt, double t_max,
                 double b_thr, double gamma_eps, pic1d_tp_result* out, double* ms_out) {
  Nvtx range("pic1d_tp_map");
  if (!p || !r_eq || !out || n < 1 || !(gamma0 >= 1.0) || !(dt > 0.0) || !(t_max > 0.0) || !(b_thr > 0.0)) {
    std::fprintf(stderr, "pic1d_tp_map: bad arguments\n");
    return PIC1D_EINVAL;
  }
  for (int i = 0; i < n; ++i)
    if (!(r_eq[i] > 1.0)) {
      std::fprintf(stderr, "pic1d_tp_map: r_eq[%d] = %g must exceed 1\n", i, r_eq[i]);
      return PIC1D_EINVAL;
    }
  double* dr = nullptr;
  pic1d_tp_result* dout = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = raw_alloc(reinterpret_cast<void**>(&dr), sizeof(double) * n);
  if (e == cudaSuccess) e = raw_alloc(reinterpret_cast<void**>(&dout), sizeof(pic1d_tp_result) * n);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(p->cuda_stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dr, r_eq, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) e = tp_launch_map(*p, dr, n, gamma0, dt, t_max, b_thr, gamma_eps, dout, s);
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, dout, sizeof(pic1d_tp_result) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (ms_out) *ms_out = ms;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  dfree(dr);
  dfree(dout);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "pic1d_tp_map: %s\n", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PIC1D_ENOMEM : PIC1D_ECUDA;
  }
  return PIC1D_OK;
}

int pic1d_gauss_mark(pic1d_ctx* c) {
  if (!c) return PIC1D_EINVAL;
  if (!c->rho) CK(dalloc(&c->rho, c->N + 1), "gauss_mark");
  if (!c->rho_ref) CK(dalloc(&c->rho_ref, c->N + 1), "gauss_mark");
  if (!c->gauss_out) CK(dalloc(&c->gauss_out, 2), "gauss_mark");
  CK(cudaMemsetAsync(c->rho_ref, 0, sizeof(long long) * (c->N + 1), c->s), "gauss_mark");
  CK(launch_rho(dev_params(c), c->rho_ref, c->sms * 8, c->s), "gauss_mark");
  CK(cudaMemsetAsync(c->jcum, 0, sizeof(long long) * c->N, c->s), "gauss_mark");
  CK(cudaStreamSynchronize(c->s), "gauss_mark");
  c->gauss_on = true;
  return PIC1D_OK;
}

int pic1d_get_rho(pic1d_ctx* c, int64_t* rho, int mem) {
  if (!c) return PIC1D_EINVAL;
  if (!rho || (mem != 0 && mem != 1)) return fail(c, PIC1D_EINVAL, "get_rho: bad arguments");
  if (!c->rho) CK(dalloc(&c->rho, c->N + 1), "get_rho");
  CK(cudaMemsetAsync(c->rho, 0, sizeof(long long) * (c->N + 1), c->s), "get_rho");
  CK(launch_rho(dev_params(c), c->rho, c->sms * 8, c->s), "get_rho");
  CK(cudaMemcpyAsync(rho, c->rho, sizeof(long long) * (c->N + 1),
                     mem ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s), "get_rho");
  CK(cudaStreamSynchronize(c->s), "get_rho");
  return PIC1D_OK;
}

int pic1d_philox(const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out, int mem) {
  if (n < 0 || (n > 0 && (!ctr || !out)) || (mem != 0 && mem != 1)) {
    std::fprintf(stderr, "pic1d_philox: bad arguments\n");
    return PIC1D_EINVAL;
  }
  if (n == 0) return PIC1D_OK;
  if (mem == 1 && ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) & 15u)) {
    std::fprintf(stderr, "pic1d_philox: device arrays must be 16-byte aligned\n");
    return PIC1D_EINVAL;
  }
  const size_t bytes = (size_t)n * 4 * sizeof(uint32_t);
  void* dc = const_cast<uint32_t*>(ctr);
  void* dout = out;
  cudaError_t e = cudaSuccess;
  if (mem == 0) {
    dc = nullptr;
    dout = nullptr;
    e = raw_alloc(&dc, bytes);
    if (e == cudaSuccess) e = raw_alloc(&dout, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, bytes, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = launch_philox(dc, n, key, dout, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e == cudaSuccess && mem == 0) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
  if (mem == 0) {
    dfree(dc);
    dfree(dout);
  }
  if (e != cudaSuccess) {
    std::fprintf(stderr, "pic1d_philox: %s\n", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PIC1D_ENOMEM : PIC1D_ECUDA;
  }
  return PIC1D_OK;
}

int pic1d_set_allocator(pic1d_alloc_fn alloc, pic1d_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    std::fprintf(stderr, "pic1d_set_allocator: give both hooks or neither\n");
    return PIC1D_EINVAL;
  }
  if (g_live.load() != 0) {
    std::fprintf(stderr, "pic1d_set_allocator: %lld contexts are alive; free them first\n", g_live.load());
    return PIC1D_EINVAL;
  }
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_user = user;
  return PIC1D_OK;
}

const char* pic1d_last_error(const pic1d_ctx* c) {
  if (!c) return "no context";
  return c->err.c_str();
}

void pic1d_free(pic1d_ctx* c) {
  if (!c) return;
  if (c->s) cudaStreamSynchronize(c->s);
  else cudaDeviceSynchronize();
  free_particles(c);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  void* ptrs[] = {c->E64, c->E32, c->J, c->dens[0], c->dens[1], c->nb, c->nmu, c->nx, c->zone, c->dens_flag, c->fast_cell, c->table,
                  c->ctr, c->st, c->ke_partial, c->field_partial, c->counts, c->offsets, c->spc, c->slot_log,
                  c->tpair, c->bsum, c->sur.master, c->sur.m, c->sur.v, c->sur.img, c->sur.small,
                  c->sur.part, c->sur.loss_part, c->sur.err, c->sur_gx, c->sur_gw, c->sur_grad, c->sur_loss, c->rho,
                  c->G32, c->atmo_flag, c->atmo_w, c->atmo_cells, c->atmo_target, c->ann_list, c->ann_amount,
                  c->ann_count, c->cflag, c->dflag, c->nmu2, c->jcum, c->rho_ref, c->gauss_out, c->check,
                  c->guard_arrays, c->guard_widths};
  for (void* q : ptrs) dfree(q);
  delete c;
  g_live.fetch_sub(1);
}

}  // extern "C"
