// pic1d_internal.h -- data shared between the host glue and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pic1d.h"

namespace pic1d {

constexpr int kBlock = 256;          // threads per block of the particle kernels
constexpr int kPerThread = 4;        // particles per thread (128-bit SoA loads)
constexpr int kTile = kBlock * kPerThread;
constexpr int kWindow = 2048;        // cells of the shared-memory deposit window
constexpr int kChunkTiles = 32;      // tiles per dynamically scheduled chunk of the push
constexpr int kWBits = 12;           // weight fixed point: w_int = rint(w * 2^12)
constexpr uint32_t kTagRics = 0x52494353u;
constexpr uint32_t kTagInj = 0x494E4A31u;
constexpr uint32_t kTagAtmo = 0x41544D4Fu;   // atmosphere top-up draws
constexpr uint32_t kTagInit = 0x494E4954u;   // initial load draws
constexpr int kMaxFieldBlocks = 1024;
// cell flags of the streaming push
constexpr uint8_t CF_ZONE = 1;       // pair zone: Monte-Carlo RICS instead of continuous drag (SPLIT)
constexpr uint8_t CF_WALL = 2;       // end cell: a particle can leave the line
constexpr uint8_t CF_DENSN = 4;      // a cell of the pair cap's density within one cell
constexpr uint8_t CF_ATMO = 8;       // an atmosphere cell within one cell (gravity, weight sums)
// bins of the cell sort's key inside one cell (octaves of gamma^2, the last open)
constexpr int kSortBands = 32;
// entries of the branch-certainty table
constexpr uint8_t kDampCertain = 1;  // the limiter test chooses damping
constexpr uint8_t kNewtonStill = 2;  // it chooses Newton, whose update leaves u unchanged in FP32
constexpr uint8_t kRateNil = 4;      // the scattering probability is below the draw's resolution 2^-24
// index of the branch-certainty table in gamma^2: the exponent and the top
// kDampMant mantissa bits of (float)gamma^2, (bits >> kDampShift) -
// kDampE2Base, kDampNE of them (gamma^2 up to 2^64)
constexpr int kDampMant = 1;
constexpr int kDampShift = 23 - kDampMant;
constexpr unsigned kDampE2Base = 0x3F800000u >> kDampShift;   // 1.0f
constexpr int kDampNE = 64 << kDampMant;

// Device-side counters, accumulated over the life of the context.
struct Counters {
  unsigned long long pairs_created, pairs_dropped_cap, pairs_rejected_nmax, pairs_lost_wall;
  unsigned long long lost_north, lost_south, injected, injected_dropped;
  unsigned long long scatters, psc_clamped, limiter_branch, newton_branch, nonfinite;
  unsigned long long rng_draws;
  unsigned long long sur_rows;   // rows evaluated by the surrogate network inside the push
  unsigned long long sur_rows_tangent;   // of which with the forward-mode tangent
  unsigned long long annihilated;        // weight removed by annihilation (w_int units)
  unsigned long long waits_timed_out;    // push blocks whose bounded wait on a copy gave up
};

// Per-step device scalars.
struct StepState {
  long long n_slots;        // slots read by the particle kernels
  long long append;         // slots appended during the current step
  long long sorted_total;   // alive count produced by the sort scan
  double inj_acc[2];        // RATE injection accumulators (north, south)
  double field_energy, vc, ext_work, kinetic, ke_lost;
  unsigned long long work;  // next chunk of the push's dynamic schedule (cleared before each push)
  long long step;           // steps taken (kept on the device for the ensemble's captured graphs)
};

// Everything a particle kernel needs, passed by value.
// Checking build (compiled with -DPIC1D_CHECK, libpic1d_check.so): the
// kernels test the indexes below before they use them, record a failed test
// as a bit of *P.check and skip the access; the host fills the slack past
// every particle array with a guard pattern and tests it after each step.
// In the product build the tests compile to nothing.
enum CheckBit : unsigned {
  kChkCell = 1u,       // a cell index from a position outside [0, N)
  kChkSlot = 2u,       // a slot index at or past the capacity
  kChkGather = 4u,     // a field gather outside [0, N)
  kChkSortDst = 8u,    // a sort destination at or past the capacity
  kChkSortKey = 16u,   // a sort key outside the histogram
  kChkGuard = 32u,     // the guard region past a particle array was written
};
#ifdef PIC1D_CHECK
#define PIC1D_BOUND(P, cond, bit) ((cond) ? true : (atomicOr((P).check, (unsigned)(bit)), false))
#else
#define PIC1D_BOUND(P, cond, bit) true
#endif

struct DevParams {
  int N, F;
  long long top;            // N << F
  uint32_t top1;            // top - 1
  float inv2F;              // 2^-F
  float dt, half_dt;
  float qm[4];              // q/m per species in units of e/m_e
  int qs[4];                // charge sign per species
  float mass[4];
  int drag_law, rics_mode, mc_on, pairs_on, limiter_on, use_nmax;
  float drag_k;             // drag_scale / R_cells: F^ and N^ per R_star/c -> per cell-crossing time
  float tau_min, damp;      // limiter floor and exp(-dt/(2 tau_min))
  float pair_e_thr;
  long long nmax_int;
  // table
  int Ng, Ns;
  float t_scale;            // log2(gamma) -> table index
  float dtdu_scale;         // 1/(ln 10 * dlog10g)
  float v_scale;            // pos -> s/L index
  // closed form (radial photons)
  float theta_T;            // kT / m_e c^2
  float closedK;            // r_e R* theta^3 / (4 lbar^2)  (divide by x^2)
  float closedN;            // r_e R* / (4 lbar^2)          (divide by x^2 gamma)
  uint32_t key0, key1;
  long long step;
  // arrays
  uint32_t* pos; float* u; float* w; uint8_t* sp; uint64_t* id;
  const float* E32;
  long long* J;
  const float4* tpair;      // table with neighbouring s-rows paired
  const float* nb; const float* nmu; const float* nx;
  const float2* nmu2;       // (mu[c], mu[c+1]) per cell
  const uint8_t* zone;
  const uint8_t* dens_flag; // cells where the pair cap can be tested: zone cells and their neighbours
  const uint8_t* fast_cell; // no zone cell within two cells and not at a wall: the push's fast path
  const uint8_t* cflag;     // per cell: CF_* bits of the streaming push
  const uint8_t* dflag;     // branch certain: [sign][s-row pair][half-octave of gamma^2] (table law, limiter on)
  long long* dens_cur; long long* dens_next;
  // atmosphere (inject mode TOPUP; null otherwise)
  const float* G32;         // gravity along s per unit mass at cell centres (zero outside the atmosphere)
  const uint8_t* atmo_flag; // cells of the atmosphere
  long long* jcum;          // cumulative J per cell since pic1d_gauss_mark (null: not kept)
  long long* atmo_w;        // plasma weight (w_int) per cell after the move, summed by the push
  unsigned* check;          // checking build: bits of the bounds that failed (null otherwise)
  long long cap;
  Counters* ctr;
  StepState* st;
  double* ke_partial;       // one per block of the push
  // learned surrogate (drag law SURROGATE)
  const uint8_t* sur_img;   // BF16 operand images of layers 2 and 3
  const float* sur_small;   // FP32 layers 1 and 4 and the biases
  float sur_G;              // table_log10g_max: f0 = 2 log10(gamma)/G - 1
  float sur_lnP;            // ln(r_e R* / (4 lbar^2))
  unsigned* sur_err;
};

}  // namespace pic1d

// kernel launchers (kernels.cu)
namespace pic1d {
cudaError_t launch_push(const DevParams& P, int variant, int grid, cudaStream_t s);
cudaError_t launch_push_sur(const DevParams& P, int grid, cudaStream_t s);   // drag law SURROGATE
int push_variant_count();
int push_variant_ppt(int v);
int push_variant_minb(int v);
cudaError_t launch_inject(const DevParams& P, double carriers_per_step, float sig_e, float sig_i,
                          cudaStream_t s);
// annihilation at n_max, right after a sort (offsets: the sort's bin ends, counts: its histogram);
// list/amount/count: scratch of N cells, N cells, 1 counter; cJ: E change per unit of J_int
cudaError_t launch_annihilate(const DevParams& P, const uint32_t* counts, const long long* offsets, int* list,
                              long long* amount, unsigned* count, double* E64, float* E32, double cJ, int sms,
                              cudaStream_t s);
// Philox4x32-10 of n counters (16-byte aligned device arrays of n x 4 u32), key (lo, hi)
cudaError_t launch_philox(const void* ctr, long long n, unsigned long long key, void* out, cudaStream_t s);
// atmosphere top-up (TOPUP): n_cells cells of the atmosphere with their target weights (w_int)
cudaError_t launch_topup(const DevParams& P, const int* cells, const long long* target, int n_cells, float sig_e,
                         float sig_i, cudaStream_t s);
cudaError_t launch_field(const DevParams& P, double* E64, float* E32, double four_pi_dt_jext, double cJ,
                         double dt_jext, double* field_partial, int grid_push, cudaStream_t s);
cudaError_t launch_sort(const DevParams& P, uint32_t* counts, long long* offsets, long long* bsum,
                        uint32_t* pos2, float* u2, float* w2, uint8_t* sp2, uint64_t* id2, int sms,
                        cudaStream_t s);
cudaError_t launch_pair_table(const float2* t, int Ng, int Ns, float4* out, cudaStream_t s);
int sort_bins(int N);
int scan_blocks(int N);
cudaError_t launch_table(int Ng, int Ns, int n_mu, int n_phi, double log10g_max, double theta_T,
                         double pref, const double* xs, const double* bs, const double* mus, const double* gx,
                         const double* gw, int photon_model, float2* out, cudaStream_t s);
cudaError_t launch_deposit(const DevParams& P, long long n, const long long* p0, const long long* p1,
                           const float* w, const uint8_t* sp, long long* J, cudaStream_t s);
cudaError_t launch_count_species(const DevParams& P, unsigned long long* out4, cudaStream_t s);
cudaError_t launch_rho(const DevParams& P, long long* rho, int grid, cudaStream_t s);
cudaError_t launch_guard_check(const uint8_t* const* arrays, const int* widths, int n_arrays, long long cap,
                               long long alloc, unsigned* check, cudaStream_t s);
cudaError_t launch_gauss_residual(const DevParams& P, const long long* rho, const long long* rho_ref,
                                  unsigned long long* out2, cudaStream_t s);
int push_blocks_per_sm(int variant, bool nmax);
// the streaming push (push_stream.cu): one block per SM, `shape` one of
// stream_variant_count() (consumer warps x slots per lane)
cudaError_t launch_push_stream(const DevParams& P, int shape, int grid, cudaStream_t s);
int stream_variant_count();
// a bounded wait that nothing completes, for pic1d_check_wait
cudaError_t launch_wait_check(Counters* ctr, long long limit_clocks, cudaStream_t s);
int stream_variant_ppl(int shape);
// the damping-certainty table from the paired drag table (table law, limiter on)
cudaError_t launch_damp_flags(const float4* tpair, int Ng, int Ns, float t_scale, float drag_k, float tau_min,
                              float dt, uint8_t* out, cudaStream_t s);
}  // namespace pic1d

// learned surrogate of the photon-field quadrature (surrogate.cu)
namespace pic1d {
// flat parameter layout: W[out][in] then b, layer by layer (4-64-64-64-2)
constexpr int W_OW1 = 0, W_OB1 = 256, W_OW2 = 320, W_OB2 = 4416, W_OW3 = 4480, W_OB3 = 8576, W_OW4 = 8640,
              W_OB4 = 8768, W_N_PARAMS = 8770;
constexpr int kSurRecord = 16;   // floats per sample record

struct SurPhys {              // what the quadrature needs about the star and the photon field
  double theta_T;             // kT / (m_e c^2)
  double pref;                // r_e R* / (4 pi lbar^2)
  double log10g_max;          // gamma range of the samples: [1, 10^log10g_max]
  double b_star;
  int b_convention, photon_model, n_mu, n_phi;
  const double* gx;           // Gauss-Legendre nodes and weights on [-1, 1] (device)
  const double* gw;
};

struct SurBufs {              // device buffers of one network
  float* master;              // FP32 master parameters
  float* m;                   // Adam moments
  float* v;
  uint8_t* img;               // BF16 tensor-core operand images (32 KB)
  float* small;               // FP32 copies of layers 1 and 4 and the biases
  float* part;                // gradient partials [tiles][W_N_PARAMS]
  float* loss_part;           // [tiles]
  unsigned* err;              // set when a wait inside a kernel gave up
  int max_tiles;
};

cudaError_t sur_launch_samples(const SurPhys& Q, unsigned long long seed, unsigned long long start, long long n,
                               double r_lo, double r_hi, float* out, cudaStream_t s);
cudaError_t sur_launch_train(const SurBufs& B, const float* samples, long long n, unsigned long long perm_a,
                             unsigned long long perm_c, long long row0, int rows, cudaStream_t s);
cudaError_t sur_launch_update(const SurBufs& B, int tiles, int mode, float lr, int adam_t, float* grad_out,
                              float* loss_out, cudaStream_t s);
cudaError_t sur_launch_infer(const SurBufs& B, const float* feat, int stride, long long n, float* out, int grid,
                             cudaStream_t s);
cudaError_t sur_launch_val(const float* rec, const float* y, long long n, float* err2, cudaStream_t s);
}  // namespace pic1d

// ensemble of lines (kernels.cu, pic1d.cu)
namespace pic1d {
// device record of one line of an ensemble
struct EnsLine {
  DevParams P;                       // pointers of the current particle buffer
  uint32_t* pos[2];
  float* u[2];
  float* w[2];
  uint8_t* sp[2];
  uint64_t* id[2];
  long long* dens[2];
  double* E64;
  float* E32;
  double a, cJ, dt_jext;             // field update constants of the line
  double acc[4];                     // per-step sums: E_old, E_new, E_new^2, kinetic energy
  unsigned long long cycles;         // SM clocks spent on the line's push items (autotuner)
  int cur;
  int pad;
};

// per-step record of every line (pic1d_ens_record): V_c and the cumulative
// pair count after each step, line l's step k at [l * cap + k]
struct EnsRec {
  double* vc;
  long long* pairs;
  int* n;                            // steps recorded per line
  int cap;                           // steps per line the buffers hold (0: not recording)
  int pad;
};

struct EnsArgs {
  EnsLine* lines;
  int n_lines;
  const int4* push_items;            // (line, first tile, tiles, 0)
  int n_push_items;
  const int2* cell_items;            // (line, first cell) of 256-cell blocks
  int n_cell_items;
  unsigned long long* work;          // next push item
  const uint8_t* sur_img;            // the shared network
  const float* sur_small;
  unsigned* sur_err;
  EnsRec* rec;                       // the record's descriptor (device; cap 0 when off)
};

cudaError_t ens_launch_clear(const EnsArgs& A, cudaStream_t s);
cudaError_t ens_launch_push(const EnsArgs& A, int grid, cudaStream_t s);
cudaError_t ens_launch_field(const EnsArgs& A, cudaStream_t s);
cudaError_t ens_launch_finalize(const EnsArgs& A, cudaStream_t s);
cudaError_t ens_launch_flip(EnsLine* lines, int line, cudaStream_t s);
}  // namespace pic1d

// test-particle drag maps (tp_map.cu)
namespace pic1d {
cudaError_t tp_launch_map(const pic1d_params& p, const double* r_eq_dev, int n, double gamma0, double dt,
                          double t_max, double b_thr, double gamma_eps, pic1d_tp_result* out_dev,
                          cudaStream_t s);
}  // namespace pic1d
