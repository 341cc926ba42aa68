/*
 * pic1d.h -- C ABI of the B300 (sm_103a) library that advances the per-step
 * particle loop of the 1D particle-in-cell method for resonant inverse
 * Compton (RICS) drag and pair cascades on one dipole field line of a
 * magnetar (Mahlmann, Philippov, Soudais, Beloborodov, Sironi, "1D PIC
 * Simulations of Resonant Scattering-Driven Pair Cascades in Magnetar
 * Magnetospheres").
 *
 * One step (Sec. 3 of the paper) gathers E_parallel at every particle,
 * applies the continuous RICS drag in a Strang split around the Lorentz kick
 * (limiter, implicit midpoint by Newton, or damping toward p~ = mu/sqrt(1 -
 * mu^2)), draws Monte-Carlo RICS scatterings with recoil and injects e+e-
 * pairs when the scattered photon exceeds 2 m_e c^2 (App. A), moves the
 * particle, deposits a charge-conserving current and advances E from
 * Ampere's law dE/dt = 4 pi (j_ext - j) against the external twist current.
 *
 * Code units: c = 1, one cell = 1, dt = cfl.  Momentum u = gamma beta along
 * +s in units of the species' m c.  s runs from the northern footpoint
 * (s = 0) to the southern one (s = n_cells).  Positions are stored as
 * unsigned 32-bit fixed point: pos = s * 2^F with F = 32 - ceil(log2
 * n_cells).  Weights are FP32, charges are taken in fixed point w_int =
 * rint(w * 2^12).  The current is accumulated in int64: J_int[c] = sum over
 * particles of q_sign * w_int * (signed length of the step's path inside
 * cell c, in units of 2^-F); the physical current density is
 * J = q_p 2^(-F-12) J_int / dt.  E lives at cell centres (FP64).
 *
 * Scattering draw: a lepton in a pair zone with probability p_sc = min(1,
 * Ndot dt) draws one Philox4x32-10 block with counter (id_lo, id_hi, step,
 * 'RICS') and key = seed when p_sc >= 2^-24, and scatters when U = ((x0 >>
 * 8) + 1) 2^-24 (on (0, 1]) is <= p_sc; the de-excitation angle uses
 * (x1 >> 8) 2^-24.  A p_sc below 2^-24, which the 24-bit uniform cannot
 * resolve, never scatters and takes no draw.
 *
 * Conventions for every entry point:
 *   - return 0 on success, a positive warning (state consistent) or a
 *     negative error; pic1d_last_error() gives a message.  After
 *     PIC1D_ECUDA the context must be freed.
 *   - pointers tagged "host" are caller-owned host memory, read or written
 *     only during the call; "mem" arguments select host (0) or device (1)
 *     memory for the caller's arrays; device arrays must be on the device
 *     the context was created on and are used only during the call.
 *   - work is issued on the stream given in the parameters (NULL: the
 *     legacy default stream); entry points that return data synchronise
 *     that stream.
 *   - a context is not thread-safe; different contexts are independent.
 */
#ifndef PIC1D_H
#define PIC1D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
/* the most particle slots a line holds: slot indices in the kernels are
 * 32-bit, with room for one tile of slack past the capacity */
#define PIC1D_MAX_SLOTS  ((int64_t)2147483647 - 1048576)

#define PIC1D_OK          0
#define PIC1D_WCAPACITY   1   /* pairs/injections dropped: capacity full  */
#define PIC1D_EINVAL     -1   /* invalid argument                         */
#define PIC1D_ENOMEM     -2   /* device allocation failed                 */
#define PIC1D_ECUDA      -3   /* CUDA runtime error                       */
#define PIC1D_ENUMERIC   -4   /* non-finite momentum met in a step        */
#define PIC1D_ETIMEOUT   -5   /* a bounded wait inside a kernel gave up   */
#define PIC1D_ECHECK     -6   /* checking build (PIC1D_CHECK): an index out of bounds or a
                                 damaged guard region past a particle array */

/* photon field model (Sec. 2.2, App. B.2) */
#define PIC1D_PHOTON_RADIAL 0 /* radially streaming photons, solid angle pi/x^2 (Eq. contdrag) */
#define PIC1D_PHOTON_DISK   1 /* uniform-intensity stellar disk, quadrature over its solid angle */

/* drag law used by the push (Sec. 2.2, Sec. 3) */
#define PIC1D_DRAG_OFF       0
#define PIC1D_DRAG_CLOSED    1 /* closed form Eq. contdrag at the particle (radial photons)    */
#define PIC1D_DRAG_TABLE     2 /* bilinear table in (log10 gamma, s/L) built by quadrature      */
#define PIC1D_DRAG_SURROGATE 3 /* the learned network (pic1d_sur_*; set its parameters or train
                                  it before stepping), the closed form outside its box        */

/* RICS response (Sec. 3) */
#define PIC1D_RICS_SPLIT           0 /* b > b_thr: discrete scattering + pairs; else continuous drag */
#define PIC1D_RICS_DRAG_PLUS_PAIRS 1 /* continuous drag everywhere; scattering only creates pairs    */

/* surface supply (Sec. 3, App. B.1) */
#define PIC1D_INJECT_NONE 0
#define PIC1D_INJECT_RATE 1 /* neutral e- + ion pairs per footpoint per step at the rate carrying j_ext */
/* The atmosphere of Sec. 3 and App. B.1 (Eq. densprofile): a cell whose centre
 * sits at radius x (in R_star) has the target density
 * n/n0 = atmo_a0 exp(-(x - 1) R_star / atmo_h), atmo_h in cells; the
 * atmosphere is the set of cells where that is >= atmo_ncut.  After each
 * push, a cell of the atmosphere whose plasma weight (every species, after
 * the move, not counting the step's new pairs) is below
 * floor(n/n0 n0_ppc 2^12) / 2^12 receives neutral e- (PIC1D_SP_ATMO) + ion
 * pairs of weight 1 until the deficit is under one pair: positions uniform
 * in the cell, momenta Maxwellian at inject_T in both directions.  Gravity,
 * the force -inject_T/atmo_h along r (-inject_T/atmo_h mu_s along s), acts
 * on every particle inside the atmosphere (linear between cell centres, like
 * E) and is zero outside it.  Not with drag law SURROGATE. */
#define PIC1D_INJECT_TOPUP 2

/* PIC1D_ANNIHILATION -- annihilation at n_max (Sec. 3: pairs are annihilated
 * where the density reaches the skin-depth limit n_max; Sec. 5 on the
 * annihilation zone).  With annihilate_every = K > 0 (and n_max_ppc > 0),
 * at the end of every K-th step, right after a cell sort (a sort is added
 * when K is not a multiple of sort_every): a cell whose lepton weight W
 * (every lepton species, integer units of 2^-12) exceeds n_max loses the
 * same weight A = min((W - n_max)/2, W+, W-) of positrons (W+) and of pair
 * electrons (W-).  Inside each species weight is taken in increasing order
 * of the key splitmix64(id ^ splitmix64(step ^ 0xA1111A7E)) (step counted
 * after the step), the last particle touched keeping the rest of its
 * weight; particles left with no weight are removed.  The removed charge is
 * carried to the cell's left node first, which adds the current through the
 * cell to E there, so the discrete Gauss law still holds exactly.  Atmospheric
 * electrons count in W but are not annihilated.  diag.annihilated sums
 * 2A over cells and passes. */

/* species codes */
#define PIC1D_SP_ELECTRON 0
#define PIC1D_SP_POSITRON 1
#define PIC1D_SP_ION      2
#define PIC1D_SP_ATMO     3   /* electron extracted from the atmosphere */
#define PIC1D_SP_DEAD     255 /* removed slot (left the line), dropped at the next sort */

typedef struct pic1d_params {
  /* geometry, App. B.2: r = r_eq sin^2(theta), footpoints at
   * theta_0 = arcsin(sqrt(R_star/r_eq)); b = b_star (R_star/r)^3 sqrt(1+3cos^2)
   * (b_convention 0) or half of it (1, the paper's polar normalisation) */
  double r_eq;              /* equatorial radius of the line, in R*     */
  int32_t n_cells;          /* cells along the line (>= 8)              */
  double cfl;               /* dt = cfl * dx / c (0 < cfl < 1)          */
  double b_star;            /* B_* / B_QED                              */
  int32_t b_convention;
  /* photon field and drag law, Sec. 2.2 */
  double kT_keV;            /* blackbody temperature                    */
  int32_t photon_model;     /* PIC1D_PHOTON_*                           */
  int32_t drag_law;         /* PIC1D_DRAG_*                             */
  double drag_scale;        /* multiplies drag and scattering rate (1 = physical) */
  int32_t table_n_gamma;    /* table points in log10 gamma (>= 2)       */
  int32_t table_n_s;        /* table points in s/L (>= 2)               */
  double table_log10g_max;  /* table spans log10 gamma in [0, max]      */
  int32_t quad_n_mu;        /* Gauss-Legendre nodes in cos(alpha) over the disk (<= 256) */
  int32_t quad_n_phi;       /* azimuth nodes on [0, pi]                 */
  double eta_min;           /* limiter: tau_min omega_p0 = eta_min sqrt(j_psi); <= 0 disables it */
  int32_t rics_mode;        /* PIC1D_RICS_*                             */
  int32_t mc_on;            /* Monte-Carlo scattering on/off            */
  /* plasma and twist, Sec. 3 */
  double cells_per_skin_depth; /* d0: skin depth at density n0, in cells */
  double j_psi;             /* j_ext / (n0 e c)                         */
  double n0_ppc;            /* weight per cell that represents n0       */
  double mass_ratio;        /* m_i / m_e (ion charge +1)                */
  /* initial plasma (Sec. 3: a pair plasma of multiplicity M drifting at
   * beta = -+1/M, the twist current's carriers), loaded by pic1d_init when
   * ppc_e > 0: per cell ppc_e electrons at stratified positions (electron k
   * of cell c in [c + k/ppc_e, c + (k+1)/ppc_e), from one Philox4x32-10 draw
   * with counter (c, k, 0, 'INIT') and key = seed), positrons on the
   * positions of its first ppc_p electrons and ions on the next ppc_i
   * (ppc_p + ppc_i = ppc_e: every node neutral), weight 1, momenta Gaussian
   * with spread u_sigma in each species' own m c around -u_d (electrons),
   * +u_d (positrons) and 0 (ions), u_d = beta_d / sqrt(1 - beta_d^2),
   * beta_d = 1 / init_multiplicity; the Gaussian of particle k of species m
   * (0 e-, 1 e+, 2 ion) in cell c is Box-Muller on words 1 and 2 of the draw
   * (c, k, m, 'INIT').  Slots and ids: electrons cell by cell, then the
   * positrons, then the ions. */
  int32_t ppc_e, ppc_p, ppc_i;
  double init_multiplicity; /* M (> 1)                                  */
  double u_sigma;           /* spread of the initial momenta (>= 0)     */
  /* supply and pairs */
  int32_t inject_mode;      /* PIC1D_INJECT_*                           */
  double inject_T;          /* temperature of injected particles, m_e c^2 */
  double atmo_a0;           /* TOPUP: n/n0 of the atmosphere at the surface */
  double atmo_h;            /* TOPUP: scale height, cells               */
  double atmo_ncut;         /* TOPUP: the atmosphere ends where n/n0 < atmo_ncut */
  int32_t pairs_on;
  double b_pair_threshold;  /* b above which scattering is discrete and may make pairs (0.09) */
  double pair_energy_threshold; /* photon energy for a pair, m_e c^2 (2.0) */
  double n_max_ppc;         /* no pair in a cell holding this lepton weight (<= 0: off) */
  int32_t annihilate_every; /* > 0: annihilation at n_max every this many steps (PIC1D_ANNIHILATION) */
  uint64_t seed;            /* Philox key                               */
  double r_star_cm;         /* stellar radius, cm                       */
  /* library */
  int64_t capacity;         /* particle slots (0: grown on demand); at most
                               PIC1D_MAX_SLOTS (slot indices are 32-bit) */
  int32_t sort_every;       /* cell sort cadence in steps (>= 1)        */
  void* cuda_stream;        /* cudaStream_t for all work, may be NULL   */
} pic1d_params;

typedef struct pic1d_diag_t {
  int64_t step;
  int64_t n_slots;          /* used slots, including removed ones before the next sort */
  int64_t n_alive[4];       /* per species                              */
  int64_t pairs_created, pairs_dropped_cap, pairs_rejected_nmax, pairs_lost_wall;
  int64_t lost_north, lost_south, injected, injected_dropped;
  int64_t scatters, psc_clamped, limiter_branch, newton_branch, nonfinite;
  int64_t rng_draws;        /* Philox draws (one 8-byte id read each) */
  int64_t annihilated;      /* weight removed by annihilation, both species, units of 2^-12 */
  int64_t sur_rows;         /* network rows evaluated inside the push (drag law SURROGATE;
                               each row: 2 x 64 x 64 multiply-adds on the tensor cores) */
  int64_t sur_rows_tangent; /* of which with the forward-mode tangent (as many again) */
  int64_t push_launches;    /* push kernels timed since pic1d_timing(c, 1) */
  double push_ms;           /* their summed CUDA-event durations, ms     */
  int64_t push_slots;       /* sum over those launches of the slots read */
  double field_energy;      /* sum_c E_c^2 / (8 pi) after the last step          */
  double kinetic_energy;    /* q_p sum w m (gamma - 1) at the last half step     */
  double ext_work;          /* cumulative sum_n dt j_ext sum_c (E^n + E^{n+1})/2 */
  double vc;                /* circuit potential V_c = - sum_c E_c dx            */
  double ke_lost;           /* cumulative kinetic energy carried out at the walls */
  double q_p, j_ext, dt, tau_min, R_cells, L_Rstar; /* derived constants         */
  int32_t fbits, status;
  int32_t push_variant;     /* push kernel variant in use (pic1d_set_variant) */
  int32_t gauss_marked;     /* 1 after pic1d_gauss_mark (until the next set_state/load) */
  int64_t gauss_residual_max;  /* discrete continuity since the mark (pic1d_gauss_mark):
                                  max over interior nodes of |residual|, integer, 0 when
                                  charge is conserved exactly; -1 without a mark */
  int64_t gauss_residual_node; /* first node reaching it (-1 without a mark) */
} pic1d_diag_t;

typedef struct pic1d_ctx pic1d_ctx;

/* Create a context: validates the parameters, builds the geometry tables of
 * App. B.2 (host FP64), builds the drag/rate table by quadrature on the
 * device (drag_law TABLE), allocates device memory for `capacity` particles
 * (double-buffered) and leaves an empty line with E = 0 at step 0.
 * out: receives the context (NULL on failure).  Errors: EINVAL, ENOMEM, ECUDA. */
int pic1d_init(const pic1d_params* p, pic1d_ctx** out);

/* Replace the particle state and E (Sec. 3 state at time step `step`): n
 * particles in SoA form, pos fixed point (see above), u, w, species, id;
 * E has n_cells values (NULL: zero).  mem = 0 host arrays, 1 device arrays.
 * Grows the capacity if needed.  The copied state is validated on the
 * device; if any particle has a bad species or a position beyond the line
 * the call returns EINVAL and leaves an empty line (no particles).
 * Errors: EINVAL (n < 0, bad species, pos out of the line), ENOMEM, ECUDA. */
int pic1d_set_state(pic1d_ctx* c, int64_t n, const uint32_t* pos, const float* u, const float* w,
                    const uint8_t* sp, const uint64_t* id, const double* E, int64_t step, int mem);

/* Advance n_steps PIC cycles (Sec. 3) on the context's stream.  One cycle:
 * the push (gather, drag, kick, scattering and pairs, move, deposit), the
 * surface supply (RATE injection or the TOPUP atmosphere), the field update;
 * then a cell sort every sort_every steps and, with annihilate_every > 0,
 * the annihilation pass every annihilate_every steps (after a sort).
 * Asynchronous: returns after issuing the work (errors of the step show up
 * in pic1d_diag).  Errors: EINVAL (n_steps < 0), ECUDA. */
int pic1d_step(pic1d_ctx* c, int n_steps);

/* Synchronise and fill `out` (host).  Returns PIC1D_ENUMERIC if a step met
 * a non-finite momentum, PIC1D_WCAPACITY if creations were dropped since
 * init, otherwise 0. */
int pic1d_diag(pic1d_ctx* c, pic1d_diag_t* out);

/* Copy E (n_cells doubles) and/or the integer current J_int of the last
 * step (n_cells int64, zero before the first step) out; either may be NULL.  mem as above.  Synchronises. */
int pic1d_get_fields(pic1d_ctx* c, double* E, int64_t* J, int mem);

/* Number of used particle slots (alive + removed-but-unsorted); synchronises. */
int64_t pic1d_slots(pic1d_ctx* c);

/* Copy the first `n` slots (n <= pic1d_slots) of the SoA out; removed
 * slots carry species PIC1D_SP_DEAD.  Any array may be NULL.  mem as above.
 * Synchronises. */
int pic1d_get_particles(pic1d_ctx* c, int64_t n, uint32_t* pos, float* u, float* w, uint8_t* sp,
                        uint64_t* id, int mem);

/* Sort the particles by cell now (histogram, scan, scatter) and drop the
 * removed slots.  Key ((2*(ion) + (u < 0)) * n_cells + cell) * 32 + band:
 * four runs (leptons moving +s, leptons moving -s, ions moving +s, ions
 * moving -s), each in cell order, and inside a cell 32 bands of gamma,
 * band = min(floor(log2 gamma^2), 31) from the exponent of the FP32
 * gamma^2 = 1 + u^2 (rounded once).  The order inside a key is not fixed.
 * Asynchronous.  Errors: ECUDA. */
int pic1d_sort(pic1d_ctx* c);

/* Copy the drag/rate table (drag_law TABLE) out as FP32 pairs (F^, ln N^),
 * layout ((sign * n_s + js) * n_gamma + ig) * 2, sign 0 for u >= 0:
 * 2 * table_n_s * table_n_gamma * 2 floats, host memory.  F^ = F R_star/(m_e c^2)
 * (Eq. contdrag normalisation), N^ = Ndot R_star/c (Eq. scatteringNdot). */
int pic1d_get_table(pic1d_ctx* c, float* out);

/* Charge-conserving integer deposit alone (the deposit of the step, Sec. 3):
 * for n particles moving from pos0 to pos1 (int64 fixed point, pos1 may lie
 * outside [0, n_cells 2^F): the path is clamped at the walls) add
 * q_sign * rint(w 2^12) * (path length inside cell c) to J[c].  All arrays
 * are device arrays; J (n_cells int64) is accumulated into, not cleared.
 * Issued on the context's stream; synchronises. */
int pic1d_deposit(pic1d_ctx* c, int64_t n, const int64_t* pos0, const int64_t* pos1, const float* w,
                  const uint8_t* sp, int64_t* J);

/* Per-launch timing of the push kernel (the step's dominant kernel): with
 * on = 1, every push launch is bracketed by CUDA events on the context's
 * stream and pic1d_diag reports the launches, their summed duration and the
 * particle slots they read since the call; on = 0 stops it.  No effect on
 * results.  Errors: ECUDA. */
int pic1d_timing(pic1d_ctx* c, int on);

/* Check of the library's failure path for device waits: runs, on the
 * context's stream, the bounded wait that the push kernels use on their
 * copies' mbarriers, on a barrier that nothing completes (no copy is issued,
 * nothing arrives), with a limit of limit_clocks SM clocks (1 .. 4e9; at
 * 2 GHz 2e6 clocks are a millisecond).  The wait gives up, is counted like a
 * push block whose copy never landed, and the call returns PIC1D_OK once
 * the kernel has ended; the next pic1d_diag then returns PIC1D_ETIMEOUT
 * (the count restarts, so the one after it does not) and the context stays
 * usable.  The paper has no counterpart.  Errors: EINVAL, ECUDA. */
int pic1d_check_wait(pic1d_ctx* c, int64_t limit_clocks);

/* Choose the push kernel variant.  0 (the default): the streaming push, one
 * block of 32 warps per SM staging slices of the particle arrays in shared
 * memory by bulk copies (on a line with the table law and the limiter, split
 * RICS, Monte-Carlo and pairs on, its instantiation with those switches as
 * constants); 1-4: one thread per particle (or two), particles per thread x
 * minimum resident blocks per SM as pic1d_variant_info reports them; 5: the
 * per-thread push with the branch-certainty table and the current window;
 * 6, 7: the streaming push with warp-collective current flushes (32 and 24
 * warps).  Results do not depend on the variant (integer deposit, the same
 * per-particle arithmetic).  Errors: EINVAL. */
int pic1d_set_variant(pic1d_ctx* c, int variant);

/* Describe push variant `variant`; returns the number of variants, or EINVAL.
 * Either output may be NULL.  Needs no context. */
int pic1d_variant_info(int variant, int* particles_per_thread, int* min_blocks_per_sm);

/* Cell sort without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code that
 * runs inside a device memory pool it does not own, or on a device whose
 * memory an application has reserved in full -- and so cannot create a
 * context, whose sort scratch comes from cudaMalloc.  It sorts n particles of
 * a line of n_cells cells (SoA device arrays in the layout above) by the key
 * ((2*(ion) + (u < 0)) * n_cells + cell) * 32 + band (the key of pic1d_sort), drops removed slots (species PIC1D_SP_DEAD), writes
 * the sorted particles to the *_out device arrays (capacity n each) and the
 * number kept to *n_out (a device int64).  The order inside one key is not
 * specified.  Input and output arrays must not overlap.
 *
 * Its scratch (histogram, offsets, block sums, counters; about 100.7 MB) is one
 * fixed-size device array inside this library: every GPU that loads the
 * library holds it until the process exits, so n_cells is limited to
 * PIC1D_SORT_STATIC_MAX_CELLS and larger lines are rejected with
 * PIC1D_EINVAL and a message on stderr.  Every call looks up the array's
 * device address in the current context (cudaGetSymbolAddress, no stream
 * work; after a cudaDeviceReset the module is loaded again and the new
 * address is found); make the first call on a device outside any stream
 * capture, since it may load the module.  Every call uses the same array:
 * calls that overlap on
 * the GPU (on different streams, or from different host threads) race and
 * corrupt each other's results; serialise them.  The histogram is cleared
 * by each call.  Work is issued on cuda_stream (NULL: legacy default
 * stream) and the call returns without synchronising.
 * Errors: EINVAL (n_cells outside [8, PIC1D_SORT_STATIC_MAX_CELLS], n < 0 or
 * n >= 2^31, a NULL array), ECUDA. */
#define PIC1D_SORT_STATIC_MAX_CELLS 65536
int pic1d_sort_static(int32_t n_cells, int64_t n, const uint32_t* pos, const float* u, const float* w,
                      const uint8_t* sp, const uint64_t* id, uint32_t* pos_out, float* u_out, float* w_out,
                      uint8_t* sp_out, uint64_t* id_out, int64_t* n_out, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Test-particle drag maps (the paper's appendix on the extent of the
 * pair-producing region, Figs. 6 and 7).  For each of n field lines of
 * equatorial radius r_eq[i], a lepton enters at the northern footpoint with
 * gamma0 and moves under the drag alone, from radially streaming photons
 * (Eq. contdrag) with the physics of `p` (b_star, b_convention, kT_keV,
 * r_star_cm, drag_scale; the other fields are not used).  One GPU thread
 * follows one line in FP64 with steps of dt (R_star/c): the drag update
 * u1 - u0 - dt/2 (F(u0) + F(u1)) = 0 by Newton at fixed theta, the expected
 * scatterings tau += dt/2 (N(u0) + N(u1)), and theta += dt/2 (beta0 + beta1) /
 * (ds/dtheta).  It stops at the equator or at t_max.  Per line: gamma_min;
 * the first scattering (tau = 1) as theta_first and s_first (-1: none); the
 * point where b falls below b_thr (theta_b, s_b; the equator if it does not);
 * the line length L; l_pp = s_b - s_first, or L - 2 s_first when b stays
 * above b_thr to the equator (the zone spans both hemispheres); b at the
 * equator; region 1 (b > b_thr everywhere, gamma_min > 1 + gamma_eps), 2 (b
 * falls below b_thr, gamma_min > 1 + gamma_eps) or 3 (gamma_min <= 1 +
 * gamma_eps).  out: host, n results; ms_out (may be NULL): the kernel's
 * device time.  Errors: EINVAL, ENOMEM, ECUDA.
 * ------------------------------------------------------------------------ */
typedef struct pic1d_tp_result {
  double gamma_min, theta_first, theta_b, s_first, s_b, L, l_pp, b_eq, t_end, u_end;
  int64_t steps;
  int32_t region, pad;
} pic1d_tp_result;

int pic1d_tp_map(const pic1d_params* p, const double* r_eq, int32_t n, double gamma0, double dt, double t_max,
                 double b_thr, double gamma_eps, pic1d_tp_result* out, double* ms_out);

/* Charge density at the N+1 nodes (the CIC shape of Sec. 3's grid): for a
 * live particle at pos = i 2^F + f, node i gets q w_int (2^F - f) and node
 * i+1 gets q w_int f, in the units of the current J (charge x 2^F, w_int =
 * rint(w 2^12)).  The discrete Gauss law then reads rho^{n+1} - rho^n =
 * -(J_i - J_{i-1}) at every interior node, exactly.  rho: N+1 int64, host
 * (mem 0) or device (mem 1).  Synchronises.  Errors: EINVAL, ECUDA. */
int pic1d_get_rho(pic1d_ctx* c, int64_t* rho, int mem);

/* Mark the state for the discrete continuity check (Sec. 3: the deposit
 * conserves charge, so Gauss's law dE/ds = 4 pi rho stays satisfied if it
 * held).  Records the node charge rho_ref (as pic1d_get_rho) and restarts
 * the cumulative current Jcum of every cell, which each step's field update
 * and each annihilation pass (a current -X in the cell whose left node takes
 * the removed charge) add to.  From then on pic1d_diag reports, in the
 * integer units of pic1d_get_rho,
 *   max over nodes 1..N-1 of |rho_i - rho_ref_i - (Jcum_{i-1} - Jcum_i)|,
 * which is 0 as long as every particle's charge moves only by the deposit
 * (pairs and supply are created neutral at one position; losses change only
 * the wall nodes; a particle removed for a non-finite momentum breaks it).
 * set_state and load clear the mark.  Costs one charge deposit per mark and
 * per diag call.  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA. */
int pic1d_gauss_mark(pic1d_ctx* c);

/* Checkpoint and resume.  pic1d_save writes the context's whole state to a
 * file: the parameters (to be checked on load), the step, the particle slots
 * (including removed ones not yet dropped by a sort), E (FP64), the last
 * step's J, the pair-cap densities of this step and the next, the counters
 * and per-step scalars (with the surface-supply accumulators), and the
 * surrogate network with its Adam state if the context has one.
 * pic1d_load restores such a file into a context created with the same
 * parameters (the stream and the capacity may differ; the capacity must hold
 * the saved slots): stepping on from there gives what the saved context
 * would have given.  Push timing records are not saved.  Both synchronise.
 * Errors: EINVAL (cannot open, not a checkpoint, other parameters, truncated),
 * ENOMEM, ECUDA. */
int pic1d_save(pic1d_ctx* c, const char* path);
int pic1d_load(pic1d_ctx* c, const char* path);

/* ------------------------------------------------------------------------
 * Learned surrogate of the photon-field quadrature (Sec. 2.2, Eq.
 * scatteringNdot and the momentum given per scattering).
 *
 * An MLP 4 -> 64 -> 64 -> 64 -> 2 with SiLU activations, BF16 weights and
 * activations and FP32 accumulation.  Per photon direction a scattering gives
 * the lepton the momentum gamma b mu~ along s (mu~ the cosine of the
 * direction in the lepton frame), so F^ = gamma b N^ <mu~>, <mu~> the
 * rate-weighted mean of mu~ (in [-1, 1]).  The network maps
 *   f0 = 2 log10(gamma)/G - 1, f1 = 2 s/L - 1, f2 = (log10 b + 1.25)/2.75,
 *   f3 = sign(u)
 * to y0 ~ <mu~> and y1 ~ max(ln N^, -30) - max(B, -30), where B = ln(0.9
 * N^_rad(mu_s) + 0.1 N^_rad(mu_e)) is the closed form for photons along one
 * direction [contdrag] taken along the radial and along the disk edge most
 * favourable to the resonance; -30 clamps the targets, and the network is
 * scored where ln N^ > -20 (below it a rate is negligible).  G is the
 * context's table_log10g_max; the quadrature uses the context's photon
 * model, kT, quad_n_mu x quad_n_phi nodes, b_star and b_convention.
 *
 * Parameters: PIC1D_SUR_N_PARAMS FP32 values, layer by layer W[out][in]
 * then b (W1 64x4, b1, W2 64x64, b2, W3 64x64, b3, W4 2x64, b4).  The
 * context keeps FP32 master values; the tensor-core layers use the BF16
 * roundings of W2 and W3 (and BF16 activations), the rest stays FP32.
 *
 * Sample records (PIC1D_SUR_RECORD floats each, device memory):
 *   0-3 f0..f3 | 4 t1 = <mu~> | 5 t2 (the y1 target) | 6 mask (1 where
 *   ln N^ > -30) | 7 B | 8 ln N^ | 9 F^ | 10 F^_abs (the quadrature of
 *   |momentum| x rate, the scale of the drag error) | 11 gamma | 12 b |
 *   13 u | 14 x = r/R* | 15 mu_s
 * Loss of a batch: mean of mask (y0 - t1)^2 + (y1 - t2)^2.
 * ------------------------------------------------------------------------ */
#define PIC1D_SUR_N_PARAMS 8770
#define PIC1D_SUR_RECORD 16

typedef struct {
  int64_t n_samples;   /* training samples (1e7)                           */
  int32_t epochs;      /* 20                                               */
  int32_t batch;       /* 8192 (a multiple of 128)                         */
  double lr;           /* Adam learning rate (1e-3; beta 0.9, 0.999, eps 1e-8) */
  double lr_final;     /* > 0: cosine decay from lr to lr_final over the run; <= 0: constant */
  double r_lo, r_hi;   /* r_eq of the sampled lines, log-uniform (equal: one line) */
  uint64_t seed;       /* Philox key of the training samples and the shuffles */
  int64_t n_val;       /* held-out validation samples                      */
  uint64_t val_seed;   /* their Philox key                                 */
} pic1d_train_cfg;

typedef struct {
  int64_t steps, n_samples, n_val, val_count;   /* val_count: records with ln N^ > -20 */
  double samples_ms, train_ms, val_ms;          /* device time of each phase */
  double loss_first, loss_last;                 /* mean batch loss, first and last step */
  double drag_err_max, drag_err_p99, drag_err_median;  /* |F_nn - F_q| / (|F_q| + F_abs) */
  double lnN_err_max, lnN_err_p99, lnN_err_median;     /* |ln N_nn - ln N_q| */
} pic1d_train_report;

/* Set (host, PIC1D_SUR_N_PARAMS values) or read back the master parameters.
 * Setting resets the Adam moments and step count.  Errors: EINVAL, ECUDA. */
int pic1d_sur_set_params(pic1d_ctx* c, const float* theta);
int pic1d_sur_get_params(pic1d_ctx* c, float* theta);

/* n sample records from index `start` of the set keyed by `seed` (one
 * Philox4x32-10 draw per record, counter (index, 0, 0x53555247), key = seed:
 * log10 gamma = G U0, s/L = U1, sign from the top bit of word 2, r_eq =
 * r_lo (r_hi/r_lo)^U3, U = (word >> 8) 2^-24), by FP64 quadrature on the
 * device.  out: device, n x PIC1D_SUR_RECORD floats.  Errors: EINVAL, ECUDA. */
int pic1d_sur_samples(pic1d_ctx* c, uint64_t seed, uint64_t start, int64_t n, double r_lo, double r_hi,
                      float* out_dev);

/* Gradient of the mean loss over n records (device, 1 <= n <= 65536) at the
 * current parameters: grad_host receives PIC1D_SUR_N_PARAMS values, loss_host
 * the mean loss.  Errors: EINVAL, ECUDA, ETIMEOUT. */
int pic1d_sur_grad(pic1d_ctx* c, const float* samples_dev, int64_t n, float* grad_host, double* loss_host);

/* `steps` Adam steps on consecutive batches of `batch` records (device),
 * batch k taking records k*batch .. k*batch+batch-1 modulo n (no shuffle).
 * Errors: EINVAL, ECUDA, ETIMEOUT. */
int pic1d_sur_train_steps(pic1d_ctx* c, const float* samples_dev, int64_t n, int32_t batch, int32_t steps,
                          double lr);

/* Network outputs for n rows of `stride` floats (device; inputs f0..f3 in
 * the first four columns): out (device, n x 4) = y0, y1, dy0/df0, dy1/df0.
 * Errors: EINVAL, ECUDA, ETIMEOUT. */
int pic1d_sur_infer(pic1d_ctx* c, const float* feat_dev, int32_t stride, int64_t n, float* out_dev);

/* Train the context's network from its current parameters: n_samples records
 * by quadrature (seed), epochs x (n_samples / batch) Adam steps over
 * batches drawn without replacement (a fresh affine permutation of the
 * records per epoch), then the drag and rate errors on n_val held-out
 * records (val_seed).  rep (host) receives the timings and errors.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
int pic1d_train_surrogate(pic1d_ctx* c, const pic1d_train_cfg* cfg, pic1d_train_report* rep);

/* ------------------------------------------------------------------------
 * Ensemble: many independent field lines advanced together (the paper runs
 * one line per simulation; batching lines of uneven lengths and particle
 * counts is this library's addition).  Each line is a full context of its
 * own (its geometry, particles, fields, counters; pic1d_ens_line gives it
 * for set_state, diag, get_fields, get_particles).  Every phase of a step is
 * one launch for all lines: a persistent push kernel takes (line, tiles)
 * items from one queue, one field kernel and one finalize kernel cover all
 * lines, and each line is sorted every sort_every of its own steps.  A
 * super-step of 80 steps is captured once as a CUDA graph and replayed
 * (sort cadences are 10, 20 or 40 steps, so every line's buffer flips an
 * even number of times per super-step).  Per line the results are those of
 * the line advanced alone.
 *
 * The ensemble runs drag law PIC1D_DRAG_SURROGATE with one network for all
 * lines: the network of line 0's context (pic1d_sur_set_params or
 * pic1d_train_surrogate on pic1d_ens_line(e, 0)).  A line may have a surface
 * supply (RATE or the atmosphere, TOPUP) and annihilation at n_max: its
 * supply runs after the push of every step, its annihilation after the sort
 * at the end of every annihilate_every-th step, as for the line alone (the
 * kernels read the step from the line's device state, so that the captured
 * super-steps draw the random numbers of the steps they replay).  The
 * ensemble works on a stream of its own (cuda_stream of the parameters is
 * not used); pic1d_ens_step is asynchronous, the per-line calls synchronise.
 * ------------------------------------------------------------------------ */
typedef struct pic1d_ens pic1d_ens;

/* Create n_lines lines from params[0..n_lines-1] (drag_law SURROGATE, one
 * stream for all, capacity per line; annihilate_every, where set, divides the
 * super-step of 80).  Errors: EINVAL, ENOMEM, ECUDA. */
int pic1d_ens_init(const pic1d_params* params, int32_t n_lines, pic1d_ens** out);

/* The context of one line (owned by the ensemble; NULL if out of range). */
pic1d_ctx* pic1d_ens_line(pic1d_ens* e, int32_t line);

/* Per-line schedule: push items of chunk_tiles x 128 slots and a sort every
 * sort_every steps (10, 20 or 40).  Either array may be NULL (unchanged).
 * Errors: EINVAL. */
int pic1d_ens_set_schedule(pic1d_ens* e, const int32_t* chunk_tiles, const int32_t* sort_every);
int pic1d_ens_get_schedule(pic1d_ens* e, int32_t* chunk_tiles, int32_t* sort_every);

/* Advance every line by n_steps: whole super-steps of 80 replay the captured
 * graph (captured again when the schedule or a line's buffer or step phase
 * changed), the rest is launched directly.  Errors: EINVAL (no network),
 * ECUDA. */
int pic1d_ens_step(pic1d_ens* e, int n_steps);

/* Autotuner: for every pair (chunk_tiles in {1, 4, 16}, sort_every in {10,
 * 20, 40}) run max(trial_steps, sort_every) real steps of all lines, with
 * each line's push time measured in SM clocks inside the push and each sort
 * timed with events; per line keep the pair of least push time per step
 * plus sort time per sort / sort_every.  The trial steps advance the lines.
 * Outputs (host, n_lines each, may be NULL): the chosen chunk_tiles and
 * sort_every and the estimated ms per step.  Errors: EINVAL, ECUDA. */
int pic1d_ens_tune(pic1d_ens* e, int32_t trial_steps, int32_t* chunk_out, int32_t* cadence_out,
                   double* cost_ms);

/* The ensemble's CUDA stream (a cudaStream_t), for events and synchronisation. */
void* pic1d_ens_stream(pic1d_ens* e);

/* Per-step history of every line, kept on the device by the step's last
 * kernel (recorded inside captured super-steps too, no host
 * synchronisation): after each of the next `capacity` steps, the line's
 * circuit potential V_c = -sum_c E_c dx (Sec. 3) and its cumulative count of
 * created pairs.  A call re-arms the record (the previous one is dropped);
 * capacity 0 stops recording.  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA. */
int pic1d_ens_record(pic1d_ens* e, int32_t capacity);

/* Line `line`'s record: *n_out steps (<= capacity); vc[k] = V_c after the
 * k-th recorded step, pairs[k] = pairs created since the record was armed,
 * pair_rate[k] = pairs created per unit time (cell-crossing times) over the
 * last `window` steps, over the k + 1 steps recorded while k + 1 < window --
 * with window = n_cells / cfl steps, the rate averaged over a light-crossing
 * time of the line that the paper reports.  Output arrays are caller-owned
 * host memory of `capacity` entries, each may be NULL.  Synchronises.
 * Errors: EINVAL (no such line, window < 1 with pair_rate), ECUDA. */
int pic1d_ens_history(pic1d_ens* e, int32_t line, int32_t window, double* vc, int64_t* pairs, double* pair_rate,
                      int32_t* n_out);

const char* pic1d_ens_last_error(const pic1d_ens* e);
void pic1d_ens_free(pic1d_ens* e);

/* The library's random numbers on caller-given counters: Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, SC'11; ten rounds) with key (key & 0xffffffff,
 * key >> 32), so that a caller can reproduce any draw of a step.  The push
 * draws the scattering of a lepton with counter (id_lo, id_hi, step,
 * 0x52494353) and key = seed; the RATE supply with (slot, footpoint, step,
 * 0x494E4A31) and the atmosphere with (slot, cell, step, 0x41544D4F).
 * ctr: n counters of four u32 words; out: n outputs of four u32 words.
 * mem 0: host arrays; 1: device arrays, 16-byte aligned.  Needs no context;
 * runs on the default stream and synchronises.
 * Errors: EINVAL (n < 0, NULL arrays, misaligned device arrays), ENOMEM, ECUDA. */
int pic1d_philox(const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out, int mem);

/* Device memory.  Contexts and ensembles take all their device memory from
 * one process-wide allocator: cudaMalloc / cudaFree by default, or the
 * caller's pair of hooks (for instance a framework's caching allocator, so
 * that the library's buffers and the framework's share one pool).  alloc
 * returns a device pointer to `bytes` bytes aligned to at least 256 bytes,
 * or NULL on failure (the call then fails with ENOMEM); free_fn releases
 * it.  Both NULL restores cudaMalloc / cudaFree.  The hooks may be changed
 * only while no context is alive, so that every buffer is freed by the
 * allocator that made it.  Errors: EINVAL (one hook without the other,
 * contexts alive). */
typedef void* (*pic1d_alloc_fn)(size_t bytes, void* user);
typedef void (*pic1d_free_fn)(void* ptr, void* user);
int pic1d_set_allocator(pic1d_alloc_fn alloc, pic1d_free_fn free_fn, void* user);

/* Message of the last error on this context (never NULL). */
const char* pic1d_last_error(const pic1d_ctx* c);

/* Release the context and its device memory (NULL is a no-op). */
void pic1d_free(pic1d_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* PIC1D_H */
