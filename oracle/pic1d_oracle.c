/*
 * pic1d_oracle.c -- plain FP64 CPU oracle of the per-step particle loop of the
 * 1D particle-in-cell method for resonant-inverse-Compton (RICS) pair
 * cascades on one dipole field line (Mahlmann, Philippov, Soudais,
 * Beloborodov, Sironi: "1D PIC Simulations of Resonant Scattering-Driven Pair
 * Cascades in Magnetar Magnetospheres").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or constant generator with the CUDA library; it is written to
 * be read against the paper, not to be fast.  Every quantity is FP64.
 *
 * Sections of the paper followed (LaTeX equation labels in brackets):
 *   geometry            App. B.2 (dipole B_d, theta_0, mu = B^r/B_d)
 *   resonance           Sec. 2.1 [elandau, resonancerest, resomega]
 *   scattering rate     Sec. 2.2 [scatteringNdot]
 *   drag force          Sec. 2.2 [contdrag]
 *   PIC cycle           Sec. 3 (CFL step, Ampere with external current,
 *                       conductor walls, Strang-split drag, limiter,
 *                       implicit midpoint [implicit], damping to p~)
 *   MC RICS + pairs     Sec. 3, App. A.1-A.3 [exen, excitedgamma, scatlim1,
 *                       perpemit, paremit] and the E_gamma(theta) formula
 *
 * Readings where the paper is silent or ambiguous (each one is a parameter or
 * a documented choice, the CUDA library follows the same one):
 *   - E at cell centres, charge at nodes, linear (CIC) shape; the current
 *     through a face is the signed length of the particle path inside that
 *     cell (the 1D charge-conserving deposit); gather interpolates E
 *     linearly between cell centres, constant beyond the outer centres.
 *   - RICS zones are decided per cell: b at the cell centre > b_thr gives
 *     discrete scattering (+ pairs), otherwise continuous drag (SPLIT mode).
 *   - tau_min = eta_min * sqrt(n_psi/n0) / omega_p0 with omega_p0 = 1/d0.
 *   - Newton: 4 fixed iterations from the explicit-Euler guess.
 *   - rest-frame photon direction before excitation: sign(mu_s - beta_s);
 *     de-excitation angle drawn from (3/8)(1 + cos^2).
 *   - the scattering draw: one Philox4x32-10 block per lepton and step;
 *     U = ((x0 >> 8) + 1) 2^-24 on (0, 1], the lepton scatters when
 *     U <= p_sc, and no draw is made for p_sc < 2^-24 (which the 24-bit
 *     uniform cannot resolve: such a lepton never scatters).
 *   - pair members each take half the photon momentum along s, placed at
 *     the parent's new position; none is made if that position left the line.
 *   - the pair cap compares the cell's lepton weight at the start of the
 *     step (integer fixed-point sums) against n_max.
 *   - surface supply (RATE): neutral e- + ion pairs injected per footpoint
 *     per step at the rate that carries j_ext, inward half-Maxwellian.
 *   - atmosphere (TOPUP, Sec. 3 and App. B.1 [densprofile]): a cell whose
 *     centre sits at radius x has the target density
 *     n/n0 = a0 exp(-(x - 1) R_star / h) (h in cells); the atmosphere is the
 *     set of cells where that is >= n_cut (gravity is off elsewhere, where
 *     n/n0 << 1).  After the move, a cell's plasma weight W (all species,
 *     integer fixed point, this step's pairs not included) is compared with
 *     the target weight floor(n/n0 n0_ppc 2^12); the deficit is filled with
 *     neutral e- + ion pairs of weight 1, uniform in the cell, Maxwellian at
 *     T in both directions.  Gravity: the force -T/h along r, i.e.
 *     -T/h mu_s along s, on every particle, kept at cell centres of the
 *     atmosphere (zero elsewhere) and gathered like E; du = (q/m E + g/m) dt.
 *   - annihilation at n_max (Sec. 3; Sec. 5 on the annihilation zone): every
 *     annihilate_every steps, at the end of the step, a cell whose lepton
 *     weight W (all leptons) exceeds n_max loses the same weight
 *     A = min((W - n_max)/2, W+, W-) of positrons and of pair electrons
 *     (integer fixed point).  Within each species, weight goes in increasing
 *     order of the key splitmix64(id ^ splitmix64(step ^ salt)) (a bijection
 *     of the id, so there are no ties); the last particle touched may keep
 *     part of its weight.  The removed charge is first carried to the cell's
 *     left node, which deposits the current (q delta (s - c)) through the
 *     cell; then the removed positive and negative weight, equal and at one
 *     point, vanish: the discrete Gauss law holds exactly.
 *
 * Parity unpinned (the paper leaves them open; pinned only by internal
 * identities): the de-excitation angular law, the pair-momentum split, the
 * choice of omega_p in tau_min, the b convention, the initial species split
 * and the photon model (stellar disk or radial).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* physical constants (CODATA 2018)                                          */
/* ------------------------------------------------------------------------ */
#define ORC_R_E      2.8179403262e-13   /* classical electron radius [cm]   */
#define ORC_LAMBDABAR 3.8615926796e-11  /* reduced Compton wavelength [cm]  */
#define ORC_ME_KEV   510.99895          /* m_e c^2 [keV]                    */
#define ORC_PI       3.14159265358979323846

/* enums shared by value with the Python side */
enum { ORC_PHOTON_RADIAL = 0, ORC_PHOTON_DISK = 1 };
enum { ORC_DRAG_OFF = 0, ORC_DRAG_CLOSED = 1, ORC_DRAG_TABLE = 2, ORC_DRAG_SURROGATE = 3 };
enum { ORC_RICS_SPLIT = 0, ORC_RICS_DRAG_PLUS_PAIRS = 1 };
enum { ORC_INJECT_NONE = 0, ORC_INJECT_RATE = 1, ORC_INJECT_TOPUP = 2 };
enum { ORC_SP_ELEC = 0, ORC_SP_POSI = 1, ORC_SP_ION = 2, ORC_SP_ATMO = 3 };

#define ORC_TAG_RICS 0x52494353u   /* counter word 3 of the scattering draw */
#define ORC_TAG_INJ  0x494E4A31u   /* counter word 3 of the injection draw  */
#define ORC_TAG_ATM  0x41544D4Fu   /* counter word 3 of the atmosphere draw */
#define ORC_TAG_INIT 0x494E4954u   /* counter word 3 of the initial load    */
#define ORC_S_BITS   12            /* weight fixed point: w_int = rint(w*2^12) */

typedef struct {
  double r_eq; int32_t n_cells; double cfl; double b_star; int32_t b_convention;
  double kT_keV; int32_t photon_model; int32_t drag_law; double drag_scale;
  int32_t table_n_gamma; int32_t table_n_s; double table_log10g_max;
  int32_t quad_n_mu; int32_t quad_n_phi;
  double eta_min; int32_t rics_mode; int32_t mc_on;
  double cells_per_skin_depth; double j_psi; double n0_ppc; double mass_ratio;
  int32_t ppc_e; int32_t ppc_p; int32_t ppc_i; double init_multiplicity; double u_sigma;
  int32_t inject_mode; double inject_T; double atmo_a0; double atmo_h; double atmo_ncut;
  int32_t pairs_on; double b_pair_threshold; double pair_energy_threshold; double n_max_ppc;
  int32_t annihilate_every;
  uint64_t seed; double r_star_cm;
} orc_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random        */
/* numbers: as easy as 1, 2, 3"): 10 rounds of a multiply-xor bijection on   */
/* a 128-bit counter under a 64-bit key bumped by Weyl constants.            */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24-bit uniform in [0,1): identical in FP32 and FP64 */
static double orc_u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
/* a uniform on (0, 1]: ((x >> 8) + 1) 2^-24 */
static double orc_u24_open(uint32_t x) { return (double)((x >> 8) + 1u) * (1.0 / 16777216.0); }
#define ORC_DRAW_MIN (1.0 / 16777216.0)

/* SplitMix64 finaliser (Steele, Lea, Flood 2014) -- used only to derive
 * stable identifiers for created particles. */
/* the generator on n counters (4 words each): out[4i..] = Philox4x32-10(ctr[4i..], key) */
void orc_philox4x32_10_n(const uint32_t* ctr, int64_t n, const uint32_t key_in[2], uint32_t* out)
{
  for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key_in, out + 4 * i);
}

uint64_t orc_splitmix64(uint64_t z)
{
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t orc_child_id(uint64_t parent, int64_t step, int member)
{
  return orc_splitmix64(parent ^ orc_splitmix64((uint64_t)step * 2u + (uint64_t)member))
         | 0x8000000000000000ull;
}

uint64_t orc_inject_id(int64_t step, int foot, int64_t slot, int member)
{
  uint64_t key = ((uint64_t)step << 24) ^ ((uint64_t)foot << 23) ^ ((uint64_t)slot << 1) ^ (uint64_t)member;
  return orc_splitmix64(key ^ 0x5A17A5EEDull) | 0x8000000000000000ull;
}

/* atmosphere particle `slot` (member 0: e-, 1: ion) of cell `cell` at `step` */
uint64_t orc_atmo_id(int64_t step, int cell, int64_t slot, int member)
{
  uint64_t a = orc_splitmix64(((uint64_t)step << 1) | (uint64_t)member);
  uint64_t b = ((uint64_t)(uint32_t)cell << 32) | (uint64_t)(uint32_t)slot;
  return orc_splitmix64(a ^ b ^ 0xA7305EEDull) | 0x8000000000000000ull;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1,1] (Newton on the three-term recurrence).     */
/* ------------------------------------------------------------------------ */
void orc_gauss_legendre(int n, double* x, double* w)
{
  for (int i = 0; i < n; ++i) {
    double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2; p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2; p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
    }
    x[i] = -z;                                   /* ascending order */
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

/* ------------------------------------------------------------------------ */
/* Dipole field-line geometry (App. B.2).  The line r = r_eq sin^2(theta)     */
/* runs from the northern footpoint theta_0 = arcsin(sqrt(R_star/r_eq)) to the    */
/* southern one pi - theta_0.  Arc length (in R_star):                           */
/*   ds/dtheta = r_eq sin(theta) sqrt(1 + 3 cos^2 theta).                    */
/* s(theta) is the integral written out with composite Gauss-Legendre.       */
/* ------------------------------------------------------------------------ */
static double orc_dsdtheta(double r_eq, double th)
{
  double c = cos(th);
  return r_eq * sin(th) * sqrt(1.0 + 3.0 * c * c);
}

double orc_theta0(double r_eq) { return asin(sqrt(1.0 / r_eq)); }

double orc_arc_length(double r_eq, double theta)
{
  static int init = 0;
  static double gx[16], gw[16];
  if (!init) { orc_gauss_legendre(16, gx, gw); init = 1; }
  double a = orc_theta0(r_eq), b = theta;
  const int panels = 8;
  double h = (b - a) / panels, sum = 0.0;
  for (int k = 0; k < panels; ++k) {
    double lo = a + k * h;
    for (int i = 0; i < 16; ++i) {
      double th = lo + 0.5 * h * (gx[i] + 1.0);
      sum += 0.5 * h * gw[i] * orc_dsdtheta(r_eq, th);
    }
  }
  return sum;
}

double orc_line_length(double r_eq) { return orc_arc_length(r_eq, ORC_PI - orc_theta0(r_eq)); }

/* invert s(theta) = s_target (s in R_star): Newton from the linear guess,
 * kept inside a shrinking bracket (bisection when Newton leaves it) */
double orc_theta_of_s(double r_eq, double s_target)
{
  double t0 = orc_theta0(r_eq), t1 = ORC_PI - t0;
  double L = orc_line_length(r_eq);
  double lo = t0, hi = t1;
  double th = t0 + (t1 - t0) * s_target / L;
  for (int it = 0; it < 100; ++it) {
    double f = orc_arc_length(r_eq, th) - s_target;
    if (f > 0.0) hi = th; else lo = th;
    double d = orc_dsdtheta(r_eq, th);
    double nt = (d > 0.0) ? th - f / d : 0.5 * (lo + hi);
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    if (fabs(nt - th) < 1e-15) { th = nt; break; }
    th = nt;
  }
  if (th < t0) th = t0;
  if (th > t1) th = t1;
  return th;
}

/* x = r/R_star, b = B/B_QED, mu_s = B^r/B (cosine between the outward radial
 * direction and +s, the direction of increasing theta). */
void orc_field_at_theta(const orc_params* p, double th, double* x, double* b, double* mu)
{
  double c = cos(th), s = sin(th);
  double xr = p->r_eq * s * s;
  double root = sqrt(1.0 + 3.0 * c * c);
  double bb = p->b_star * root / (xr * xr * xr);
  if (p->b_convention == 1) bb *= 0.5;
  *x = xr; *b = bb; *mu = 2.0 * c / root;
}

/* ------------------------------------------------------------------------ */
/* RICS physics (Sec. 2.2).  Momentum u = gamma*beta_s along +s.              */
/* Theta = kT/(m_e c^2).  Resonant photon energy in units of m_e c^2:          */
/*   eps = b / (gamma (1 - beta_s mu_k))                       [resomega]    */
/* Rate per lepton (per R_star/c, i.e. N^ = Ndot R_star/c)            [scatteringNdot] */
/*   N^ = r_e R_star/(4 pi lbar^2 gamma) Int dOmega eps^2/(exp(eps/Theta) - 1)   */
/* Momentum given per scattering along s: gamma b mu~_k, mu~ = (mu_k - beta)/ */
/* (1 - beta mu_k); the drag F^ = F R_star/(m_e c^2) is the rate-weighted sum.    */
/* For radially streaming photons (solid angle pi/x^2, mu_k = mu_s) the sum   */
/* is the closed form                                           [contdrag]   */
/*   F^ = r_e R_star Theta^3/(4 x^2 lbar^2) gamma (mu_s - beta_s) g(y),          */
/*   g(y) = y^3/(e^y - 1), y = eps/Theta.                                    */
/* ------------------------------------------------------------------------ */
double orc_g(double y) { return y * y * y / expm1(y); }

static double orc_theta_T(const orc_params* p) { return p->kT_keV / ORC_ME_KEV; }

/* 1 - beta_s*m computed without cancellation when beta -> 1 */
static double orc_one_minus_beta_m(double u, double gam, double m)
{
  double beta = fabs(u) / gam;
  double sm = (u >= 0.0) ? m : -m;              /* cosine to the velocity */
  double omb = 1.0 / (gam * (gam + fabs(u)));   /* 1 - |beta| */
  (void)beta;
  return (1.0 - sm) + sm * omb;
}

void orc_radial(const orc_params* p, double u, double x, double b, double mu,
                double* F, double* Nhat)
{
  double th = orc_theta_T(p);
  double gam = sqrt(1.0 + u * u);
  double beta = u / gam;
  double D = orc_one_minus_beta_m(u, gam, mu);
  double eps = b / (gam * D);
  double y = eps / th;
  double pref = ORC_R_E * p->r_star_cm / (ORC_LAMBDABAR * ORC_LAMBDABAR);
  *F = pref * th * th * th / (4.0 * x * x) * gam * (mu - beta) * orc_g(y);
  *Nhat = pref / (4.0 * x * x * gam) * eps * eps / expm1(y);
}

/* Stellar disk of uniform blackbody intensity: directions within alpha_max
 * = arcsin(1/x) of the radial; mu_k = cos(a) mu_s + sin(a) cos(phi) sqrt(1-mu_s^2).
 * Gauss-Legendre in cos(a) x midpoint rule in phi on [0, pi] (the integrand
 * is even in phi). */
/* The three rate-weighted sums over the disk: sum dN, sum dN * (momentum per
 * scattering), sum dN * |momentum per scattering| (the last one is the scale
 * of the surrogate's error metric), in units of the prefactor below. */
static void orc_disk_sums(const orc_params* p, double u, double x, double b, double mu,
                          double* sN, double* sF, double* sFa)
{
  int na = p->quad_n_mu, nph = p->quad_n_phi;
  double gx[256], gw[256];
  if (na > 256) na = 256;
  orc_gauss_legendre(na, gx, gw);
  double th = orc_theta_T(p);
  double gam = sqrt(1.0 + u * u);
  double beta = u / gam;
  double cmax = (x > 1.0) ? sqrt(1.0 - 1.0 / (x * x)) : 0.0;   /* cos(alpha_max) */
  double smu = sqrt(fmax(0.0, 1.0 - mu * mu));
  double sumN = 0.0, sumF = 0.0, sumFa = 0.0;
  for (int i = 0; i < na; ++i) {
    double ca = cmax + (1.0 - cmax) * 0.5 * (gx[i] + 1.0);
    double wa = (1.0 - cmax) * 0.5 * gw[i];
    double sa = sqrt(fmax(0.0, 1.0 - ca * ca));
    for (int j = 0; j < nph; ++j) {
      double ph = ORC_PI * (j + 0.5) / nph;
      double wph = 2.0 * ORC_PI / nph;           /* 2 * (pi/nph) */
      double mk = ca * mu + sa * cos(ph) * smu;
      double D = orc_one_minus_beta_m(u, gam, mk);
      double eps = b / (gam * D);
      double y = eps / th;
      double occ = eps * eps / expm1(y);         /* eps^2/(e^y - 1) */
      double dN = wa * wph * occ;
      double dNP = dN * gam * b * (mk - beta) / D;   /* dN x momentum per scattering */
      sumN += dN;
      sumF += dNP;
      sumFa += fabs(dNP);
    }
  }
  *sN = sumN; *sF = sumF; *sFa = sumFa;
}

void orc_disk(const orc_params* p, double u, double x, double b, double mu,
              double* F, double* Nhat)
{
  double sumN, sumF, sumFa;
  orc_disk_sums(p, u, x, b, mu, &sumN, &sumF, &sumFa);
  double gam = sqrt(1.0 + u * u);
  double pref = ORC_R_E * p->r_star_cm / (4.0 * ORC_PI * ORC_LAMBDABAR * ORC_LAMBDABAR * gam);
  *Nhat = pref * sumN;
  *F = pref * sumF;
}

void orc_photon_field(const orc_params* p, double u, double x, double b, double mu,
                      double* F, double* Nhat)
{
  if (p->photon_model == ORC_PHOTON_DISK) orc_disk(p, u, x, b, mu, F, Nhat);
  else orc_radial(p, u, x, b, mu, F, Nhat);
}

/* ------------------------------------------------------------------------ */
/* Drag/rate table: axes log10(gamma) in [0, G] (n_g points), s/L in [0,1]    */
/* (n_s points), sign of u; entries F^ and ln N^ (floored at -700).           */
/* layout: ((sign * n_s + js) * n_g + ig) * 2 + {0: F^, 1: ln N^}             */
/* ------------------------------------------------------------------------ */
void orc_build_table(const orc_params* p, double* table)
{
  int ng = p->table_n_gamma, ns = p->table_n_s;
  double L = orc_line_length(p->r_eq);
  for (int js = 0; js < ns; ++js) {
    double sR = L * (double)js / (ns - 1);
    double th = orc_theta_of_s(p->r_eq, sR);
    double x, b, mu;
    orc_field_at_theta(p, th, &x, &b, &mu);
    for (int sg = 0; sg < 2; ++sg) {
      for (int ig = 0; ig < ng; ++ig) {
        double lg = p->table_log10g_max * (double)ig / (ng - 1);
        double gam = pow(10.0, lg);
        double au = sqrt(fmax(0.0, gam * gam - 1.0));
        double u = sg ? -au : au;
        double F, N;
        orc_photon_field(p, u, x, b, mu, &F, &N);
        double lnN = (N > 0.0) ? log(N) : -700.0;
        if (lnN < -700.0) lnN = -700.0;
        size_t k = (((size_t)sg * ns + js) * ng + ig) * 2;
        table[k] = F;
        table[k + 1] = lnN;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Learned surrogate of the photon-field quadrature: one training sample.    */
/*                                                                           */
/* Per photon direction the momentum given per scattering is gamma b mu~,    */
/* mu~ = (mu_k - beta)/(1 - beta mu_k) (Sec. 2.2), so the drag is            */
/*   F^ = gamma b N^ <mu~>,                                                  */
/* <mu~> the rate-weighted mean of mu~ over the photon directions, which     */
/* lies in [-1, 1].  The network learns                                      */
/*   t1 = <mu~>                                                              */
/*   t2 = max(ln N^, LT) - max(B, LT)                                        */
/* with the baseline B = ln(0.9 N^_rad(mu_s) + 0.1 N^_rad(mu_e)): N^_rad is  */
/* the closed form for photons streaming along one direction [contdrag] and  */
/* mu_e the edge of the stellar disk most favourable to the resonance (the   */
/* largest 1 - beta mu_k), whose Wien factor dominates the rate near the     */
/* star.  Two floors: rates below LE = -20 are negligible (less than one     */
/* scattering per 1e12 particle-steps; the drag then moves u by less than    */
/* FP32 rounding), and the surrogate is scored only above LE; the targets   */
/* are clamped at LT = -30, ten e-folds lower, so that the kink of the clamp */
/* lies outside the scored region.  t1 is masked (weight 0) where ln N^ <=   */
/* LT.                                                                       */
/* Inputs, each in [-1, 1] over the training box:                            */
/*   f0 = 2 log10(gamma)/G - 1, f1 = 2 s/L - 1,                              */
/*   f2 = (log10 b - B_MID)/B_HALF, f3 = sign(u).                            */
/* ------------------------------------------------------------------------ */
#define ORC_TAG_SUR    0x53555247u   /* counter word 3 of a sample draw */
#define ORC_SUR_LT     (-30.0)   /* clamp of the targets */
#define ORC_SUR_B_MID  (-1.25)
#define ORC_SUR_B_HALF 2.75

/* cosine of the disk edge direction with the largest 1 - beta mu_k */
double orc_sur_edge_mu(double u, double x, double mu)
{
  double ths = acos(fmax(-1.0, fmin(1.0, mu)));
  double am = asin(fmin(1.0, 1.0 / x));
  return (u >= 0.0) ? cos(fmin(ORC_PI, ths + am)) : cos(fmax(0.0, ths - am));
}

/* the rate baseline B of the surrogate (see above) */
double orc_sur_baseline(const orc_params* q, double u, double x, double b, double mu)
{
  double Fr, Nr, Fe, Ne;
  orc_radial(q, u, x, b, mu, &Fr, &Nr);
  orc_radial(q, u, x, b, orc_sur_edge_mu(u, x, mu), &Fe, &Ne);
  double N = 0.9 * Nr + 0.1 * Ne;
  return (N > 0.0) ? log(N) : -745.0;
}

/* out[15]: f0 f1 f2 f3 | t1 t2 mask | lnN B F^ F^_abs | b x mu u */
void orc_sur_point(const orc_params* p, double r_eq, double s_frac, double log10g, int neg, double* out)
{
  orc_params q = *p;
  q.r_eq = r_eq;
  double L = orc_line_length(r_eq);
  double th = orc_theta_of_s(r_eq, s_frac * L);
  double x, b, mu;
  orc_field_at_theta(&q, th, &x, &b, &mu);
  double gam = pow(10.0, log10g);
  double au = sqrt(fmax(0.0, gam * gam - 1.0));
  double u = neg ? -au : au;
  gam = sqrt(1.0 + u * u);
  double beta = u / gam;
  double F, N, Fa, mubar;
  if (p->photon_model == ORC_PHOTON_DISK) {
    double sN, sF, sFa;
    orc_disk_sums(&q, u, x, b, mu, &sN, &sF, &sFa);
    double pref = ORC_R_E * p->r_star_cm / (4.0 * ORC_PI * ORC_LAMBDABAR * ORC_LAMBDABAR * gam);
    N = pref * sN; F = pref * sF; Fa = pref * sFa;
    mubar = (sN > 0.0) ? sF / (gam * b * sN) : (mu - beta) / orc_one_minus_beta_m(u, gam, mu);
  } else {
    orc_radial(&q, u, x, b, mu, &F, &N);
    Fa = fabs(F);
    mubar = (mu - beta) / orc_one_minus_beta_m(u, gam, mu);
  }
  double lnN = (N > 0.0) ? log(N) : -745.0;
  double lnNr = orc_sur_baseline(&q, u, x, b, mu);
  out[0] = 2.0 * log10g / p->table_log10g_max - 1.0;
  out[1] = 2.0 * s_frac - 1.0;
  out[2] = (log10(b) - ORC_SUR_B_MID) / ORC_SUR_B_HALF;
  out[3] = neg ? -1.0 : 1.0;
  out[4] = mubar;
  out[5] = fmax(lnN, ORC_SUR_LT) - fmax(lnNr, ORC_SUR_LT);
  out[6] = (lnN > ORC_SUR_LT) ? 1.0 : 0.0;
  out[7] = lnN; out[8] = lnNr; out[9] = F; out[10] = Fa;
  out[11] = b; out[12] = x; out[13] = mu; out[14] = u;
}

/* Sample `index` of a training set: one Philox4x32-10 draw with counter
 * (index_lo, index_hi, 0, TAG_SUR) and key = seed gives log10 gamma uniform in
 * [0, G] (log-uniform gamma), s/L uniform in [0, 1), the sign of u from the
 * top bit of the third word, and r_eq log-uniform in [r_lo, r_hi]. */
void orc_sur_sample(const orc_params* p, uint64_t seed, uint64_t index, double r_lo, double r_hi, double* out)
{
  uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), 0u, ORC_TAG_SUR};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  double log10g = p->table_log10g_max * orc_u24(r[0]);
  double s_frac = orc_u24(r[1]);
  int neg = (int)(r[2] >> 31);
  double r_eq = (r_hi > r_lo) ? r_lo * pow(r_hi / r_lo, orc_u24(r[3])) : r_lo;
  orc_sur_point(p, r_eq, s_frac, log10g, neg, out);
}

/* n consecutive samples from index `start` (out: n x 15, row-major) */
void orc_sur_samples(const orc_params* p, uint64_t seed, uint64_t start, int64_t n, double r_lo, double r_hi,
                     double* out)
{
  for (int64_t i = 0; i < n; ++i) orc_sur_sample(p, seed, start + (uint64_t)i, r_lo, r_hi, out + 15 * i);
}

/* ------------------------------------------------------------------------ */
/* Test-particle drag maps (App. on the extent of the pair-producing region): */
/* a lepton enters a field line at the northern footpoint with gamma0 and    */
/* moves under the drag alone (radially streaming photons, Eq. contdrag).    */
/* The line is followed in theta (ds = r_eq sin(theta) sqrt(1+3cos^2) dtheta, */
/* time in R_star/c).  One step of dt:                                       */
/*   u1 from u1 - u0 - dt/2 (F(u0) + F(u1)) = 0 at fixed theta (Newton on the */
/*      exact derivative of the closed form),                                 */
/*   tau += dt/2 (N(u0) + N(u1))    (expected scatterings, N^ = Ndot R_star / c), */
/*   theta += dt/2 (beta0 + beta1) / (ds/dtheta at theta0).                  */
/* It stops at the equator (theta = pi/2; the line is symmetric) or at      */
/* t_max.  Reported: gamma_min over the path; the first scattering where tau */
/* reaches 1 (linear in the step); the point where b falls below b_thr.      */
/* out[12]: gamma_min, theta_first (-1: none), theta_b, s_first, s_b, L,     */
/*          l_pp, region (1, 2, 3), b_eq, steps, t_end, u_end                */
/* ------------------------------------------------------------------------ */
static void orc_tp_drag(const orc_params* p, double u, double x, double b, double mu, double* F, double* dF,
                        double* N)
{
  double Fh, Nh;
  orc_radial(p, u, x, b, mu, &Fh, &Nh);
  double th = orc_theta_T(p);
  double gam = sqrt(1.0 + u * u), beta = u / gam;
  double D = gam * orc_one_minus_beta_m(u, gam, mu);
  double y = b / (th * D);
  double g = orc_g(y);
  double K = ORC_R_E * p->r_star_cm / (ORC_LAMBDABAR * ORC_LAMBDABAR) * th * th * th / (4.0 * x * x);
  double gp = g * (3.0 / y - 1.0 / (-expm1(-y)));
  double dydu = -y * (beta - mu) / D;
  *F = p->drag_scale * Fh;
  *dF = p->drag_scale * K * ((beta * mu - 1.0) * g + gam * (mu - beta) * gp * dydu);
  *N = p->drag_scale * Nh;
}

void orc_tp_line(const orc_params* p0, double r_eq, double gamma0, double dt, double t_max, double b_thr,
                 double gamma_eps, double* out)
{
  orc_params q = *p0;
  q.r_eq = r_eq;
  const orc_params* p = &q;
  double th = orc_theta0(r_eq);
  double u = sqrt(gamma0 * gamma0 - 1.0);
  double gmin = gamma0, tau = 0.0, t = 0.0, th_first = -1.0;
  long steps = 0;
  while (th < 0.5 * ORC_PI && t < t_max) {
    double x, b, mu;
    orc_field_at_theta(p, th, &x, &b, &mu);
    double F0, dF0, N0;
    orc_tp_drag(p, u, x, b, mu, &F0, &dF0, &N0);
    double u1 = u + dt * F0;
    for (int it = 0; it < 50; ++it) {
      double F1, dF1, N1;
      orc_tp_drag(p, u1, x, b, mu, &F1, &dF1, &N1);
      double G = u1 - u - 0.5 * dt * (F0 + F1);
      double dG = 1.0 - 0.5 * dt * dF1;
      if (dG < 0.5) dG = 0.5;
      double un = u1 - G / dG;
      int done = fabs(un - u1) <= 1e-14 * (1.0 + fabs(un));
      u1 = un;
      if (done) break;
    }
    double F1, dF1, N1;
    orc_tp_drag(p, u1, x, b, mu, &F1, &dF1, &N1);
    double tau1 = tau + 0.5 * dt * (N0 + N1);
    double beta0 = u / sqrt(1.0 + u * u), beta1 = u1 / sqrt(1.0 + u1 * u1);
    double c = cos(th);
    double h = r_eq * sin(th) * sqrt(1.0 + 3.0 * c * c);
    double th1 = th + 0.5 * dt * (beta0 + beta1) / h;
    if (th_first < 0.0 && tau < 1.0 && tau1 >= 1.0) th_first = th + (1.0 - tau) / (tau1 - tau) * (th1 - th);
    u = u1;
    tau = tau1;
    th = th1;
    t += dt;
    ++steps;
    double g1 = sqrt(1.0 + u * u);
    if (g1 < gmin) gmin = g1;
  }
  /* where b falls below b_thr (b decreases from the footpoint to the equator) */
  double xe, be, me;
  orc_field_at_theta(p, 0.5 * ORC_PI, &xe, &be, &me);
  double th_b = 0.5 * ORC_PI;
  if (be < b_thr) {
    double lo = orc_theta0(r_eq), hi = 0.5 * ORC_PI;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi), xm, bm, mm;
      orc_field_at_theta(p, mid, &xm, &bm, &mm);
      if (bm >= b_thr) lo = mid; else hi = mid;
    }
    th_b = 0.5 * (lo + hi);
  }
  double L = orc_line_length(r_eq);
  double s_first = (th_first >= 0.0) ? orc_arc_length(r_eq, th_first) : -1.0;
  double s_b = orc_arc_length(r_eq, th_b);
  double lpp = 0.0;
  if (s_first >= 0.0) {
    if (be >= b_thr) lpp = L - 2.0 * s_first;           /* across the equator, symmetric */
    else lpp = (s_b > s_first) ? s_b - s_first : 0.0;
  }
  int region = (gmin <= 1.0 + gamma_eps) ? 3 : ((be >= b_thr) ? 1 : 2);
  out[0] = gmin; out[1] = th_first; out[2] = th_b; out[3] = s_first; out[4] = s_b; out[5] = L;
  out[6] = lpp; out[7] = region; out[8] = be; out[9] = (double)steps; out[10] = t; out[11] = u;
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n_alive[4];
  int64_t pairs_created, pairs_dropped_cap, pairs_rejected_nmax, pairs_lost_wall;
  int64_t lost_north, lost_south, injected, scatters, psc_clamped, limiter_branch, newton_branch;
  int64_t annihilated;            /* weight removed by annihilation, units of 2^-12 */
  double field_energy, kinetic_energy, ext_work, vc, charge, ke_lost;
} orc_diag;

typedef struct {
  orc_params p;
  int N;
  double L_R;       /* line length in R_star                                  */
  double R_cells;   /* R_star in cells                                        */
  double dt;        /* time step in cell-crossing times                   */
  double q_p;       /* macro charge per unit weight                       */
  double j_ext;     /* external (twist) current density                   */
  double tau_min;   /* drag-time floor [code time]                        */
  double *node_x, *node_b, *node_mu;   /* N+1 nodes                       */
  unsigned char* zone;                 /* N cells: b(centre) > b_thr      */
  int64_t* atmo_target;                /* N cells: TOPUP target weight (w_int), -1 outside */
  double* grav;                        /* N cell centres: gravity along s (per unit mass) */
  int grav_on;
  double* table;
  double* sur;                         /* surrogate parameters (8770) or NULL */
  double *E, *J;
  int64_t* dens;                       /* lepton weight per cell, w_int   */
  int64_t n, cap;
  double *s, *u, *w;
  int32_t* sp;
  uint64_t* id;
  int64_t step;
  double inj_acc[2];
  orc_diag d;
} orc_sim;

static const double ORC_QM[4]   = { -1.0, 1.0, 0.0 /* set per sim */, -1.0 };
static const double ORC_QS[4]   = { -1.0, 1.0, 1.0, -1.0 };   /* charge sign */

static int orc_is_lepton(int sp) { return sp != ORC_SP_ION; }
static double orc_mass(const orc_sim* S, int sp) { return sp == ORC_SP_ION ? S->p.mass_ratio : 1.0; }
static double orc_qm(const orc_sim* S, int sp) { return sp == ORC_SP_ION ? 1.0 / S->p.mass_ratio : ORC_QM[sp]; }

static int64_t orc_wint(double w) { return (int64_t)llrint(w * (double)(1 << ORC_S_BITS)); }

size_t orc_sim_size(void) { return sizeof(orc_sim); }

static void orc_grow(orc_sim* S, int64_t need)
{
  if (need <= S->cap) return;
  int64_t cap = S->cap ? S->cap : 1024;
  while (cap < need) cap *= 2;
  S->s = realloc(S->s, cap * sizeof(double));
  S->u = realloc(S->u, cap * sizeof(double));
  S->w = realloc(S->w, cap * sizeof(double));
  S->sp = realloc(S->sp, cap * sizeof(int32_t));
  S->id = realloc(S->id, cap * sizeof(uint64_t));
  S->cap = cap;
}

/* linear interpolation of a node table at s (cells) */
static double orc_node_interp(const orc_sim* S, const double* tab, double s)
{
  if (s <= 0.0) return tab[0];
  if (s >= S->N) return tab[S->N];
  int i = (int)floor(s);
  if (i >= S->N) i = S->N - 1;
  double f = s - i;
  return (1.0 - f) * tab[i] + f * tab[i + 1];
}

static void orc_recount_density(orc_sim* S);

/* The initial plasma of Sec. 3: a pair plasma of multiplicity M whose
 * leptons drift at beta = -+1/M (the carriers of the twist current), with
 * ions, by the recipe the parameters document.  Electron k of cell c sits at
 * the fixed-point position c 2^F + floor((k 2^24 + (X >> 8)) 2^F / (ppc_e
 * 2^24)), X word 0 of Philox(c, k, 0, INIT): uniform inside the k-th of
 * ppc_e equal parts of the cell.  Positrons take the positions of the cell's
 * first ppc_p electrons and ions those of the next ppc_i, so that every node
 * is neutral.  Momenta are u = drift + sigma g with g = sqrt(-2 ln U1)
 * cos(2 pi U2) (Box-Muller), U1 = ((Y >> 8) + 1) 2^-24, U2 = (Z >> 8) 2^-24
 * from words 1 and 2 of Philox(c, k, m, INIT), m = 0, 1, 2 for e-, e+, ion;
 * drift -u_d, +u_d, 0 with u_d = beta_d / sqrt(1 - beta_d^2), beta_d = 1/M. */
static void orc_initial_load(orc_sim* S)
{
  const orc_params* p = &S->p;
  int N = S->N;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  int F = 32 - lg;
  int64_t ne = (int64_t)N * p->ppc_e, np = (int64_t)N * p->ppc_p, ni = (int64_t)N * p->ppc_i;
  int64_t n = ne + np + ni;
  orc_grow(S, n);
  double beta_d = 1.0 / p->init_multiplicity;
  double u_d = beta_d / sqrt(1.0 - beta_d * beta_d);
  uint32_t key[2] = { (uint32_t)p->seed, (uint32_t)(p->seed >> 32) };
  for (int c = 0; c < N; ++c) {
    for (int k = 0; k < p->ppc_e; ++k) {
      uint32_t r[4], ctr[4] = { (uint32_t)c, (uint32_t)k, 0u, ORC_TAG_INIT };
      orc_philox4x32_10(ctr, key, r);
      uint64_t A = ((uint64_t)k << 24) + (uint64_t)(r[0] >> 8);
      uint64_t frac = F >= 24 ? (A << (F - 24)) / (uint64_t)p->ppc_e : A / ((uint64_t)p->ppc_e << (24 - F));
      double s = (double)(((uint64_t)c << F) + frac) / (double)((uint64_t)1 << F);
      for (int m = 0; m < 3; ++m) {
        int64_t slot;
        if (m == 0) slot = (int64_t)c * p->ppc_e + k;
        else if (m == 1 && k < p->ppc_p) slot = ne + (int64_t)c * p->ppc_p + k;
        else if (m == 2 && k >= p->ppc_p) slot = ne + np + (int64_t)c * p->ppc_i + (k - p->ppc_p);
        else continue;
        uint32_t q[4];
        if (m == 0) { q[1] = r[1]; q[2] = r[2]; }
        else {
          uint32_t cm[4] = { (uint32_t)c, (uint32_t)k, (uint32_t)m, ORC_TAG_INIT };
          orc_philox4x32_10(cm, key, q);
        }
        double U1 = (double)((q[1] >> 8) + 1u) * (1.0 / 16777216.0);
        double U2 = (double)(q[2] >> 8) * (1.0 / 16777216.0);
        double g = sqrt(-2.0 * log(U1)) * cos(2.0 * ORC_PI * U2);
        double drift = m == 0 ? -u_d : (m == 1 ? u_d : 0.0);
        S->s[slot] = s;
        S->u[slot] = drift + p->u_sigma * g;
        S->w[slot] = 1.0;
        S->sp[slot] = m == 0 ? ORC_SP_ELEC : (m == 1 ? ORC_SP_POSI : ORC_SP_ION);
        S->id[slot] = (uint64_t)slot;
      }
    }
  }
  S->n = n;
  orc_recount_density(S);
}

orc_sim* orc_create(const orc_params* p, const double* table_or_null)
{
  orc_sim* S = (orc_sim*)calloc(1, sizeof(orc_sim));
  S->p = *p;
  S->N = p->n_cells;
  S->L_R = orc_line_length(p->r_eq);
  S->R_cells = S->N / S->L_R;
  S->dt = p->cfl;
  /* omega_p0 = 1/d0 at density n0 (weight n0_ppc per cell): 4 pi q_p n0 =
   * omega_p0^2 with q/m = 1.  j_ext = j_psi n0 e c (Sec. 3: j_psi/(n0 e c)). */
  double n0 = p->n0_ppc;
  S->q_p = 1.0 / (4.0 * ORC_PI * p->cells_per_skin_depth * p->cells_per_skin_depth * n0);
  S->j_ext = p->j_psi * n0 * S->q_p;
  /* eta_min = tau_min omega_p0 = eta_min_param (n_psi/n0)^(1/2), n_psi/n0 = j_psi */
  S->tau_min = (p->eta_min > 0.0 && p->j_psi > 0.0) ? p->eta_min * sqrt(p->j_psi) * p->cells_per_skin_depth : 0.0;
  int N = S->N;
  S->node_x = malloc((N + 1) * sizeof(double));
  S->node_b = malloc((N + 1) * sizeof(double));
  S->node_mu = malloc((N + 1) * sizeof(double));
  for (int k = 0; k <= N; ++k) {
    double th = orc_theta_of_s(p->r_eq, S->L_R * (double)k / N);
    orc_field_at_theta(p, th, &S->node_x[k], &S->node_b[k], &S->node_mu[k]);
  }
  S->zone = malloc(N);
  S->atmo_target = malloc(N * sizeof(int64_t));
  S->grav = malloc(N * sizeof(double));
  for (int c = 0; c < N; ++c) {
    double th = orc_theta_of_s(p->r_eq, S->L_R * (c + 0.5) / N);
    double x, b, mu;
    orc_field_at_theta(p, th, &x, &b, &mu);
    S->zone[c] = (b > p->b_pair_threshold) ? 1 : 0;
    S->atmo_target[c] = -1;
    S->grav[c] = 0.0;
    if (p->inject_mode == ORC_INJECT_TOPUP) {
      /* [densprofile]: n/n0 = a0 exp(-(r - R_star)/h), r - R_star in cells */
      double n = p->atmo_a0 * exp(-(x - 1.0) * S->R_cells / p->atmo_h);
      if (n >= p->atmo_ncut) {
        S->atmo_target[c] = (int64_t)floor(n * p->n0_ppc * (double)(1 << ORC_S_BITS));
        /* hydrostatic: T dn/dr = n g, g = -T/h along r; along s: g mu_s */
        S->grav[c] = -(p->inject_T / p->atmo_h) * mu;
      }
    }
  }
  S->grav_on = (p->inject_mode == ORC_INJECT_TOPUP);
  /* the table law's table; a SURROGATE line given one keeps it as the
   * network's fallback outside its training box (else it is built on first use) */
  if (p->drag_law == ORC_DRAG_TABLE || (p->drag_law == ORC_DRAG_SURROGATE && table_or_null)) {
    size_t nt = (size_t)2 * p->table_n_s * p->table_n_gamma * 2;
    S->table = malloc(nt * sizeof(double));
    if (table_or_null) memcpy(S->table, table_or_null, nt * sizeof(double));
    else orc_build_table(p, S->table);
  }
  S->E = calloc(N, sizeof(double));
  S->J = calloc(N, sizeof(double));
  S->dens = calloc(N, sizeof(int64_t));
  if (p->ppc_e > 0) orc_initial_load(S);
  return S;
}

void orc_free(orc_sim* S)
{
  if (!S) return;
  free(S->node_x); free(S->node_b); free(S->node_mu); free(S->zone); free(S->table);
  free(S->atmo_target); free(S->grav);
  free(S->E); free(S->J); free(S->dens); free(S->sur);
  free(S->s); free(S->u); free(S->w); free(S->sp); free(S->id);
  free(S);
}

static void orc_recount_density(orc_sim* S)
{
  memset(S->dens, 0, S->N * sizeof(int64_t));
  for (int64_t k = 0; k < S->n; ++k) {
    if (!orc_is_lepton(S->sp[k])) continue;
    int c = (int)floor(S->s[k]);
    if (c < 0) c = 0;
    if (c >= S->N) c = S->N - 1;
    S->dens[c] += orc_wint(S->w[k]);
  }
}

void orc_set_particles(orc_sim* S, int64_t n, const double* s, const double* u,
                       const double* w, const int32_t* sp, const uint64_t* id)
{
  orc_grow(S, n);
  S->n = n;
  memcpy(S->s, s, n * sizeof(double));
  memcpy(S->u, u, n * sizeof(double));
  memcpy(S->w, w, n * sizeof(double));
  memcpy(S->sp, sp, n * sizeof(int32_t));
  memcpy(S->id, id, n * sizeof(uint64_t));
  orc_recount_density(S);
}

void orc_set_field(orc_sim* S, const double* E) { memcpy(S->E, E, S->N * sizeof(double)); }
void orc_set_step(orc_sim* S, int64_t step) { S->step = step; }
int64_t orc_get_n(const orc_sim* S) { return S->n; }

void orc_get_particles(const orc_sim* S, double* s, double* u, double* w, int32_t* sp, uint64_t* id)
{
  memcpy(s, S->s, S->n * sizeof(double));
  memcpy(u, S->u, S->n * sizeof(double));
  memcpy(w, S->w, S->n * sizeof(double));
  memcpy(sp, S->sp, S->n * sizeof(int32_t));
  memcpy(id, S->id, S->n * sizeof(uint64_t));
}

void orc_get_fields(const orc_sim* S, double* E, double* J)
{
  if (E) memcpy(E, S->E, S->N * sizeof(double));
  if (J) memcpy(J, S->J, S->N * sizeof(double));
}

void orc_get_nodes(const orc_sim* S, double* x, double* b, double* mu, unsigned char* zone)
{
  if (x) memcpy(x, S->node_x, (S->N + 1) * sizeof(double));
  if (b) memcpy(b, S->node_b, (S->N + 1) * sizeof(double));
  if (mu) memcpy(mu, S->node_mu, (S->N + 1) * sizeof(double));
  if (zone) memcpy(zone, S->zone, S->N);
}

void orc_get_scalars(const orc_sim* S, double* out)
{
  out[0] = S->L_R; out[1] = S->R_cells; out[2] = S->dt; out[3] = S->q_p;
  out[4] = S->j_ext; out[5] = S->tau_min; out[6] = S->inj_acc[0]; out[7] = S->inj_acc[1];
}

void orc_get_density(const orc_sim* S, int64_t* dens) { memcpy(dens, S->dens, S->N * sizeof(int64_t)); }

/* ------------------------------------------------------------------------ */
/* Drag and rate at (u, s) in code units: du/dt = drag_scale F^ / R_cells,    */
/* p_sc rate = drag_scale N^ / R_cells per cell-crossing time.               */
/* dF is dF/du of the same interpolant (Newton derivative).                  */
/* ------------------------------------------------------------------------ */
static void orc_table_eval(const orc_sim* S, double u, double s, double* F, double* dF, double* lnN)
{
  const orc_params* p = &S->p;
  int ng = p->table_n_gamma, ns = p->table_n_s;
  double gam = sqrt(1.0 + u * u);
  double dg = p->table_log10g_max / (ng - 1);
  double t = log10(gam) / dg;
  int clamped = 0;
  if (t < 0.0) t = 0.0;
  if (t > ng - 1) { t = ng - 1; clamped = 1; }
  int i = (int)floor(t);
  if (i > ng - 2) i = ng - 2;
  double a = t - i;
  double v = s / S->N * (ns - 1);
  if (v < 0.0) v = 0.0;
  if (v > ns - 1) v = ns - 1;
  int j = (int)floor(v);
  if (j > ns - 2) j = ns - 2;
  double c = v - j;
  int sg = (u >= 0.0) ? 0 : 1;
  const double* T0 = S->table + (((size_t)sg * ns + j) * ng) * 2;
  const double* T1 = S->table + (((size_t)sg * ns + j + 1) * ng) * 2;
  double f00 = T0[2 * i], f10 = T0[2 * (i + 1)], f01 = T1[2 * i], f11 = T1[2 * (i + 1)];
  double n00 = T0[2 * i + 1], n10 = T0[2 * (i + 1) + 1], n01 = T1[2 * i + 1], n11 = T1[2 * (i + 1) + 1];
  *F = (1 - a) * (1 - c) * f00 + a * (1 - c) * f10 + (1 - a) * c * f01 + a * c * f11;
  *lnN = (1 - a) * (1 - c) * n00 + a * (1 - c) * n10 + (1 - a) * c * n01 + a * c * n11;
  if (dF) {
    double dFdt = (1 - c) * (f10 - f00) + c * (f11 - f01);
    double dtdu = clamped ? 0.0 : u / (gam * gam * log(10.0) * dg);
    *dF = dFdt * dtdu;
  }
}

/* closed-form (radial) drag derivative: d[gamma(mu-beta)]/du = beta mu - 1,
 * D = gamma - u mu, dy/du = -y (beta - mu)/D, g'(y) = g (3/y - e^y/(e^y-1)). */
static void orc_closed_eval(const orc_sim* S, double u, double s, double* F, double* dF, double* lnN)
{
  double x = orc_node_interp(S, S->node_x, s);
  double b = orc_node_interp(S, S->node_b, s);
  double mu = orc_node_interp(S, S->node_mu, s);
  double Fh, Nh;
  orc_radial(&S->p, u, x, b, mu, &Fh, &Nh);
  *F = Fh;
  *lnN = (Nh > 0.0) ? log(Nh) : -700.0;
  if (dF) {
    double th = orc_theta_T(&S->p);
    double gam = sqrt(1.0 + u * u), beta = u / gam;
    double D = gam * orc_one_minus_beta_m(u, gam, mu);
    double y = b / (th * D);
    double g = orc_g(y);
    double K = ORC_R_E * S->p.r_star_cm / (ORC_LAMBDABAR * ORC_LAMBDABAR) * th * th * th / (4.0 * x * x);
    double gp = g * (3.0 / y - 1.0 / (-expm1(-y)));
    double dydu = -y * (beta - mu) / D;
    *dF = K * ((beta * mu - 1.0) * g + gam * (mu - beta) * gp * dydu);
  }
}

/* ------------------------------------------------------------------------ */
/* The learned surrogate as a drag law (FP64 network; see orc_sur_point for  */
/* its inputs and targets).  Parameters: W1[64][4] b1 W2[64][64] b2          */
/* W3[64][64] b3 W4[2][64] b4, 8770 values.                                  */
/* ------------------------------------------------------------------------ */
#define ORC_SUR_NP 8770

void orc_set_surrogate(orc_sim* S, const double* theta)
{
  if (!S->sur) S->sur = malloc(ORC_SUR_NP * sizeof(double));
  memcpy(S->sur, theta, ORC_SUR_NP * sizeof(double));
}

static double orc_silu(double z) { return z / (1.0 + exp(-z)); }
static double orc_dsilu(double z) { double q = 1.0 / (1.0 + exp(-z)); return q * (1.0 + z * (1.0 - q)); }

/* outputs y and their derivatives dy in the first input (forward mode) */
void orc_sur_forward(const double* th, const double* x, double* y, double* dy)
{
  static const int in_n[4] = {4, 64, 64, 64}, out_n[4] = {64, 64, 64, 2};
  double h[64], hd[64], z[64], zd[64];
  for (int i = 0; i < 4; ++i) { h[i] = x[i]; hd[i] = (i == 0) ? 1.0 : 0.0; }
  const double* p = th;
  for (int l = 0; l < 4; ++l) {
    const double* W = p;
    const double* bb = p + out_n[l] * in_n[l];
    for (int j = 0; j < out_n[l]; ++j) {
      double a = bb[j], ad = 0.0;
      for (int i = 0; i < in_n[l]; ++i) { a += W[j * in_n[l] + i] * h[i]; ad += W[j * in_n[l] + i] * hd[i]; }
      z[j] = a; zd[j] = ad;
    }
    for (int j = 0; j < out_n[l]; ++j) {
      if (l < 3) { h[j] = orc_silu(z[j]); hd[j] = orc_dsilu(z[j]) * zd[j]; }
      else { h[j] = z[j]; hd[j] = zd[j]; }
    }
    p = bb + out_n[l];
  }
  y[0] = h[0]; y[1] = h[1]; dy[0] = hd[0]; dy[1] = hd[1];
}

/* ln N^_rad (the single-direction closed form, solid angle pi/x^2) and its
 * derivative in u, in log form (no underflow):
 *   ln N = ln(P/x^2) + 2 ln eps - ln gamma - ln(e^y - 1), eps = b/(gamma D),
 *   D = 1 - beta mu, y = eps/Theta. */
static void orc_ln_nrad(const orc_params* p, double u, double x, double b, double mu, double* lnN, double* dlnN)
{
  double th = orc_theta_T(p);
  double gam = sqrt(1.0 + u * u);
  double D = orc_one_minus_beta_m(u, gam, mu);
  double eps = b / (gam * D), y = eps / th;
  double P = ORC_R_E * p->r_star_cm / (4.0 * ORC_LAMBDABAR * ORC_LAMBDABAR);
  double lnem1 = (y > 20.0) ? y + log1p(-exp(-y)) : log(expm1(y));
  *lnN = log(P / (x * x)) + 2.0 * log(eps) - log(gam) - lnem1;
  double dlng = u / (gam * gam);
  double dlnD = (-mu / (gam * gam * gam)) / D;
  double dlne = -dlng - dlnD;
  *dlnN = (2.0 - y / (-expm1(-y))) * dlne - dlng;
}

/* surrogate F^ (per R_star), dF^/du and ln N^ at (u, s); outside the training
 * box (gamma above 10^G or b outside the range of f2), or with no network set,
 * the table law on the line's quadrature table (Sec. 2.2; the quadrature is
 * the network's fallback) */
static void orc_sur_eval(const orc_sim* S, double u, double s, double* F, double* dF, double* lnN)
{
  const orc_params* p = &S->p;
  double x = orc_node_interp(S, S->node_x, s);
  double b = orc_node_interp(S, S->node_b, s);
  double mu = orc_node_interp(S, S->node_mu, s);
  double gam = sqrt(1.0 + u * u);
  double G = p->table_log10g_max;
  double f[4];
  f[0] = 2.0 * log10(gam) / G - 1.0;
  f[1] = 2.0 * s / S->N - 1.0;
  f[2] = (log10(b) - ORC_SUR_B_MID) / ORC_SUR_B_HALF;
  f[3] = (u < 0.0) ? -1.0 : 1.0;
  if (f[0] > 1.0 || f[2] < -1.0 || f[2] > 1.0 || !S->sur) {
    if (!S->table) {
      /* a cache of the line's fixed table, built the first time it is needed */
      orc_sim* W = (orc_sim*)S;
      W->table = malloc((size_t)2 * p->table_n_s * p->table_n_gamma * 2 * sizeof(double));
      orc_build_table(p, W->table);
    }
    orc_table_eval(S, u, s, F, dF, lnN);
    return;
  }
  double y[2], dy[2];
  orc_sur_forward(S->sur, f, y, dy);
  double l1, d1, l2, d2;
  orc_ln_nrad(p, u, x, b, mu, &l1, &d1);
  orc_ln_nrad(p, u, x, b, orc_sur_edge_mu(u, x, mu), &l2, &d2);
  double a1 = log(0.9) + l1, a2 = log(0.1) + l2;
  double mx = fmax(a1, a2);
  double e1 = exp(a1 - mx), e2 = exp(a2 - mx);
  double B = mx + log(e1 + e2);
  double dB = (e1 * d1 + e2 * d2) / (e1 + e2);
  double Bc = fmax(B, ORC_SUR_LT), dBc = (B > ORC_SUR_LT) ? dB : 0.0;
  double ln_n = Bc + y[1];
  double N = exp(ln_n);
  *lnN = ln_n;
  *F = gam * b * N * y[0];
  if (dF) {
    double df0 = 2.0 / G * u / (gam * gam * log(10.0));
    double dln = dBc + dy[1] * df0;
    *dF = b * N * ((u / gam) * y[0] + gam * y[0] * dln + gam * dy[0] * df0);
  }
}

/* F and dF in code units (du per cell-crossing time), rate in code units */
void orc_drag_code(const orc_sim* S, double u, double s, double* F, double* dF, double* rate)
{
  double Fh = 0.0, dFh = 0.0, lnN = -700.0;
  if (S->p.drag_law == ORC_DRAG_TABLE) orc_table_eval(S, u, s, &Fh, &dFh, &lnN);
  else if (S->p.drag_law == ORC_DRAG_CLOSED) orc_closed_eval(S, u, s, &Fh, &dFh, &lnN);
  else if (S->p.drag_law == ORC_DRAG_SURROGATE) orc_sur_eval(S, u, s, &Fh, &dFh, &lnN);
  double k = S->p.drag_scale / S->R_cells;
  *F = k * Fh;
  if (dF) *dF = k * dFh;
  if (rate) *rate = k * exp(lnN);
}

/* One drag update over dt/2 at fixed s (Sec. 3): limiter test, then either
 * the implicit midpoint [implicit] by Newton or exponential damping to
 * p~ = mu/sqrt(1-mu^2). */
static double orc_drag_half_n(const orc_sim* S, double u0, double s, int64_t* n_newton, int64_t* n_limiter)
{
  double h = 0.5 * S->dt;
  double F0, dF0;
  orc_drag_code(S, u0, s, &F0, &dF0, NULL);
  int newton = 1;
  /* |dp/p0| ~ |F dt/(2 p0)| < dt/(2 tau_min)  <=>  |F| tau_min < |p0|;
   * p0 = 0 always takes the damping branch */
  if (S->tau_min > 0.0) newton = fabs(F0) * S->tau_min < fabs(u0);
  if (newton) {
    (*n_newton)++;
    double u1 = u0 + h * F0;
    for (int it = 0; it < 4; ++it) {
      double F1, dF1;
      orc_drag_code(S, u1, s, &F1, &dF1, NULL);
      double G = u1 - u0 - 0.5 * h * (F0 + F1);
      double dG = 1.0 - 0.5 * h * dF1;
      if (dG < 0.5) dG = 0.5;
      u1 -= G / dG;
    }
    return u1;
  }
  (*n_limiter)++;
  double mu = orc_node_interp(S, S->node_mu, s);
  double ut = mu / sqrt(1.0 - mu * mu);
  return ut + (u0 - ut) * exp(-h / S->tau_min);
}

static double orc_drag_half(orc_sim* S, double u0, double s)
{
  return orc_drag_half_n(S, u0, s, &S->d.newton_branch, &S->d.limiter_branch);
}

/* ------------------------------------------------------------------------ */
/* RICS event kinematics (App. A).  Lepton u_i along +s, field b, photon      */
/* arriving in the lepton rest frame along direction d = +-1 (along +s).     */
/* Excitation [exen, excitedgamma]: the excited lepton (rest energy E_B =     */
/* sqrt(1+2b)) moves in the old rest frame with gamma* = (E_B + 1/E_B)/2,    */
/* gamma* beta* = b/E_B, along d.  De-excitation in its own rest frame at     */
/* angle ct = cos(theta~): E'_g = (E_B - 1/E_B)/(1 + sqrt(ct^2 + (1-ct^2)/   */
/* E_B^2)) (the E_gamma(theta) formula of App. A.2 without cancellation),     */
/* lepton E'_e = E_B - E'_g, p'_e = -E'_g ct.  Boost back to the lab.         */
/* out: [0] u_f, [1] E_gamma, [2] P_gamma (along s), [3] gamma_e, [4] u_e     */
/* ------------------------------------------------------------------------ */
void orc_rics_kinematics(double b, double d, double u_i, double ct, double* out)
{
  double EB = sqrt(1.0 + 2.0 * b);
  double gs = 0.5 * (EB + 1.0 / EB);
  double gbs = b / EB;                  /* gamma* beta* */
  double gi = sqrt(1.0 + u_i * u_i);
  double ge = gs * gi + d * gbs * u_i;  /* lab Lorentz factor of the excited lepton */
  double ue = gs * u_i + d * gbs * gi;
  double st2 = 1.0 - ct * ct;
  double Eg = (EB - 1.0 / EB) / (1.0 + sqrt(ct * ct + st2 / (EB * EB)));
  double Ee = EB - Eg, pe = -Eg * ct;
  out[0] = ue * Ee + ge * pe;
  out[1] = Eg * (ge + ue * ct);
  out[2] = Eg * (ue + ge * ct);
  out[3] = ge;
  out[4] = ue;
}

/* cos(theta~) with density (3/8)(1 + c^2) from one uniform U: CDF
 * (c^3 + 3c + 4)/8 = U, the depressed cubic solved by Cardano's formula:
 * a = 4U - 2, t = cbrt(a + sqrt(a^2 + 1)), c = t - 1/t. */
double orc_cos_dipole(double U)
{
  double a = 4.0 * U - 2.0;
  double t = cbrt(a + sqrt(a * a + 1.0));
  return t - 1.0 / t;
}

/* ------------------------------------------------------------------------ */
/* Charge-conserving deposit: the signed length of [a, b] inside every cell  */
/* (the flux through that cell's E point), weighted by q w / dt.             */
/* ------------------------------------------------------------------------ */
static void orc_deposit_path(const orc_sim* S, double* J, int* jlo, int* jhi, double a, double b, double qw)
{
  double lo = fmin(a, b), hi = fmax(a, b);
  double sgn = (b >= a) ? 1.0 : -1.0;
  int c0 = (int)floor(lo), c1 = (int)floor(hi);
  if (c1 > S->N - 1) c1 = S->N - 1;
  if (c0 < 0) c0 = 0;
  for (int c = c0; c <= c1; ++c) {
    double l = fmin(hi, (double)(c + 1)) - fmax(lo, (double)c);
    if (l > 0.0) {
      J[c] += sgn * qw * l * S->q_p / S->dt;
      if (c < *jlo) *jlo = c;
      if (c > *jhi) *jhi = c;
    }
  }
}

/* The same deposit in integers: positions in fixed point with F fractional
 * bits, weights w_int = rint(w 2^12); J_int[c] = sum q_sign w_int len_c. */
void orc_deposit_int(int N, int Fbits, int64_t n, const int64_t* p0, const int64_t* p1,
                     const double* w, const int32_t* sp, int64_t* Jint)
{
  int64_t one = (int64_t)1 << Fbits, top = (int64_t)N << Fbits;
  for (int64_t k = 0; k < n; ++k) {
    int64_t a = p0[k], b = p1[k];
    if (b < 0) b = 0;
    if (b > top) b = top;
    int64_t lo = a < b ? a : b, hi = a < b ? b : a;
    int64_t sgn = (b >= a) ? 1 : -1;
    int64_t qw = (int64_t)ORC_QS[sp[k]] * orc_wint(w[k]);
    for (int64_t c = lo / one; c <= hi / one && c < N; ++c) {
      int64_t cl = c * one, ch = cl + one;
      int64_t l = (hi < ch ? hi : ch) - (lo > cl ? lo : cl);
      if (l > 0) Jint[c] += sgn * qw * l;
    }
  }
}

/* E at s: linear between cell centres c + 1/2, constant beyond the ends */
static double orc_gather_at(const orc_sim* S, const double* a, double s)
{
  double x = s - 0.5;
  int i = (int)floor(x);
  if (i < 0) return a[0];
  if (i >= S->N - 1) return a[S->N - 1];
  double f = x - i;
  return (1.0 - f) * a[i] + f * a[i + 1];
}

static double orc_gather(const orc_sim* S, double s) { return orc_gather_at(S, S->E, s); }

/* ------------------------------------------------------------------------ */
/* Annihilation at n_max (see the readings at the top).  Called at the end of */
/* a step, after the step counter has advanced.                              */
/* ------------------------------------------------------------------------ */
/* order key of a particle in the annihilation at `step` */
uint64_t orc_annih_key(uint64_t id, int64_t step)
{
  return orc_splitmix64(id ^ orc_splitmix64((uint64_t)step ^ 0xA1111A7Eull));
}

typedef struct { uint64_t key; int64_t k; } orc_keyed;

static int orc_keyed_cmp(const void* a, const void* b)
{
  uint64_t x = ((const orc_keyed*)a)->key, y = ((const orc_keyed*)b)->key;
  return (x > y) - (x < y);
}

static void orc_annihilate(orc_sim* S)
{
  const int N = S->N;
  const int64_t nmax = (int64_t)floor(S->p.n_max_ppc * (double)(1 << ORC_S_BITS));
  int64_t *W = calloc(N, sizeof(int64_t)), *Wp = calloc(N, sizeof(int64_t)), *We = calloc(N, sizeof(int64_t));
  int64_t* cnt = calloc(N, sizeof(int64_t));
  for (int64_t k = 0; k < S->n; ++k) {
    int sp = S->sp[k];
    if (!orc_is_lepton(sp)) continue;
    int c = (int)floor(S->s[k]);
    int64_t w = orc_wint(S->w[k]);
    W[c] += w;
    if (sp == ORC_SP_POSI) { Wp[c] += w; cnt[c]++; }
    if (sp == ORC_SP_ELEC) { We[c] += w; cnt[c]++; }
  }
  /* the pair particles of every cell that annihilates, with their keys */
  int64_t* first = malloc((N + 1) * sizeof(int64_t));
  int64_t* A = calloc(N, sizeof(int64_t));
  first[0] = 0;
  for (int c = 0; c < N; ++c) {
    if (W[c] > nmax) {
      int64_t a = (W[c] - nmax) / 2;
      if (a > Wp[c]) a = Wp[c];
      if (a > We[c]) a = We[c];
      A[c] = a;
    }
    first[c + 1] = first[c] + (A[c] > 0 ? cnt[c] : 0);
  }
  orc_keyed* list = malloc((first[N] > 0 ? first[N] : 1) * sizeof(orc_keyed));
  int64_t* fill = calloc(N, sizeof(int64_t));
  for (int64_t k = 0; k < S->n; ++k) {
    int sp = S->sp[k];
    if (sp != ORC_SP_POSI && sp != ORC_SP_ELEC) continue;
    int c = (int)floor(S->s[k]);
    if (A[c] <= 0) continue;
    list[first[c] + fill[c]].key = orc_annih_key(S->id[k], S->step);
    list[first[c] + fill[c]].k = k;
    fill[c]++;
  }
  unsigned char* gone = calloc(S->n > 0 ? S->n : 1, 1);
  for (int c = 0; c < N; ++c) {
    if (A[c] <= 0) continue;
    orc_keyed* L = list + first[c];
    int64_t m = cnt[c];
    qsort(L, (size_t)m, sizeof(orc_keyed), orc_keyed_cmp);
    int64_t left[2] = { A[c], A[c] };   /* [0]: electrons, [1]: positrons */
    double X = 0.0;                      /* sum of q delta (s - c), weight units */
    for (int64_t i = 0; i < m; ++i) {
      int64_t k = L[i].k;
      int sp = S->sp[k];
      int64_t* r = &left[sp == ORC_SP_POSI ? 1 : 0];
      if (*r == 0) continue;
      int64_t w = orc_wint(S->w[k]);
      int64_t d = w < *r ? w : *r;
      *r -= d;
      X += ORC_QS[sp] * ((double)d / (double)(1 << ORC_S_BITS)) * (S->s[k] - (double)c);
      S->w[k] = (double)(w - d) / (double)(1 << ORC_S_BITS);
      if (w - d == 0) gone[k] = 1;
    }
    /* the current of the removed charge carried to node c, through cell c:
     * E_c -= 4 pi dt J with J dt = -X q_p */
    S->E[c] += 4.0 * ORC_PI * S->q_p * X;
    S->d.annihilated += 2 * A[c];
  }
  int64_t n = 0;
  for (int64_t k = 0; k < S->n; ++k) {
    if (gone[k]) continue;
    S->s[n] = S->s[k]; S->u[n] = S->u[k]; S->w[n] = S->w[k]; S->sp[n] = S->sp[k]; S->id[n] = S->id[k];
    n++;
  }
  S->n = n;
  free(W); free(Wp); free(We); free(cnt); free(first); free(A); free(list); free(fill); free(gone);
}

/* ------------------------------------------------------------------------ */
/* One PIC cycle (Sec. 3), n -> n+1.  E at integer times, u at half times.    */
/* ------------------------------------------------------------------------ */
/* The particles of a step are taken in fixed blocks of ORC_BLOCK; each block
 * sums its current, tallies, lost energy and created particles on its own,
 * and the blocks are merged in block order.  The result is then the same,
 * bit for bit, whether the blocks run one after another or on several
 * threads (orc_set_threads, an OpenMP build): the sums group the particles
 * by block in both cases.  (Grouping a sum changes it only at rounding.) */
#define ORC_BLOCK 4096

static int orc_threads = 1;

void orc_set_threads(int n) { orc_threads = n > 0 ? n : 1; }

int orc_get_threads(void)
{
#ifdef _OPENMP
  return orc_threads;
#else
  return 1;
#endif
}

typedef struct {
  double* J;                           /* N, zero outside [jlo, jhi] */
  int jlo, jhi;
  int64_t psc_clamped, scatters, lost_north, lost_south, pairs_lost_wall, pairs_rejected_nmax, pairs_created;
  int64_t newton_branch, limiter_branch;
  double ke_lost;
  int64_t nc, ccap;                    /* created particles, in particle order */
  double *cs, *cu, *cw;
  int32_t* csp;
  uint64_t* cid;
} orc_acc;

static void orc_acc_init(orc_acc* A, int N)
{
  memset(A, 0, sizeof(*A));
  A->J = calloc(N, sizeof(double));
  A->jlo = N; A->jhi = -1;
  A->ccap = 256;
  A->cs = malloc(A->ccap * sizeof(double)); A->cu = malloc(A->ccap * sizeof(double));
  A->cw = malloc(A->ccap * sizeof(double)); A->csp = malloc(A->ccap * sizeof(int32_t));
  A->cid = malloc(A->ccap * sizeof(uint64_t));
}

static void orc_acc_free(orc_acc* A)
{
  free(A->J); free(A->cs); free(A->cu); free(A->cw); free(A->csp); free(A->cid);
}

static void orc_acc_push(orc_acc* A, double s, double u, double w, int32_t sp, uint64_t id)
{
  if (A->nc + 1 > A->ccap) {
    A->ccap *= 2;
    A->cs = realloc(A->cs, A->ccap * sizeof(double)); A->cu = realloc(A->cu, A->ccap * sizeof(double));
    A->cw = realloc(A->cw, A->ccap * sizeof(double)); A->csp = realloc(A->csp, A->ccap * sizeof(int32_t));
    A->cid = realloc(A->cid, A->ccap * sizeof(uint64_t));
  }
  A->cs[A->nc] = s; A->cu[A->nc] = u; A->cw[A->nc] = w; A->csp[A->nc] = sp; A->cid[A->nc] = id;
  A->nc++;
}

/* Steps 1-7 of the PIC cycle for particles [k0, k1) into A; writes their new
 * s, u and alive flag. */
static void orc_push_range(orc_sim* S, int64_t k0, int64_t k1, const uint32_t key[2], int64_t nmax_int,
                           unsigned char* alive, orc_acc* A)
{
  const orc_params* p = &S->p;
  int N = S->N;
  double dt = S->dt;
  for (int64_t k = k0; k < k1; ++k) {
    int sp = S->sp[k];
    double s = S->s[k], u = S->u[k], w = S->w[k];
    int lep = orc_is_lepton(sp);
    int cell = (int)floor(s);
    if (cell < 0) cell = 0;
    if (cell >= N) cell = N - 1;
    int zone = S->zone[cell];
    int cont = lep && p->drag_law != ORC_DRAG_OFF && (p->rics_mode == ORC_RICS_DRAG_PLUS_PAIRS || !zone);
    /* 1. gather */
    double Ep = orc_gather(S, s);
    /* 2-4. Strang: drag dt/2, Lorentz kick dt, drag dt/2 */
    if (cont) u = orc_drag_half_n(S, u, s, &A->newton_branch, &A->limiter_branch);
    if (S->grav_on) u += (orc_qm(S, sp) * Ep + orc_gather_at(S, S->grav, s) / orc_mass(S, sp)) * dt;
    else u += orc_qm(S, sp) * Ep * dt;
    if (cont) u = orc_drag_half_n(S, u, s, &A->newton_branch, &A->limiter_branch);
    /* 5. Monte-Carlo RICS in the pair zone */
    int make_pair = 0;
    double Pg = 0.0;
    if (lep && p->mc_on && p->drag_law != ORC_DRAG_OFF && zone) {
      double F, rate;
      orc_drag_code(S, u, s, &F, NULL, &rate);
      double psc = rate * dt;
      if (psc > 1.0) { psc = 1.0; A->psc_clamped++; }
      /* the draw's uniform lies on the lattice (0, 1] in steps of 2^-24 and
       * the lepton scatters when it is <= p_sc: below 2^-24 there is nothing
       * to draw */
      if (psc >= ORC_DRAW_MIN) {
        uint32_t ctr[4] = { (uint32_t)S->id[k], (uint32_t)(S->id[k] >> 32), (uint32_t)S->step, ORC_TAG_RICS };
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        if (orc_u24_open(r[0]) <= psc) {
          A->scatters++;
          double b = orc_node_interp(S, S->node_b, s);
          double mu = orc_node_interp(S, S->node_mu, s);
          double gam = sqrt(1.0 + u * u);
          double d = (mu > u / gam) ? 1.0 : -1.0;
          double ct = orc_cos_dipole(orc_u24(r[1]));
          double kin[5];
          orc_rics_kinematics(b, d, u, ct, kin);
          if (p->rics_mode == ORC_RICS_SPLIT) u = kin[0];
          if (p->pairs_on && kin[1] >= p->pair_energy_threshold) { make_pair = 1; Pg = kin[2]; }
        }
      }
    }
    /* 6. move */
    double gam = sqrt(1.0 + u * u);
    double s1 = s + dt * u / gam;
    int lost = (s1 < 0.0) || (s1 >= (double)N);
    /* 7. deposit along the path, clamped at the conducting walls */
    double s1c = s1 < 0.0 ? 0.0 : (s1 > (double)N ? (double)N : s1);
    orc_deposit_path(S, A->J, &A->jlo, &A->jhi, s, s1c, ORC_QS[sp] * w);
    S->s[k] = s1;
    S->u[k] = u;
    alive[k] = !lost;
    if (lost) {
      if (s1 < 0.0) A->lost_north++; else A->lost_south++;
      A->ke_lost += S->q_p * w * orc_mass(S, sp) * (gam - 1.0);   /* energy carried out */
    }
    if (make_pair) {
      if (lost) { A->pairs_lost_wall++; }
      else {
        int pc = (int)floor(s1);
        if (nmax_int >= 0 && S->dens[pc] >= nmax_int) { A->pairs_rejected_nmax++; }
        else {
          for (int m = 0; m < 2; ++m)
            orc_acc_push(A, s1, 0.5 * Pg, w, (m == 0) ? ORC_SP_ELEC : ORC_SP_POSI, orc_child_id(S->id[k], S->step, m));
          A->pairs_created++;
        }
      }
    }
  }
}

/* a block's sums into the step's (in block order), then A is cleared */
static void orc_acc_merge(orc_sim* S, orc_acc* A, orc_acc* G)
{
  for (int c = A->jlo; c <= A->jhi; ++c) { S->J[c] += A->J[c]; A->J[c] = 0.0; }
  A->jlo = S->N; A->jhi = -1;
  S->d.psc_clamped += A->psc_clamped; S->d.scatters += A->scatters;
  S->d.lost_north += A->lost_north; S->d.lost_south += A->lost_south;
  S->d.pairs_lost_wall += A->pairs_lost_wall; S->d.pairs_rejected_nmax += A->pairs_rejected_nmax;
  S->d.pairs_created += A->pairs_created;
  S->d.newton_branch += A->newton_branch; S->d.limiter_branch += A->limiter_branch;
  S->d.ke_lost += A->ke_lost;
  for (int64_t i = 0; i < A->nc; ++i) orc_acc_push(G, A->cs[i], A->cu[i], A->cw[i], A->csp[i], A->cid[i]);
  A->psc_clamped = A->scatters = A->lost_north = A->lost_south = 0;
  A->pairs_lost_wall = A->pairs_rejected_nmax = A->pairs_created = 0;
  A->newton_branch = A->limiter_branch = 0;
  A->ke_lost = 0.0;
  A->nc = 0;
}

/* ------------------------------------------------------------------------ */
/* One PIC cycle (Sec. 3), n -> n+1.  E at integer times, u at half times.    */
/* ------------------------------------------------------------------------ */
void orc_step(orc_sim* S)
{
  const orc_params* p = &S->p;
  int N = S->N;
  double dt = S->dt;
  int64_t n0 = S->n;
  unsigned char* alive = malloc(n0 > 0 ? n0 : 1);
  uint32_t key[2] = { (uint32_t)p->seed, (uint32_t)(p->seed >> 32) };
  int64_t nmax_int = (p->n_max_ppc > 0.0) ? (int64_t)floor(p->n_max_ppc * (double)(1 << ORC_S_BITS)) : -1;
  memset(S->J, 0, N * sizeof(double));
  /* created particles, collected in particle order and appended at the end */
  orc_acc G;
  orc_acc_init(&G, 1);
  int64_t nblk = (n0 + ORC_BLOCK - 1) / ORC_BLOCK;
  int nthr = orc_get_threads();
  if (nthr > 1 && p->drag_law == ORC_DRAG_SURROGATE && !S->table) {
    /* the surrogate's table fallback is built on first use: build it before
     * the threads start */
    S->table = malloc((size_t)2 * p->table_n_s * p->table_n_gamma * 2 * sizeof(double));
    orc_build_table(p, S->table);
  }
#pragma omp parallel num_threads(nthr) if (nthr > 1 && nblk > 1)
  {
    orc_acc A;
    orc_acc_init(&A, N);
#pragma omp for ordered schedule(static, 1)
    for (int64_t b = 0; b < nblk; ++b) {
      int64_t k1 = (b + 1) * ORC_BLOCK < n0 ? (b + 1) * ORC_BLOCK : n0;
      orc_push_range(S, b * ORC_BLOCK, k1, key, nmax_int, alive, &A);
#pragma omp ordered
      orc_acc_merge(S, &A, &G);
    }
    orc_acc_free(&A);
  }
  int64_t nc = G.nc;
  double *cs = G.cs, *cu = G.cu, *cw = G.cw;
  int32_t* csp = G.csp;
  uint64_t* cid = G.cid;

  /* 8. Ampere with the external current: dE/dt = 4 pi (j_ext - J) */
  double E_new_sum = 0.0, E_old_sum = 0.0;
  for (int c = 0; c < N; ++c) {
    double Eo = S->E[c];
    S->E[c] = Eo + 4.0 * ORC_PI * dt * (S->j_ext - S->J[c]);
    E_old_sum += Eo; E_new_sum += S->E[c];
  }
  S->d.ext_work += dt * S->j_ext * 0.5 * (E_old_sum + E_new_sum);

  /* 9. remove losses, append pairs then surface injection */
  int64_t* wcell = S->grav_on ? calloc(N, sizeof(int64_t)) : NULL;   /* plasma weight after the move */
  int64_t m = 0;
  for (int64_t k = 0; k < n0; ++k) {
    if (!alive[k]) continue;
    S->s[m] = S->s[k]; S->u[m] = S->u[k]; S->w[m] = S->w[k]; S->sp[m] = S->sp[k]; S->id[m] = S->id[k];
    if (wcell) wcell[(int)floor(S->s[m])] += orc_wint(S->w[m]);
    m++;
  }
  S->n = m;
  orc_grow(S, S->n + nc);
  for (int64_t k = 0; k < nc; ++k) {
    S->s[S->n] = cs[k]; S->u[S->n] = cu[k]; S->w[S->n] = cw[k]; S->sp[S->n] = csp[k]; S->id[S->n] = cid[k];
    S->n++;
  }
  if (p->inject_mode == ORC_INJECT_RATE) {
    for (int foot = 0; foot < 2; ++foot) {
      /* carriers of weight 1 per step that carry j_ext = j_psi n0 e c through
       * the footpoint: j_psi n0 c dt */
      S->inj_acc[foot] += p->j_psi * p->n0_ppc * dt;
      int64_t cnt = (int64_t)floor(S->inj_acc[foot]);
      S->inj_acc[foot] -= (double)cnt;
      orc_grow(S, S->n + 2 * cnt);
      for (int64_t slot = 0; slot < cnt; ++slot) {
        uint32_t ctr[4] = { (uint32_t)slot, (uint32_t)foot, (uint32_t)S->step, ORC_TAG_INJ };
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        double frac = (double)(r[0] >> 16) * (1.0 / 65536.0);
        double pos = foot == 0 ? frac : (double)N - (1.0 / 65536.0) - frac;
        double rad = sqrt(-2.0 * log(1.0 - orc_u24(r[1])));
        double ang = 2.0 * ORC_PI * orc_u24(r[2]);
        double dir = foot == 0 ? 1.0 : -1.0;
        double ue = dir * fabs(sqrt(p->inject_T) * rad * cos(ang));
        double ui = dir * fabs(sqrt(p->inject_T / p->mass_ratio) * rad * sin(ang));
        for (int mem = 0; mem < 2; ++mem) {
          S->s[S->n] = pos; S->w[S->n] = 1.0;
          S->u[S->n] = mem == 0 ? ue : ui;
          S->sp[S->n] = mem == 0 ? ORC_SP_ATMO : ORC_SP_ION;
          S->id[S->n] = orc_inject_id(S->step, foot, slot, mem);
          S->n++;
        }
        S->d.injected += 2;
      }
    }
  }
  if (p->inject_mode == ORC_INJECT_TOPUP) {
    /* atmosphere: fill each cell's deficit with neutral pairs of weight 1 */
    const int64_t pair_w = 2 * (int64_t)(1 << ORC_S_BITS);
    for (int c = 0; c < N; ++c) {
      if (S->atmo_target[c] < 0) continue;
      int64_t deficit = S->atmo_target[c] - wcell[c];
      int64_t cnt = deficit > 0 ? deficit / pair_w : 0;
      orc_grow(S, S->n + 2 * cnt);
      for (int64_t slot = 0; slot < cnt; ++slot) {
        uint32_t ctr[4] = { (uint32_t)slot, (uint32_t)c, (uint32_t)S->step, ORC_TAG_ATM };
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        double pos = (double)c + (double)(r[0] >> 16) * (1.0 / 65536.0);
        double rad = sqrt(-2.0 * log(1.0 - orc_u24(r[1])));
        double ang = 2.0 * ORC_PI * orc_u24(r[2]);
        double ue = sqrt(p->inject_T) * rad * cos(ang);
        double ui = sqrt(p->inject_T / p->mass_ratio) * rad * sin(ang);
        for (int mem = 0; mem < 2; ++mem) {
          S->s[S->n] = pos; S->w[S->n] = 1.0;
          S->u[S->n] = mem == 0 ? ue : ui;
          S->sp[S->n] = mem == 0 ? ORC_SP_ATMO : ORC_SP_ION;
          S->id[S->n] = orc_atmo_id(S->step, c, slot, mem);
          S->n++;
        }
        S->d.injected += 2;
      }
    }
  }
  free(wcell);
  S->step++;
  if (p->annihilate_every > 0 && p->n_max_ppc > 0.0 && S->step % p->annihilate_every == 0) orc_annihilate(S);
  orc_recount_density(S);
  orc_acc_free(&G);
  free(alive);
}

void orc_run(orc_sim* S, int64_t steps) { for (int64_t i = 0; i < steps; ++i) orc_step(S); }

/* charge density at nodes (CIC), rho_k = q_p sum q w W_k(s) */
void orc_rho(const orc_sim* S, double* rho)
{
  memset(rho, 0, (S->N + 1) * sizeof(double));
  for (int64_t k = 0; k < S->n; ++k) {
    double s = S->s[k];
    int i = (int)floor(s);
    if (i < 0) i = 0;
    if (i > S->N - 1) i = S->N - 1;
    double f = s - i;
    double q = ORC_QS[S->sp[k]] * S->w[k] * S->q_p;
    rho[i] += q * (1.0 - f);
    rho[i + 1] += q * f;
  }
}

void orc_get_diag(orc_sim* S, orc_diag* out)
{
  orc_diag d = S->d;
  for (int i = 0; i < 4; ++i) d.n_alive[i] = 0;
  double ke = 0.0, ch = 0.0;
  for (int64_t k = 0; k < S->n; ++k) {
    int sp = S->sp[k];
    d.n_alive[sp]++;
    double gam = sqrt(1.0 + S->u[k] * S->u[k]);
    ke += S->w[k] * orc_mass(S, sp) * (gam - 1.0);
    ch += ORC_QS[sp] * S->w[k];
  }
  double fe = 0.0, vc = 0.0;
  for (int c = 0; c < S->N; ++c) { fe += S->E[c] * S->E[c] / (8.0 * ORC_PI); vc -= S->E[c]; }
  d.kinetic_energy = S->q_p * ke;
  d.field_energy = fe;
  d.vc = vc;
  d.charge = S->q_p * ch;
  *out = d;
}

/* Exposed for unit tests of the push pieces */
double orc_drag_half_public(orc_sim* S, double u0, double s) { return orc_drag_half(S, u0, s); }
double orc_gather_public(const orc_sim* S, double s) { return orc_gather(S, s); }
double orc_node_interp_public(const orc_sim* S, int which, double s)
{
  const double* t = which == 0 ? S->node_x : (which == 1 ? S->node_b : S->node_mu);
  return orc_node_interp(S, t, s);
}
