// tp_map.cu -- test-particle drag maps over many field lines (the paper's
// appendix on the extent of the pair-producing region, Figs. 6 and 7).
//
// A lepton enters each dipole line r = r_eq sin^2(theta) at the northern
// footpoint with gamma0 and moves under the RICS drag alone, from radially
// streaming photons (Eq. contdrag).  One thread follows one line in FP64,
// in theta (ds = r_eq sin(theta) sqrt(1 + 3 cos^2 theta) dtheta), time in
// R*/c.  A step of dt:
//   u1 - u0 - dt/2 (F(u0) + F(u1)) = 0 at fixed theta, Newton on the exact
//     derivative of the closed form;
//   tau += dt/2 (N(u0) + N(u1))    (expected scatterings);
//   theta += dt/2 (beta0 + beta1) / (ds/dtheta at theta0).
// It stops at the equator (the line is symmetric) or at t_max, and reports
// gamma_min, the first scattering (tau = 1), where b falls below b_thr, the
// extent l_pp of the pair-producing region and the region (I: b > b_thr to
// the equator and gamma_min > 1; II: b falls below b_thr, gamma_min > 1;
// III: gamma_min ~ 1).  Lines are independent: the map is one launch.
#include <cuda_runtime.h>
#include <math.h>

#include "pic1d_internal.h"

namespace pic1d {
namespace {

constexpr double kPiD = 3.141592653589793;

struct TpPhys {
  double theta_T;      // kT / (m_e c^2)
  double pref;         // r_e R* / lbar^2
  double b_star;
  int b_convention;
  double drag_scale;
};

__device__ void tp_field(const TpPhys& Q, double r_eq, double th, double& x, double& b, double& mu) {
  const double c = cos(th), s = sin(th);
  x = r_eq * s * s;
  const double root = sqrt(1.0 + 3.0 * c * c);
  b = Q.b_star * root / (x * x * x);
  if (Q.b_convention == 1) b *= 0.5;
  mu = 2.0 * c / root;
}

__device__ double tp_omb(double u, double gam, double m) {   // 1 - beta m without cancellation
  const double sm = (u >= 0.0) ? m : -m;
  const double omb = 1.0 / (gam * (gam + fabs(u)));
  return (1.0 - sm) + sm * omb;
}

// drag F^ (per R*), dF^/du and rate N^ (per R*/c) of the closed form
__device__ void tp_drag(const TpPhys& Q, double u, double x, double b, double mu, double& F, double& dF,
                        double& N) {
  const double th = Q.theta_T;
  const double gam = sqrt(1.0 + u * u), beta = u / gam;
  const double Dm = tp_omb(u, gam, mu);
  const double eps = b / (gam * Dm), y = eps / th;
  const double em = expm1(y);
  const double g = y * y * y / em;
  const double Fh = Q.pref * th * th * th / (4.0 * x * x) * gam * (mu - beta) * g;
  const double Nh = Q.pref / (4.0 * x * x * gam) * eps * eps / em;
  const double D = gam * Dm;
  const double K = Q.pref * th * th * th / (4.0 * x * x);
  const double gp = g * (3.0 / y - 1.0 / (-expm1(-y)));
  const double dydu = -y * (beta - mu) / D;
  F = Q.drag_scale * Fh;
  dF = Q.drag_scale * K * ((beta * mu - 1.0) * g + gam * (mu - beta) * gp * dydu);
  N = Q.drag_scale * Nh;
}

__device__ double tp_arcA(double c) {
  return 0.5 * c * sqrt(1.0 + 3.0 * c * c) + asinh(sqrt(3.0) * c) / (2.0 * sqrt(3.0));
}

// arc length from the northern footpoint to theta
__device__ double tp_arc(double r_eq, double th) {
  const double c0 = sqrt(1.0 - 1.0 / r_eq);
  return r_eq * (tp_arcA(c0) - tp_arcA(cos(th)));
}

__global__ void k_tp_map(TpPhys Q, const double* r_eqs, int n, double gamma0, double dt, double t_max,
                         double b_thr, double gamma_eps, pic1d_tp_result* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double r_eq = r_eqs[k];
  double th = asin(sqrt(1.0 / r_eq));
  double u = sqrt(gamma0 * gamma0 - 1.0);
  double gmin = gamma0, tau = 0.0, t = 0.0, th_first = -1.0;
  long long steps = 0;
  while (th < 0.5 * kPiD && t < t_max) {
    double x, b, mu;
    tp_field(Q, r_eq, th, x, b, mu);
    double F0, dF0, N0;
    tp_drag(Q, u, x, b, mu, F0, dF0, N0);
    double u1 = u + dt * F0;
    for (int it = 0; it < 50; ++it) {
      double F1, dF1, N1;
      tp_drag(Q, u1, x, b, mu, F1, dF1, N1);
      const double G = u1 - u - 0.5 * dt * (F0 + F1);
      double dG = 1.0 - 0.5 * dt * dF1;
      if (dG < 0.5) dG = 0.5;
      const double un = u1 - G / dG;
      const bool done = fabs(un - u1) <= 1e-14 * (1.0 + fabs(un));
      u1 = un;
      if (done) break;
    }
    double F1, dF1, N1;
    tp_drag(Q, u1, x, b, mu, F1, dF1, N1);
    const double tau1 = tau + 0.5 * dt * (N0 + N1);
    const double beta0 = u / sqrt(1.0 + u * u), beta1 = u1 / sqrt(1.0 + u1 * u1);
    const double c = cos(th);
    const double h = r_eq * sin(th) * sqrt(1.0 + 3.0 * c * c);
    const double th1 = th + 0.5 * dt * (beta0 + beta1) / h;
    if (th_first < 0.0 && tau < 1.0 && tau1 >= 1.0) th_first = th + (1.0 - tau) / (tau1 - tau) * (th1 - th);
    u = u1;
    tau = tau1;
    th = th1;
    t += dt;
    ++steps;
    const double g1 = sqrt(1.0 + u * u);
    if (g1 < gmin) gmin = g1;
  }
  double xe, be, me;
  tp_field(Q, r_eq, 0.5 * kPiD, xe, be, me);
  double th_b = 0.5 * kPiD;
  if (be < b_thr) {
    double lo = asin(sqrt(1.0 / r_eq)), hi = 0.5 * kPiD;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      double xm, bm, mm;
      tp_field(Q, r_eq, mid, xm, bm, mm);
      if (bm >= b_thr) lo = mid;
      else hi = mid;
    }
    th_b = 0.5 * (lo + hi);
  }
  const double L = 2.0 * r_eq * tp_arcA(sqrt(1.0 - 1.0 / r_eq));
  const double s_first = (th_first >= 0.0) ? tp_arc(r_eq, th_first) : -1.0;
  const double s_b = tp_arc(r_eq, th_b);
  double lpp = 0.0;
  if (s_first >= 0.0) {
    if (be >= b_thr) lpp = L - 2.0 * s_first;
    else lpp = (s_b > s_first) ? s_b - s_first : 0.0;
  }
  pic1d_tp_result R;
  R.gamma_min = gmin;
  R.theta_first = th_first;
  R.theta_b = th_b;
  R.s_first = s_first;
  R.s_b = s_b;
  R.L = L;
  R.l_pp = lpp;
  R.b_eq = be;
  R.t_end = t;
  R.u_end = u;
  R.steps = steps;
  R.region = (gmin <= 1.0 + gamma_eps) ? 3 : ((be >= b_thr) ? 1 : 2);
  R.pad = 0;
  out[k] = R;
}

}  // namespace

cudaError_t tp_launch_map(const pic1d_params& p, const double* r_eq_dev, int n, double gamma0, double dt,
                          double t_max, double b_thr, double gamma_eps, pic1d_tp_result* out_dev,
                          cudaStream_t s) {
  TpPhys Q;
  Q.theta_T = p.kT_keV / 510.99895;
  Q.pref = 2.8179403262e-13 * p.r_star_cm / (3.8615926796e-11 * 3.8615926796e-11);
  Q.b_star = p.b_star;
  Q.b_convention = p.b_convention;
  Q.drag_scale = p.drag_scale;
  k_tp_map<<<(n + 63) / 64, 64, 0, s>>>(Q, r_eq_dev, n, gamma0, dt, t_max, b_thr, gamma_eps, out_dev);
  return cudaGetLastError();
}

}  // namespace pic1d
