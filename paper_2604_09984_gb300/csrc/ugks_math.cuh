// ugks_math.cuh -- per-item arithmetic of the implicit UGKS (Sec. 2 of
// arXiv 2604.09984), written as __host__ __device__ functions templated on
// the arithmetic type R (double for the FP64 path, float for the per-velocity
// arithmetic of the mixed path).  Reduced distributions (h, b), D = 2,
// Keff = 1 + K components of the internal variable, R_gas = 1.
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define UG_HD __host__ __device__ __forceinline__
#else
#define UG_HD inline
#endif

namespace ugks {

template <typename R> struct V2 { R h, b; };

template <typename R> UG_HD R r_exp(R x);
template <> UG_HD double r_exp<double>(double x) { return exp(x); }
// FP32 path: the hardware exponential (relative error a few ulp plus
// |x| * 2^-24, below the FP32 path's tolerance for the arguments that carry
// weight in the velocity sums)
template <> UG_HD float r_exp<float>(float x) {
#ifdef __CUDA_ARCH__
  return __expf(x);
#else
  return expf(x);
#endif
}

// ---------------------------------------------------------------- primitives
// (rho, Vx, Vy, lambda) from W = (rho, rho V, rho E);
// rho E = rho |V|^2 / 2 + (2 + Keff) rho / (4 lambda)   (Sec. 2.1)
struct Prim { double rho, ux, uy, lam; };

UG_HD Prim primitive(const double W[4], int Keff) {
  Prim p;
  p.rho = W[0];
  p.ux = W[1] / W[0];
  p.uy = W[2] / W[0];
  double eint = W[3] - 0.5 * p.rho * (p.ux * p.ux + p.uy * p.uy);
  p.lam = (2.0 + Keff) * p.rho / (4.0 * eint);
  return p;
}

UG_HD void conservative(double rho, double ux, double uy, double lam, int Keff, double W[4]) {
  W[0] = rho;
  W[1] = rho * ux;
  W[2] = rho * uy;
  W[3] = 0.5 * rho * (ux * ux + uy * uy) + (2.0 + Keff) * rho / (4.0 * lam);
}

// tau = mu(T) / p, mu = mu_ref T^omega, T = 1/(2 lam), p = rho T
UG_HD double collision_time(double rho, double lam, double mu_ref, double omega) {
  double T = 1.0 / (2.0 * lam);
  return mu_ref * pow(T, omega) / (rho * T);
}

// ------------------------------------------------------------ equilibria
// Reduced Maxwellian H = rho (lam/pi) exp(-lam |v-V|^2), B = Keff/(2 lam) H.
template <typename R>
UG_HD V2<R> maxwellian(R rho, R ux, R uy, R lam, R vx, R vy, R Keff) {
  R cx = vx - ux, cy = vy - uy;
  R H = rho * (lam * R(M_1_PI)) * r_exp<R>(-lam * (cx * cx + cy * cy));
  return {H, Keff / (R(2) * lam) * H};
}

// Same with the per-state constants precomputed: hpre = rho lam / pi,
// bfac = Keff / (2 lam) (no division per velocity).
template <typename R>
UG_HD V2<R> maxwellian_pre(R hpre, R ux, R uy, R lam, R bfac, R vx, R vy) {
  R cx = vx - ux, cy = vy - uy;
  R H = hpre * r_exp<R>(-lam * (cx * cx + cy * cy));
  return {H, bfac * H};
}

// Division used inside per-velocity loops: exact in FP64, the fast
// approximate quotient (2 ulp) in FP32.
template <typename R> UG_HD R qdiv(R a, R b) { return a / b; }
template <> UG_HD float qdiv<float>(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}

// ---------------------------------------------- interface-flux parameters
// Per-face record of the equilibrium state g0 and its slopes, all at the
// face (Sec. 2.1 "equilibrium state is approximated"), plus the time
// integrals of the coefficients c1..c5 of Eq. fullSolution divided by dt_s.
enum {
  FP_RHO = 0, FP_UX, FP_UY, FP_LAM, FP_QX, FP_QY,
  FP_AX = 6,  FP_AY = 10, FP_AT = 14,
  FP_Q1 = 18, FP_Q2, FP_Q3, FP_Q4, FP_Q5,
  FP_RHOW = 23, FP_LAMW, FP_UFX, FP_UFY, FP_PREF,
  // face geometry for the tiled kernels: S n, S U.n, and the vectors from the
  // (periodic image of the) L cell centre and from the R cell centre to the
  // face centre
  FP_SNX = 28, FP_SNY, FP_SUN, FP_DXLX, FP_DXLY, FP_DXRX, FP_DXRY,
  // per-face constants of the velocity loops: rho lam / pi, 1/(2 lam),
  // Keff/(4 lam), (Keff+2)/(4 lam)
  FP_HPRE = 35, FP_IL, FP_EH, FP_EB,
  NFP = 40
};

// Time integrals q_m = int_0^dts c_m(t) dt (Eq. fullSolution), x = dts/tau;
// closed forms for x >= 1, Taylor series in x below (the closed forms
// cancel catastrophically for small x).
UG_HD void time_integrals(double dts, double tau, double q[5]) {
  double x = dts / tau;
  if (x >= 1.0) {
    double E = exp(-x);
    double em = -expm1(-x);
    q[0] = tau * em;
    q[1] = tau * (dts + tau) * E - tau * tau;
    q[2] = dts - tau * em;
    q[3] = -tau * dts * (1.0 + E) + 2.0 * tau * tau * em;
    q[4] = 0.5 * dts * dts - tau * dts + tau * tau * em;
    return;
  }
  // q1/dts = sum_{m>=1} (-1)^{m+1} x^{m-1}/m!
  // q2/dts^2 = sum_{m>=2} (-1)^{m+1} (m-1) x^{m-2}/m!
  // q4/dts^2 = sum_{m>=3} (-1)^{m+1} (2-m) x^{m-2}/m!
  // q5/dts^2 = sum_{m>=3} (-1)^{m+1} x^{m-2}/m!
  double s1 = 0, s2 = 0, s4 = 0, s5 = 0;
  double xp = 1.0;       // x^{m-1}
  double xm2 = 0.0;      // x^{m-2}
  double ifac = 1.0;     // 1/m!
  for (int m = 1; m <= 24; ++m) {
    ifac *= 1.0 / m;
    double t = ((m & 1) ? 1.0 : -1.0) * ifac;
    s1 += t * xp;
    if (m >= 2) {
      s2 += t * (m - 1) * xm2;
      if (m >= 3) {
        s4 += t * (2 - m) * xm2;
        s5 += t * xm2;
      }
    }
    xm2 = xp;
    xp *= x;
  }
  q[0] = dts * s1;
  q[1] = dts * dts * s2;
  q[2] = dts - dts * s1;
  q[3] = dts * dts * s4;
  q[4] = dts * dts * s5;
}

// Micro slope a with int Psi (a.Psi) g = dW (continuous moments of the
// Maxwellian with N = 2 + Keff thermal components, Psi = (1, u, v,
// (u^2+v^2+xi^2)/2)).  With centred velocity c = v - V and
// a.Psi = b1 + b2 cx + b3 cy + a4 (c^2 + xi^2)/2:
//   b2 = 2 lam (dW2 - Vx dW1)/rho, b3 = 2 lam (dW3 - Vy dW1)/rho,
//   a4 = 8 lam^2/N [dW4/rho - |V|^2 dW1/(2 rho) - (Vx b2 + Vy b3)/(2 lam)
//                    - N dW1/(4 lam rho)],
//   b1 = dW1/rho - a4 N/(4 lam), then back to (a1..a4).
UG_HD void micro_slope(const Prim &g, int Keff, const double dW[4], double a[4]) {
  double N = 2.0 + Keff;
  double lam = g.lam, rho = g.rho, U = g.ux, V = g.uy;
  double d1 = dW[0] / rho, d2 = dW[1] / rho, d3 = dW[2] / rho, d4 = dW[3] / rho;
  double b2 = 2.0 * lam * (d2 - U * d1);
  double b3 = 2.0 * lam * (d3 - V * d1);
  double a4 = 8.0 * lam * lam / N *
              (d4 - 0.5 * (U * U + V * V) * d1 - (U * b2 + V * b3) / (2.0 * lam) - N * d1 / (4.0 * lam));
  double b1 = d1 - a4 * N / (4.0 * lam);
  double a2 = b2 - a4 * U;
  double a3 = b3 - a4 * V;
  a[0] = b1 - a2 * U - a3 * V - 0.5 * a4 * (U * U + V * V);
  a[1] = a2;
  a[2] = a3;
  a[3] = a4;
}

// G = int Psi u_dir (a.Psi) g / rho  (dir 0: u = vx, dir 1: u = vy), closed
// form from the Gaussian moments E[c_x^2] = s2, E[c_x^2 Z] = (N+2) s2^2,
// E[Z] = N s2, E[Z^2] = N (N+2) s2^2, s2 = 1/(2 lam), Z = c^2 + xi^2.
UG_HD void flux_moment(const Prim &g, int Keff, const double a[4], int dir, double G[4]) {
  double N = 2.0 + Keff;
  double s2 = 1.0 / (2.0 * g.lam);
  double U = g.ux, V = g.uy, U2 = U * U + V * V;
  double b2 = a[1] + a[3] * U;
  double b3 = a[2] + a[3] * V;
  double b1 = a[0] + a[1] * U + a[2] * V + 0.5 * a[3] * U2;
  double m0 = b1 + a[3] * N * 0.5 * s2;                  // E[phi]
  double Ex = b2 * s2, Ey = b3 * s2;                     // E[c phi]
  double Exx = b1 * s2 + 0.5 * a[3] * (N + 2.0) * s2 * s2; // E[cx^2 phi] = E[cy^2 phi]
  double EZ = b1 * N * s2 + 0.5 * a[3] * N * (N + 2.0) * s2 * s2;   // E[Z phi]
  double EP4 = 0.5 * U2 * m0 + U * Ex + V * Ey + 0.5 * EZ;           // E[Psi4 phi]
  double Euv = U * V * m0 + U * Ey + V * Ex;
  if (dir == 0) {
    G[0] = U * m0 + Ex;
    G[1] = U * U * m0 + 2.0 * U * Ex + Exx;
    G[2] = Euv;
    G[3] = U * EP4 + 0.5 * U2 * Ex + U * Exx + 0.5 * b2 * (N + 2.0) * s2 * s2;
  } else {
    G[0] = V * m0 + Ey;
    G[1] = Euv;
    G[2] = V * V * m0 + 2.0 * V * Ey + Exx;
    G[3] = V * EP4 + 0.5 * U2 * Ey + V * Exx + 0.5 * b3 * (N + 2.0) * s2 * s2;
  }
}

// Time slope A from compatibility int Psi [(ax.Psi) wx + (ay.Psi) wy + A.Psi] g
// = 0 with w = v - U_f:  M A = -(rho Gx + rho Gy - Ufx dWx - Ufy dWy).
UG_HD void time_slope(const Prim &g, int Keff, const double ax[4], const double ay[4],
                      const double dWx[4], const double dWy[4], double Ufx, double Ufy,
                      double A[4]) {
  double Gx[4], Gy[4], r[4];
  flux_moment(g, Keff, ax, 0, Gx);
  flux_moment(g, Keff, ay, 1, Gy);
  for (int m = 0; m < 4; ++m)
    r[m] = -(g.rho * Gx[m] + g.rho * Gy[m] - Ufx * dWx[m] - Ufy * dWy[m]);
  micro_slope(g, Keff, r, A);
}

// Time-integrated interface distribution / dts for one velocity (Eq.
// fullSolution with the Sec. 2.2 average):
//   qq1 f + qq2 w.grad f + qq3 (g0 + g0+) + qq4 w.grad g0 + qq5 d_t g0
// ff = upwind face value, wgf = w.grad f of the upwind cell.
template <typename R>
UG_HD V2<R> interface_integral(const R *P, R vx, R vy, V2<R> ff, V2<R> wgf, R Keff, R Kint,
                               R Pr) {
  R ux = P[FP_UX], uy = P[FP_UY], lam = P[FP_LAM];
  R cx = vx - ux, cy = vy - uy;
  R c2 = cx * cx + cy * cy;
  R H = P[FP_HPRE] * r_exp<R>(-lam * c2);
  R il = P[FP_IL];
  R B = Keff * il * H;
  // Shakhov correction (Sec. 2.1, reduced H+, B+ as printed)
  R cq = cx * P[FP_QX] + cy * P[FP_QY];
  R pref = P[FP_PREF] * cq;      // 4 (1-Pr) lam^2 / (5 rho) * c.q
  R Hp = pref * (R(2) * lam * c2 - R(4)) * H;
  R Bp = pref * ((R(2) * lam * c2 - R(2)) * Keff - R(2) * Kint) * H * il;
  // slopes: (a.Psi) reduced over xi
  R v2 = vx * vx + vy * vy;
  R wx = vx - P[FP_UFX], wy = vy - P[FP_UFY];
  const R *ax = P + FP_AX, *ay = P + FP_AY, *at = P + FP_AT;
  R bx = ax[0] + ax[1] * vx + ax[2] * vy + R(0.5) * ax[3] * v2;
  R by = ay[0] + ay[1] * vx + ay[2] * vy + R(0.5) * ay[3] * v2;
  R bt = at[0] + at[1] * vx + at[2] * vy + R(0.5) * at[3] * v2;
  R eh = P[FP_EH], eb = P[FP_EB];
  R sgh = wx * (bx + ax[3] * eh) + wy * (by + ay[3] * eh);
  R sgb = wx * (bx + ax[3] * eb) + wy * (by + ay[3] * eb);
  R sth = bt + at[3] * eh, stb = bt + at[3] * eb;
  V2<R> out;
  out.h = P[FP_Q1] * ff.h + P[FP_Q2] * wgf.h + P[FP_Q3] * (H + Hp) + P[FP_Q4] * H * sgh +
          P[FP_Q5] * H * sth;
  out.b = P[FP_Q1] * ff.b + P[FP_Q2] * wgf.b + P[FP_Q3] * (B + Bp) + P[FP_Q4] * B * sgb +
          P[FP_Q5] * B * stb;
  (void)Pr;
  return out;
}

// Per-cell record of the Shakhov equilibrium (Sec. 2.1) with the constants
// of the velocity loop precomputed: f+ of one velocity without divisions.
enum { SH_HPRE = 0, SH_UX, SH_UY, SH_LAM, SH_QX, SH_QY, SH_PREF, SH_IL, SH_ITAU, SH_VOL, NSH = 10 };
template <typename R>
UG_HD V2<R> shakhov_rec(const R *c, R vx, R vy, R Keff, R Kint) {
  R cx = vx - c[SH_UX], cy = vy - c[SH_UY];
  R c2 = cx * cx + cy * cy;
  R lam = c[SH_LAM], il = c[SH_IL];
  R H = c[SH_HPRE] * r_exp<R>(-lam * c2);
  R pref = c[SH_PREF] * (cx * c[SH_QX] + cy * c[SH_QY]);
  R Hp = pref * (R(2) * lam * c2 - R(4)) * H;
  R Bp = pref * ((R(2) * lam * c2 - R(2)) * Keff - R(2) * Kint) * H * il;
  return {H + Hp, Keff * il * H + Bp};
}

// Shakhov equilibrium f+ = g + g+ of a cell (Sec. 2.1), one velocity.
template <typename R>
UG_HD V2<R> shakhov(R rho, R ux, R uy, R lam, R qx, R qy, R vx, R vy, R Keff, R Kint, R Pr) {
  R cx = vx - ux, cy = vy - uy;
  R c2 = cx * cx + cy * cy;
  R H = rho * (lam * R(M_1_PI)) * r_exp<R>(-lam * c2);
  R il = R(1) / (R(2) * lam);
  R pref = R(4) * (R(1) - Pr) * lam * lam / (R(5) * rho) * (cx * qx + cy * qy);
  R Hp = pref * (R(2) * lam * c2 - R(4)) * H;
  R Bp = pref * ((R(2) * lam * c2 - R(2)) * Keff - R(2) * Kint) * H * il;
  return {H + Hp, Keff * il * H + Bp};
}

// van Leer limited slope of two centre differences
template <typename R> UG_HD R vanleer(R a, R b) {
  R p = a * b;
  return p > R(0) ? qdiv<R>(R(2) * p, a + b) : R(0);
}

}  // namespace ugks
