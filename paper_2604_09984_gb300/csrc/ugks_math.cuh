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
template <typename R> struct PrimR { R rho, ux, uy, lam; };
typedef PrimR<double> Prim;

template <typename R> UG_HD PrimR<R> primitive_r(const R W[4], int Keff) {
  PrimR<R> p;
  p.rho = W[0];
  R irho = R(1) / W[0];
  p.ux = W[1] * irho;
  p.uy = W[2] * irho;
  R eint = W[3] - R(0.5) * p.rho * (p.ux * p.ux + p.uy * p.uy);
  p.lam = (R(2) + R(Keff)) * p.rho / (R(4) * eint);
  return p;
}
UG_HD Prim primitive(const double W[4], int Keff) { return primitive_r<double>(W, Keff); }

UG_HD void conservative(double rho, double ux, double uy, double lam, int Keff, double W[4]) {
  W[0] = rho;
  W[1] = rho * ux;
  W[2] = rho * uy;
  W[3] = 0.5 * rho * (ux * ux + uy * uy) + (2.0 + Keff) * rho / (4.0 * lam);
}

template <typename R> UG_HD R r_pow(R x, R y);
template <> UG_HD double r_pow<double>(double x, double y) { return pow(x, y); }
template <> UG_HD float r_pow<float>(float x, float y) { return powf(x, y); }

// tau = mu(T) / p, mu = mu_ref T^omega, T = 1/(2 lam), p = rho T
template <typename R> UG_HD R collision_time_r(R rho, R lam, R mu_ref, R omega) {
  R T = R(1) / (R(2) * lam);
  return mu_ref * r_pow<R>(T, omega) / (rho * T);
}
UG_HD double collision_time(double rho, double lam, double mu_ref, double omega) {
  return collision_time_r<double>(rho, lam, mu_ref, omega);
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
  // the equilibrium factors of the interface distribution as cubics in
  // c = v - U0 (10 coefficients each, written by the face-coefficient pass)
  FP_IH = 40, FP_IB = 50,
  NFP = 60
};

// Time integrals q_m = int_0^dts c_m(t) dt (Eq. fullSolution), x = dts/tau;
// closed forms for x >= 1, Taylor series in x below (the closed forms
// cancel catastrophically for small x).
template <typename R> UG_HD R r_expm1(R x);
template <> UG_HD double r_expm1<double>(double x) { return expm1(x); }
template <> UG_HD float r_expm1<float>(float x) { return expm1f(x); }
template <typename R> UG_HD R r_exp_full(R x);
template <> UG_HD double r_exp_full<double>(double x) { return exp(x); }
template <> UG_HD float r_exp_full<float>(float x) { return expf(x); }

// series terms: 1/m! below the type's epsilon for m past the count
template <typename R> struct SeriesTerms;
template <> struct SeriesTerms<double> { static constexpr int N = 24; };
template <> struct SeriesTerms<float> { static constexpr int N = 13; };

template <typename R> UG_HD void time_integrals_r(R dts, R tau, R q[5]) {
  R x = dts / tau;
  if (x >= R(1)) {
    R E = r_exp_full<R>(-x);
    R em = -r_expm1<R>(-x);
    q[0] = tau * em;
    q[1] = tau * (dts + tau) * E - tau * tau;
    q[2] = dts - tau * em;
    q[3] = -tau * dts * (R(1) + E) + R(2) * tau * tau * em;
    q[4] = R(0.5) * dts * dts - tau * dts + tau * tau * em;
    return;
  }
  // q1/dts = sum_{m>=1} (-1)^{m+1} x^{m-1}/m!
  // q2/dts^2 = sum_{m>=2} (-1)^{m+1} (m-1) x^{m-2}/m!
  // q4/dts^2 = sum_{m>=3} (-1)^{m+1} (2-m) x^{m-2}/m!
  // q5/dts^2 = sum_{m>=3} (-1)^{m+1} x^{m-2}/m!
  R s1 = 0, s2 = 0, s4 = 0, s5 = 0;
  R xp = 1;       // x^{m-1}
  R xm2 = 0;      // x^{m-2}
  R ifac = 1;     // 1/m!
#pragma unroll
  for (int m = 1; m <= SeriesTerms<R>::N; ++m) {
    ifac *= R(1) / R(m);
    R tm = ((m & 1) ? R(1) : R(-1)) * ifac;
    s1 += tm * xp;
    if (m >= 2) {
      s2 += tm * R(m - 1) * xm2;
      if (m >= 3) {
        s4 += tm * R(2 - m) * xm2;
        s5 += tm * xm2;
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
UG_HD void time_integrals(double dts, double tau, double q[5]) { time_integrals_r<double>(dts, tau, q); }

// Micro slope a with int Psi (a.Psi) g = dW (continuous moments of the
// Maxwellian with N = 2 + Keff thermal components, Psi = (1, u, v,
// (u^2+v^2+xi^2)/2)).  With centred velocity c = v - V and
// a.Psi = b1 + b2 cx + b3 cy + a4 (c^2 + xi^2)/2:
//   b2 = 2 lam (dW2 - Vx dW1)/rho, b3 = 2 lam (dW3 - Vy dW1)/rho,
//   a4 = 8 lam^2/N [dW4/rho - |V|^2 dW1/(2 rho) - (Vx b2 + Vy b3)/(2 lam)
//                    - N dW1/(4 lam rho)],
//   b1 = dW1/rho - a4 N/(4 lam), then back to (a1..a4).
// The reciprocals a face's slope solves share (1/rho, 1/(2 lam), 1/N), so
// the three solves of a face (two micro slopes, the time slope) divide once.
template <typename R> struct SlopeInv { R irho, il, iN; };
template <typename R> UG_HD SlopeInv<R> slope_inv(const PrimR<R> &g, int Keff) {
  return {R(1) / g.rho, R(1) / (R(2) * g.lam), R(1) / (R(2) + R(Keff))};
}

template <typename R>
UG_HD void micro_slope_r(const PrimR<R> &g, int Keff, const SlopeInv<R> &v, const R dW[4], R a[4]) {
  R N = R(2) + R(Keff);
  R lam = g.lam, U = g.ux, V = g.uy;
  R d1 = dW[0] * v.irho, d2 = dW[1] * v.irho, d3 = dW[2] * v.irho, d4 = dW[3] * v.irho;
  R b2 = R(2) * lam * (d2 - U * d1);
  R b3 = R(2) * lam * (d3 - V * d1);
  // 1/(4 lam) = il / 2
  R a4 = R(8) * lam * lam * v.iN *
         (d4 - R(0.5) * (U * U + V * V) * d1 - (U * b2 + V * b3) * v.il - N * d1 * (R(0.5) * v.il));
  R b1 = d1 - a4 * N * (R(0.5) * v.il);
  R a2 = b2 - a4 * U;
  R a3 = b3 - a4 * V;
  a[0] = b1 - a2 * U - a3 * V - R(0.5) * a4 * (U * U + V * V);
  a[1] = a2;
  a[2] = a3;
  a[3] = a4;
}

// G = int Psi u_dir (a.Psi) g / rho  (dir 0: u = vx, dir 1: u = vy), closed
// form from the Gaussian moments E[c_x^2] = s2, E[c_x^2 Z] = (N+2) s2^2,
// E[Z] = N s2, E[Z^2] = N (N+2) s2^2, s2 = 1/(2 lam), Z = c^2 + xi^2.
template <typename R>
UG_HD void flux_moment_r(const PrimR<R> &g, int Keff, R il, const R a[4], int dir, R G[4]) {
  R N = R(2) + R(Keff);
  R s2 = il;                      // 1/(2 lam)
  R U = g.ux, V = g.uy, U2 = U * U + V * V;
  R b2 = a[1] + a[3] * U;
  R b3 = a[2] + a[3] * V;
  R b1 = a[0] + a[1] * U + a[2] * V + R(0.5) * a[3] * U2;
  R m0 = b1 + a[3] * N * R(0.5) * s2;                     // E[phi]
  R Ex = b2 * s2, Ey = b3 * s2;                           // E[c phi]
  R Exx = b1 * s2 + R(0.5) * a[3] * (N + R(2)) * s2 * s2;  // E[cx^2 phi] = E[cy^2 phi]
  R EZ = b1 * N * s2 + R(0.5) * a[3] * N * (N + R(2)) * s2 * s2;   // E[Z phi]
  R EP4 = R(0.5) * U2 * m0 + U * Ex + V * Ey + R(0.5) * EZ;          // E[Psi4 phi]
  R Euv = U * V * m0 + U * Ey + V * Ex;
  if (dir == 0) {
    G[0] = U * m0 + Ex;
    G[1] = U * U * m0 + R(2) * U * Ex + Exx;
    G[2] = Euv;
    G[3] = U * EP4 + R(0.5) * U2 * Ex + U * Exx + R(0.5) * b2 * (N + R(2)) * s2 * s2;
  } else {
    G[0] = V * m0 + Ey;
    G[1] = Euv;
    G[2] = V * V * m0 + R(2) * V * Ey + Exx;
    G[3] = V * EP4 + R(0.5) * U2 * Ey + V * Exx + R(0.5) * b3 * (N + R(2)) * s2 * s2;
  }
}

// Time slope A from compatibility int Psi [(ax.Psi) wx + (ay.Psi) wy + A.Psi] g
// = 0 with w = v - U_f:  M A = -(rho Gx + rho Gy - Ufx dWx - Ufy dWy).
template <typename R>
UG_HD void time_slope_r(const PrimR<R> &g, int Keff, const SlopeInv<R> &v, const R ax[4], const R ay[4],
                        const R dWx[4], const R dWy[4], R Ufx, R Ufy, R A[4]) {
  R Gx[4], Gy[4], r[4];
  flux_moment_r<R>(g, Keff, v.il, ax, 0, Gx);
  flux_moment_r<R>(g, Keff, v.il, ay, 1, Gy);
  for (int m = 0; m < 4; ++m)
    r[m] = -(g.rho * Gx[m] + g.rho * Gy[m] - Ufx * dWx[m] - Ufy * dWy[m]);
  micro_slope_r<R>(g, Keff, v, r, A);
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
