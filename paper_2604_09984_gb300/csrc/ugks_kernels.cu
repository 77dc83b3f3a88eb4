// ugks_kernels.cu -- CUDA kernels of the implicit UGKS step (arXiv 2604.09984
// Sec. 2.2 Steps 1-8) on moving structured blocks, and the mesh-motion /
// geometry kernels (Sec. 3 Step 1).  Launch wrappers at the end are the only
// symbols used by the host orchestration (ugks_api.cu).
#include <cstdlib>
#include <cstring>
#include "ugks_internal.cuh"
#include "ugks_launch.h"

namespace ugks {

// ------------------------------------------------------------- geometry
// x = (m00 x0 + m01 y0) + b0, y = (m10 x0 + m11 y0) + b1 without contraction
// (bit-identical to the FP64 reference evaluation).
__global__ void k_move_nodes(Dev d) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.nn) return;
  const double *a = d.affine + 6 * d.node_block[n];
  double x = d.X_ref[2 * n], y = d.X_ref[2 * n + 1];
  d.X_new[2 * n] = __dadd_rn(__dadd_rn(__dmul_rn(a[0], x), __dmul_rn(a[1], y)), a[4]);
  d.X_new[2 * n + 1] = __dadd_rn(__dadd_rn(__dmul_rn(a[2], x), __dmul_rn(a[3], y)), a[5]);
}

__device__ __forceinline__ double shoelace(const double *X, const int *nd) {
  double x1 = X[2 * nd[0]], y1 = X[2 * nd[0] + 1], x2 = X[2 * nd[1]], y2 = X[2 * nd[1] + 1];
  double x3 = X[2 * nd[2]], y3 = X[2 * nd[2] + 1], x4 = X[2 * nd[3]], y4 = X[2 * nd[3] + 1];
  return 0.5 * __dsub_rn(__dmul_rn(x3 - x1, y4 - y2), __dmul_rn(y3 - y1, x4 - x2));
}

// Cell volumes at both levels (shoelace), mid-time and new vertex centres,
// period vector of the cell's row.
__global__ void k_cell_geom(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  const int *nd = d.cell_nodes + 4 * c;
  double vo = shoelace(d.X_old, nd), vn = shoelace(d.X_new, nd);
  d.vol_old[c] = vo;
  d.vol_new[c] = vn;
  if (!(vn > 0.0) || !(vo > 0.0)) atomicOr(d.err, EF_GEOMETRY);
  for (int m = 0; m < 2; ++m) {
    double pm[4], pn[4];
    for (int v = 0; v < 4; ++v) {
      pm[v] = 0.5 * (d.X_old[2 * nd[v] + m] + d.X_new[2 * nd[v] + m]);
      pn[v] = d.X_new[2 * nd[v] + m];
    }
    d.xc[2 * c + m] = 0.25 * ((pm[0] + pm[1]) + (pm[2] + pm[3]));
    d.xc_new[2 * c + m] = 0.25 * ((pn[0] + pn[1]) + (pn[2] + pn[3]));
    int r0 = d.cell_row[2 * c], r1 = d.cell_row[2 * c + 1];
    double a = 0.5 * (d.X_old[2 * r0 + m] + d.X_new[2 * r0 + m]);
    double b = 0.5 * (d.X_old[2 * r1 + m] + d.X_new[2 * r1 + m]);
    d.period[2 * c + m] = b - a;
  }
}

// Mid-time face vector S n (L -> R / outward), centre, face velocity (mean
// node velocity) and S U.n.
__global__ void k_face_geom(Dev d) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.nf) return;
  int a = d.face_a[f], b = d.face_b[f];
  double ax = 0.5 * (d.X_old[2 * a] + d.X_new[2 * a]), ay = 0.5 * (d.X_old[2 * a + 1] + d.X_new[2 * a + 1]);
  double bx = 0.5 * (d.X_old[2 * b] + d.X_new[2 * b]), by = 0.5 * (d.X_old[2 * b + 1] + d.X_new[2 * b + 1]);
  double ex = bx - ax, ey = by - ay;
  double S = sqrt(ex * ex + ey * ey);
  d.Sn[2 * f] = ey;
  d.Sn[2 * f + 1] = -ex;
  d.S[f] = S;
  d.nrm[2 * f] = ey / S;
  d.nrm[2 * f + 1] = -ex / S;
  d.xf[2 * f] = 0.5 * (ax + bx);
  d.xf[2 * f + 1] = 0.5 * (ay + by);
  double ufx = 0.5 * ((d.X_new[2 * a] - d.X_old[2 * a]) + (d.X_new[2 * b] - d.X_old[2 * b])) / d.dt;
  double ufy = 0.5 * ((d.X_new[2 * a + 1] - d.X_old[2 * a + 1]) + (d.X_new[2 * b + 1] - d.X_old[2 * b + 1])) / d.dt;
  d.Uf[2 * f] = ufx;
  d.Uf[2 * f + 1] = ufy;
  d.SUn[f] = ufx * ey + ufy * (-ex);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Lane-local sum in the arithmetic type: plain for FP64, Neumaier-compensated
// for FP32 (the mixed path keeps velocity sums accurate to a few FP32 ulps
// before the FP64 warp reduction).
template <typename T> struct Acc {
  T s = T(0);
  __device__ __forceinline__ void add(T x) { s += x; }
  __device__ __forceinline__ double get() const { return (double)s; }
};
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// Warp total of per-lane accumulators.  FP32: the (sum, compensation) pairs
// are combined in FP32 with an error-free sum at every butterfly level (no
// FP64 arithmetic on the way); FP64: plain FP64 butterfly.
__device__ __forceinline__ double warp_total(const Acc<double> &a) {
  double v = a.s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// FP32: the total rounded once to FP32 (relative error ~ulp of the total;
// the compensation only has to stop the error growing with the term count).
__device__ __forceinline__ float warp_total(const Acc<float> &a) {
  float s = a.s, c = a.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float os = __shfl_xor_sync(0xffffffffu, s, o), oc = __shfl_xor_sync(0xffffffffu, c, o);
    float t = s + os, bb = t - s;
    float e = (s - (t - bb)) + (os - bb);
    s = t;
    c = c + oc + e;
  }
  return s + c;
}


// Reading R3: dts_i = cfl_s Omega_i^{n+1} / max_k sum_faces S max(w_out, 0).
// The sum is a convex piecewise-linear function of v, so over the tensor
// velocity grid its maximum is attained at one of the four corners of the
// velocity box (which are grid points): only those are evaluated.
__global__ void k_dts(Dev d, double vx0, double vx1, double vy0, double vy1) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  double m = 0.0;
  for (int corner = 0; corner < 4; ++corner) {
    double vx = (corner & 1) ? vx1 : vx0, vy = (corner & 2) ? vy1 : vy0;
    double s = 0.0;
    for (int q = 0; q < 4; ++q) {
      int f = d.cell_faces[4 * c + q];
      double wS = vx * d.Sn[2 * f] + vy * d.Sn[2 * f + 1] - d.SUn[f];
      s += fmax(d.cell_sgn[4 * c + q] * wS, 0.0);
    }
    m = fmax(m, s);
  }
  d.dts[c] = d.cfl_s * d.vol_new[c] / m;
}

// Per-step geometry records in the arithmetic type: per face (S n, S U.n,
// U_f, vectors from the L image / R centres to the face centre), per cell
// the outward (S n, S U.n) of its four faces for the sweeps.
template <typename T> __global__ void k_geo_records(Dev d) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < d.nf) {
    int f = t, L = d.face_L[f], R = d.face_R[f];
    T *g = reinterpret_cast<T *>(d.fgeo) + (size_t)NFG * f;
    double sh = (double)d.face_shiftL[f];
    g[FG_SNX] = (T)d.Sn[2 * f];
    g[FG_SNY] = (T)d.Sn[2 * f + 1];
    g[FG_SUN] = (T)d.SUn[f];
    g[FG_UFX] = (T)d.Uf[2 * f];
    g[FG_UFY] = (T)d.Uf[2 * f + 1];
    g[FG_DXLX] = (T)(d.xf[2 * f] - (d.xc[2 * L] + sh * d.period[2 * L]));
    g[FG_DXLY] = (T)(d.xf[2 * f + 1] - (d.xc[2 * L + 1] + sh * d.period[2 * L + 1]));
    g[FG_DXRX] = R >= 0 ? (T)(d.xf[2 * f] - d.xc[2 * R]) : T(0);
    g[FG_DXRY] = R >= 0 ? (T)(d.xf[2 * f + 1] - d.xc[2 * R + 1]) : T(0);
  }
  if (t < d.nc) {
    int c = t;
    T *r = reinterpret_cast<T *>(d.srec) + (size_t)NSR * c;
    for (int s = 0; s < 4; ++s) {
      int f = d.cell_faces[4 * c + s];
      double sg = (double)d.cell_sgn[4 * c + s];
      r[3 * s] = (T)(0.5 * sg * d.Sn[2 * f]);
      r[3 * s + 1] = (T)(0.5 * sg * d.Sn[2 * f + 1]);
      r[3 * s + 2] = (T)(0.5 * sg * d.SUn[f]);
    }
  }
}

// Slope case and inverse Jacobian per cell (reading R1); depends on the
// geometry and on which neighbours are holes.
__global__ void k_slope_geo(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  double g[2][2];
  int flags = 0;
  double xcx = d.xc[2 * c], xcy = d.xc[2 * c + 1];
  for (int dir = 0; dir < 2; ++dir) {
    bool has[2];
    double px[2], py[2];
    for (int side = 0; side < 2; ++side) {
      int s = 2 * dir + side;
      int kind = d.nb_kind[4 * c + s], id = d.nb_id[4 * c + s];
      has[side] = false;
      px[side] = py[side] = 0.0;
      if (kind == NB_CELL) {
        double sh = (double)d.nb_shift[4 * c + s];
        px[side] = d.xc[2 * id] + sh * d.period[2 * c];
        py[side] = d.xc[2 * id + 1] + sh * d.period[2 * c + 1];
        has[side] = d.status[id] != ST_HOLE;
      } else if (kind == NB_GHOST) {
        double nx = d.nrm[2 * id], ny = d.nrm[2 * id + 1];
        double dd = (d.xf[2 * id] - xcx) * nx + (d.xf[2 * id + 1] - xcy) * ny;
        px[side] = xcx + 2.0 * dd * nx;
        py[side] = xcy + 2.0 * dd * ny;
        has[side] = true;
      }
    }
    int cs;
    if (has[0] && has[1]) {
      cs = SL_BOTH;
      g[dir][0] = 0.5 * (px[1] - px[0]);
      g[dir][1] = 0.5 * (py[1] - py[0]);
    } else if (has[1]) {
      cs = SL_P;
      g[dir][0] = px[1] - xcx;
      g[dir][1] = py[1] - xcy;
    } else if (has[0]) {
      cs = SL_M;
      g[dir][0] = xcx - px[0];
      g[dir][1] = xcy - py[0];
    } else {
      cs = SL_NONE;
      int fm = d.cell_faces[4 * c + 2 * dir], fp = d.cell_faces[4 * c + 2 * dir + 1];
      g[dir][0] = d.xf[2 * fp] - d.xf[2 * fm];
      g[dir][1] = d.xf[2 * fp + 1] - d.xf[2 * fm + 1];
    }
    flags |= cs << (2 * dir);
  }
  double a11 = g[0][0], a12 = g[0][1], a21 = g[1][0], a22 = g[1][1];
  double det = a11 * a22 - a12 * a21;
  d.slope_flags[c] = flags;
  // sweep mask: bit 0 solved cell, bit 1+s: neighbour across face slot s is solved
  int mask = d.status[c] == ST_FIELD ? 1 : 0;
  for (int s = 0; s < 4; ++s) {
    int f = d.cell_faces[4 * c + s];
    int nb = d.cell_sgn[4 * c + s] > 0 ? d.face_R[f] : d.face_L[f];
    if (nb >= 0 && d.status[nb] == ST_FIELD) mask |= 2 << s;
  }
  d.cmask[c] = mask;
  d.jinv[4 * c + 0] = a22 / det;
  d.jinv[4 * c + 1] = -a12 / det;
  d.jinv[4 * c + 2] = -a21 / det;
  d.jinv[4 * c + 3] = a11 / det;
  d.jinvf[c] = make_float4((float)d.jinv[4 * c + 0], (float)d.jinv[4 * c + 1], (float)d.jinv[4 * c + 2],
                           (float)d.jinv[4 * c + 3]);
}

// Ghost states of far-field / outflow faces (reading R6).
__global__ void k_ghost(Dev d) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.nf) return;
  int kind = d.face_kind[f];
  for (int m = 0; m < 4; ++m) {
    double v = 0.0;
    if (kind == BC_FARFIELD) v = d.Winf[m];
    else if (kind == BC_OUTFLOW) v = d.W[4 * d.face_L[f] + m];
    d.ghostW[4 * f + m] = v;
  }
}

// Limited gradient of the conservative W per cell (reading R1).
__global__ void k_gradW(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  int fl = d.slope_flags[c];
  const double *J = d.jinv + 4 * c;
  for (int m = 0; m < 4; ++m) {
    double wc = d.W[4 * c + m];
    double s[2];
    for (int dir = 0; dir < 2; ++dir) {
      int cs = (fl >> (2 * dir)) & 3;
      double val[2] = {0.0, 0.0};
      for (int side = 0; side < 2; ++side) {
        int sl = 2 * dir + side;
        int kind = d.nb_kind[4 * c + sl], id = d.nb_id[4 * c + sl];
        if (kind == NB_CELL) val[side] = d.W[4 * id + m];
        else if (kind == NB_GHOST) val[side] = d.ghostW[4 * id + m];
      }
      double r = 0.0;
      if (cs == SL_BOTH) r = vanleer<double>(wc - val[0], val[1] - wc);
      else if (cs == SL_P) r = val[1] - wc;
      else if (cs == SL_M) r = wc - val[0];
      s[dir] = r;
    }
    d.gradW[8 * c + 2 * m] = J[0] * s[0] + J[1] * s[1];
    d.gradW[8 * c + 2 * m + 1] = J[2] * s[0] + J[3] * s[1];
  }
}

__device__ __forceinline__ bool face_needed(const Dev &d, int f) {
  int L = d.face_L[f], R = d.face_R[f];
  return d.status[L] == ST_FIELD || (R >= 0 && d.status[R] == ST_FIELD);
}

__device__ __forceinline__ double spectral_radius(const double *Wf, double nx, double ny, double un,
                                                  int Keff) {
  Prim p = primitive(Wf, Keff);
  double pr = p.rho / (2.0 * p.lam);
  double gamma = (4.0 + Keff) / (2.0 + Keff);
  return fabs(p.ux * nx + p.uy * ny - un) + sqrt(gamma * pr / p.rho);
}

// Face coefficients, scalar part (one thread per face): g0 parameters and
// slopes (reading R2), time integrals over dts (Eq. fullSolution averaged as
// in Sec. 2.2), wall temperature parameter.
template <typename T> __global__ void k_face_scalar(Dev d) {
  int fid = blockIdx.x * blockDim.x + threadIdx.x;
  if (fid >= d.nf) return;
  int kind = d.face_kind[fid];
  if (!face_needed(d, fid) || kind == BC_OVERSET) return;
  double *P = d.fpar + (size_t)NFP * fid;
  T *PT = reinterpret_cast<T *>(d.fparT) + (size_t)NFP * fid;
  int L = d.face_L[fid], R = d.face_R[fid];
  bool wall = kind == BC_WALL;
  double W0[4], gx[4], gy[4], q0x, q0y, dts;
  double ufx = d.Uf[2 * fid], ufy = d.Uf[2 * fid + 1];
  double nx = d.nrm[2 * fid], ny = d.nrm[2 * fid + 1];
  const double *fs = d.fsum + NFS * fid;
  if (wall) {
    double dx = d.xf[2 * fid] - d.xc[2 * L], dy = d.xf[2 * fid + 1] - d.xc[2 * L + 1];
    for (int m = 0; m < 4; ++m) {
      gx[m] = d.gradW[8 * L + 2 * m];
      gy[m] = d.gradW[8 * L + 2 * m + 1];
      W0[m] = d.W[4 * L + m] + (dx * gx[m] + dy * gy[m]);
    }
    q0x = d.q[2 * L];
    q0y = d.q[2 * L + 1];
    dts = d.dts[L];
  } else {
    double sh = (double)d.face_shiftL[fid];
    double xLx = d.xc[2 * L] + sh * d.period[2 * L], xLy = d.xc[2 * L + 1] + sh * d.period[2 * L + 1];
    double xRx, xRy, WL[4], WR[4], dL[8], dR[8];
    for (int m = 0; m < 4; ++m) WL[m] = d.W[4 * L + m];
    for (int m = 0; m < 8; ++m) dL[m] = d.gradW[8 * L + m];
    if (R >= 0) {
      xRx = d.xc[2 * R];
      xRy = d.xc[2 * R + 1];
      for (int m = 0; m < 4; ++m) WR[m] = d.W[4 * R + m];
      for (int m = 0; m < 8; ++m) dR[m] = d.gradW[8 * R + m];
      q0x = 0.5 * (d.q[2 * L] + d.q[2 * R]);
      q0y = 0.5 * (d.q[2 * L + 1] + d.q[2 * R + 1]);
      dts = fmin(d.dts[L], d.dts[R]);
    } else {
      double dd = (d.xf[2 * fid] - xLx) * nx + (d.xf[2 * fid + 1] - xLy) * ny;
      xRx = xLx + 2.0 * dd * nx;
      xRy = xLy + 2.0 * dd * ny;
      for (int m = 0; m < 4; ++m) WR[m] = d.ghostW[4 * fid + m];
      for (int m = 0; m < 8; ++m) dR[m] = 0.0;
      q0x = 0.5 * d.q[2 * L];
      q0y = 0.5 * d.q[2 * L + 1];
      dts = d.dts[L];
    }
    double tx = xRx - xLx, ty = xRy - xLy, it2 = 1.0 / (tx * tx + ty * ty);
    double ex = tx * it2, ey = ty * it2;
    for (int m = 0; m < 4; ++m) {
      W0[m] = fs[FS_W0 + m];
      double avx = 0.5 * (dL[2 * m] + dR[2 * m]), avy = 0.5 * (dL[2 * m + 1] + dR[2 * m + 1]);
      double jump = (WR[m] - WL[m]) - (avx * tx + avy * ty);
      gx[m] = avx + jump * ex;
      gy[m] = avy + jump * ey;
    }
  }
  // face state, slopes, collision time and time integrals in FP64 on every
  // path (per face, not per velocity); the mixed path rounds the finished
  // record once to FP32 for its velocity loops
  typedef double RT;
  RT W0r[4], gxr[4], gyr[4];
  for (int m = 0; m < 4; ++m) { W0r[m] = (RT)W0[m]; gxr[m] = (RT)gx[m]; gyr[m] = (RT)gy[m]; }
  PrimR<RT> p0 = primitive_r<RT>(W0r, d.Keff);
  const SlopeInv<RT> inv = slope_inv<RT>(p0, d.Keff);
  RT ax[4], ay[4], At[4];
  micro_slope_r<RT>(p0, d.Keff, inv, gxr, ax);
  micro_slope_r<RT>(p0, d.Keff, inv, gyr, ay);
  time_slope_r<RT>(p0, d.Keff, inv, ax, ay, gxr, gyr, (RT)ufx, (RT)ufy, At);
  RT tau = collision_time_r<RT>(p0.rho, p0.lam, (RT)d.mu_ref, (RT)d.omega);
  RT dtsr = (RT)dts;
  RT qi[5];
  time_integrals_r<RT>(dtsr, tau, qi);
  RT par[NFP];
  for (int m = 0; m < NFP; ++m) par[m] = RT(0);
  par[FP_RHO] = p0.rho; par[FP_UX] = p0.ux; par[FP_UY] = p0.uy; par[FP_LAM] = p0.lam;
  par[FP_QX] = (RT)q0x; par[FP_QY] = (RT)q0y;
  for (int m = 0; m < 4; ++m) { par[FP_AX + m] = ax[m]; par[FP_AY + m] = ay[m]; par[FP_AT + m] = At[m]; }
  const RT idts = RT(1) / dtsr;
  for (int m = 0; m < 5; ++m) par[FP_Q1 + m] = qi[m] * idts;
  par[FP_UFX] = (RT)ufx; par[FP_UFY] = (RT)ufy;
  par[FP_PREF] = RT(0.8) * (RT(1) - (RT)d.Pr) * p0.lam * p0.lam * inv.irho;
  par[FP_HPRE] = p0.rho * p0.lam * RT(M_1_PI);
  par[FP_IL] = inv.il;
  par[FP_EH] = RT(0.5) * RT(d.Keff) * par[FP_IL];
  par[FP_EB] = RT(0.5) * (RT(d.Keff) + RT(2)) * par[FP_IL];
  par[FP_LAMW] = wall ? (RT)(1.0 / (2.0 * d.face_Tw[fid])) : RT(0);
  par[FP_RHOW] = RT(0);
  par[FP_SNX] = (RT)d.Sn[2 * fid];
  par[FP_SNY] = (RT)d.Sn[2 * fid + 1];
  par[FP_SUN] = (RT)d.SUn[fid];
  {
    double sh = (double)d.face_shiftL[fid];
    par[FP_DXLX] = (RT)(d.xf[2 * fid] - (d.xc[2 * L] + sh * d.period[2 * L]));
    par[FP_DXLY] = (RT)(d.xf[2 * fid + 1] - (d.xc[2 * L + 1] + sh * d.period[2 * L + 1]));
    par[FP_DXRX] = (R >= 0) ? (RT)(d.xf[2 * fid] - d.xc[2 * R]) : RT(0);
    par[FP_DXRY] = (R >= 0) ? (RT)(d.xf[2 * fid + 1] - d.xc[2 * R + 1]) : RT(0);
  }
  for (int m = 0; m < NFP; ++m) { P[m] = par[m]; PT[m] = (T)par[m]; }
  // Gamma from the mean of the two cells' W (boundary: the cell)
  RT Wf[4];
  for (int m = 0; m < 4; ++m)
    Wf[m] = (R >= 0) ? RT(0.5) * ((RT)d.W[4 * L + m] + (RT)d.W[4 * R + m]) : (RT)d.W[4 * L + m];
  PrimR<RT> pf = primitive_r<RT>(Wf, d.Keff);
  RT pr = pf.rho / (RT(2) * pf.lam);
  RT gamma = (RT(4) + RT(d.Keff)) / (RT(2) + RT(d.Keff));
  RT un = (RT)d.SUn[fid] / (RT)d.S[fid];
  d.gam[fid] = fabs(pf.ux * nx + pf.uy * ny - un) + sqrt(gamma * pr / pf.rho);
}

// Face coefficients, velocity part (one warp per face): the g-part of the
// macro flux by a sum over the discrete velocities, the wall density rho_w
// (Eq. maxWalldes) and the total S-weighted macro flux (Eq. macroscopicFlux).
// Equilibrium part of the macro flux of an interior face (the velocity sum
// of w wS Psi (q3 (g + g+) + q4 g (a.w Psi) + q5 g (A Psi)) in reduced form,
// Eqs. fullSolution / macroscopicFlux) through the tensor structure of the
// velocity grid: every term is g = HPRE Ex(cx) Ey(cy) (c = v - U0) times a
// polynomial of degree <= 6 in (cx, cy), so the 2D sum is exactly (up to
// rounding) sum_ab coef_ab Mx_a My_b with the 1D moments
// Mx_a = sum_ix wx cx^a Ex(cx), My_b likewise: O(nvx + nvy) work per face
// instead of O(nvx nvy).  One warp per face; out (all lanes): 4 sums.
// 1D grids of the separable sums in the arithmetic type
template <typename R> struct Grid1;
template <> struct Grid1<float> {
  __device__ static float vx(const Dev &d, int i) { return d.vxf[i]; }
  __device__ static float vy(const Dev &d, int i) { return d.vy1f[i]; }
  __device__ static float wx(const Dev &d, int i) { return d.wx1f[i]; }
  __device__ static float wy(const Dev &d, int i) { return d.wy1f[i]; }
  __device__ static float ex(float x) { return __expf(x); }
};
template <> struct Grid1<double> {
  __device__ static double vx(const Dev &d, int i) { return d.vx1[i]; }
  __device__ static double vy(const Dev &d, int i) { return d.vy1[i]; }
  __device__ static double wx(const Dev &d, int i) { return d.wx1[i]; }
  __device__ static double wy(const Dev &d, int i) { return d.wy1[i]; }
  __device__ static double ex(double x) { return exp(x); }
};

template <typename R, int GS>
__device__ __forceinline__ void face_eq_flux_separable(const Dev &d, const R *P, R snx, R sny, R sun, int lane,
                                                       R out[4]) {
  typedef Grid1<R> G;
  R ux = P[FP_UX], uy = P[FP_UY], lam = P[FP_LAM];
  // 1D moments: lane of the face's GS-lane group = grid index, a = 0..6 (x)
  // and b = 0..6 (y); every lane of the warp takes part in the shuffles
  R mx[7], my[7];
#pragma unroll
  for (int a = 0; a < 7; ++a) { mx[a] = R(0); my[a] = R(0); }
  for (int ix = lane; ix < d.nvx; ix += GS) {
    R cx = G::vx(d, ix) - ux;
    R e = G::wx(d, ix) * G::ex(-lam * cx * cx), p = e;
#pragma unroll
    for (int a = 0; a < 7; ++a) { mx[a] += p; p *= cx; }
  }
  for (int iy = lane; iy < d.nvy; iy += GS) {     // the whole grid (also when sharded)
    R cy = G::vy(d, iy) - uy;
    R e = G::wy(d, iy) * G::ex(-lam * cy * cy), p = e;
#pragma unroll
    for (int a = 0; a < 7; ++a) { my[a] += p; p *= cy; }
  }
#pragma unroll
  for (int o = GS / 2; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      mx[a] += __shfl_xor_sync(0xffffffffu, mx[a], o);
      my[a] += __shfl_xor_sync(0xffffffffu, my[a], o);
    }
  Poly2<3, R> ih, ib;
  interface_polys<R>(P, (R)d.Keff, (R)d.Kint, ih, ib);
  Poly2<1, R> vxp = p2_lin<R>(ux, R(1), R(0)), vyp = p2_lin<R>(uy, R(0), R(1));
  Poly2<2, R> v2 = p2_axpby(R(1), p2_mul(vxp, vxp), R(1), p2_mul(vyp, vyp));
  Poly2<1, R> ws = p2_lin<R>(snx * ux + sny * uy - sun, snx, sny);
  Poly2<4, R> m0 = p2_mul(ws, ih);
  R hpre = P[FP_HPRE];
  out[0] = hpre * p2_sum(m0, mx, my);
  out[1] = hpre * p2_sum(p2_mul(m0, vxp), mx, my);
  out[2] = hpre * p2_sum(p2_mul(m0, vyp), mx, my);
  Poly2<5, R> e3 = p2_axpby(R(0.5), ib, R(0.5), p2_mul(v2, ih));
  out[3] = hpre * p2_sum(p2_mul(ws, e3), mx, my);
}

// Velocity-loop face coefficients for the faces of `list` (all faces when
// null): FCW warps per face split the velocities, their warp totals meet in
// shared memory (summed in warp order).  The FP32 path runs it over the wall
// faces only.
constexpr int FCW = 4;
template <typename T> __global__ void __launch_bounds__(256, 2) k_face_coef(Dev d, const int *list, int n) {
  __shared__ double part[256 / 32][9];
  int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int w = wg / FCW, sub = wg - (wg / FCW) * FCW;
  int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  bool in = w < n;
  int fid = in ? (list ? list[w] : w) : 0;
  int kind = in ? d.face_kind[fid] : BC_OVERSET;
  bool act = in && kind != BC_OVERSET && face_needed(d, fid);
  if (in && !act && sub == 0) {
    if (lane < 4) d.fflux[4 * fid + lane] = 0.0;
    if (lane == 0) d.gam[fid] = 0.0;
  }
  bool wall = kind == BC_WALL;
  Acc<T> ags[4], ars[4], aden;
  if (act) {
    T *PT = reinterpret_cast<T *>(d.fparT) + (size_t)NFP * fid;
    __align__(16) T parT[NFP];
    load_rec<T, NFP>(PT, parT);
    T snx, sny, sun;
    if (sizeof(T) == 4) { snx = parT[FP_SNX]; sny = parT[FP_SNY]; sun = parT[FP_SUN]; }
    else { snx = (T)d.Sn[2 * fid]; sny = (T)d.Sn[2 * fid + 1]; sun = (T)d.SUn[fid]; }
    T tufx = parT[FP_UFX], tufy = parT[FP_UFY], tlamw = parT[FP_LAMW], tK = (T)d.Keff;
    V2<T> zero = {T(0), T(0)};
    // the equilibrium and reflected parts depend on no f: the whole grid
    // (also on a sharded context, so every shard gets the same totals)
    for (int k = sub * 32 + lane; k < d.nv_all; k += 32 * FCW) {
      T vx = dvxa<T>(d, k), vy = dvya<T>(d, k), w = dwa<T>(d, k);
      T wS = vx * snx + vy * sny - sun;
      T v2 = T(0.5) * (vx * vx + vy * vy);
      T cw = w * wS;
      if (!wall || wS > T(0)) {
        V2<T> I = interface_integral<T>(parT, vx, vy, zero, zero, tK, (T)d.Kint, (T)d.Pr);
        ags[0].add(cw * I.h); ags[1].add(cw * vx * I.h); ags[2].add(cw * vy * I.h);
        ags[3].add(cw * (v2 * I.h + T(0.5) * I.b));
      } else {
        T cx = vx - tufx, cy = vy - tufy;
        T Hw = (tlamw * T(M_1_PI)) * r_exp<T>(-tlamw * (cx * cx + cy * cy));
        T Bw = tK / (T(2) * tlamw) * Hw;
        aden.add(cw * Hw);
        ars[0].add(cw * Hw); ars[1].add(cw * vx * Hw); ars[2].add(cw * vy * Hw);
        ars[3].add(cw * (v2 * Hw + T(0.5) * Bw));
      }
    }
  }
  double tot[9];
  for (int m = 0; m < 4; ++m) { tot[m] = to_double(warp_total(ags[m])); tot[4 + m] = to_double(warp_total(ars[m])); }
  tot[8] = to_double(warp_total(aden));
  if (lane == 0)
    for (int m = 0; m < 9; ++m) part[wl][m] = tot[m];
  __syncthreads();
  if (act && sub == 0 && lane == 0) {
    double acc[9];
    for (int m = 0; m < 9; ++m) {
      acc[m] = part[wl][m];
      for (int j = 1; j < FCW; ++j) acc[m] += part[wl + j][m];
    }
    double *P = d.fpar + (size_t)NFP * fid;
    T *PT = reinterpret_cast<T *>(d.fparT) + (size_t)NFP * fid;
    const double *fs = d.fsum + NFS * fid;
    double F[4];
    for (int m = 0; m < 4; ++m)
      F[m] = P[FP_Q1] * fs[FS_FF + m] + P[FP_Q2] * fs[FS_WG + m] + acc[m];
    if (wall) {
      double rhow = -F[0] / acc[8];
      P[FP_RHOW] = rhow;
      PT[FP_RHOW] = (T)rhow;
      for (int m = 0; m < 4; ++m) F[m] += rhow * acc[4 + m];
    }
    {
      __align__(16) T pr[NFP];
      load_rec<T, NFP>(PT, pr);
      Poly2<3, T> ih, ib;
      interface_polys<T>(pr, (T)d.Keff, (T)d.Kint, ih, ib);
      store_polys<T>(PT, ih, ib);
    }
    for (int m = 0; m < 4; ++m) d.fflux[4 * fid + m] = F[m];
  }
}

// Face coefficients of the non-wall faces: FCG lanes per face, the
// equilibrium part of the macro flux from 1D velocity moments (exact
// separable rewrite of the tensor-grid sum); faces outside the field get
// zero flux.
constexpr int FCG = 8;
template <typename T> __global__ void __launch_bounds__(256) k_face_coef_sep(Dev d) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int fid = t / FCG, sub = t % FCG;
  bool in = fid < d.nf;
  int kind = in ? d.face_kind[fid] : BC_OVERSET;
  bool need = in && kind != BC_OVERSET && face_needed(d, fid);
  if (in && !need) {
    if (sub < 4) d.fflux[4 * fid + sub] = 0.0;
    if (sub == 0) d.gam[fid] = 0.0;
  }
  bool act = need && kind != BC_WALL;
  if (!__any_sync(0xffffffffu, act)) return;      // warp-uniform
  __align__(16) T parT[NFP];
  if (act) {
    load_rec<T, NFP>(reinterpret_cast<const T *>(d.fparT) + (size_t)NFP * fid, parT);
  } else {
#pragma unroll
    for (int q = 0; q < NFP; ++q) parT[q] = T(0);
  }
  T o[4];
  face_eq_flux_separable<T, FCG>(d, parT, parT[FP_SNX], parT[FP_SNY], parT[FP_SUN], sub, o);
  if (act) {
    // the cubics of the interface distribution for the flux pass (lane sub
    // of the face's group writes coefficients sub, sub + FCG, ...)
    Poly2<3, T> ih, ib;
    interface_polys<T>(parT, (T)d.Keff, (T)d.Kint, ih, ib);
    T *PT = reinterpret_cast<T *>(d.fparT) + (size_t)NFP * fid;
#pragma unroll
    for (int m = 0; m < 20; ++m)
      if (m % FCG == sub) PT[FP_IH + m] = m < 10 ? ih.c[m] : ib.c[m - 10];
  }
  if (act && sub < 4) {                           // lane m of the group: component m
    const double *P = d.fpar + (size_t)NFP * fid;
    const double *fs = d.fsum + NFS * fid;
    T om = sub == 0 ? o[0] : sub == 1 ? o[1] : sub == 2 ? o[2] : o[3];
    d.fflux[4 * fid + sub] = P[FP_Q1] * fs[FS_FF + sub] + P[FP_Q2] * fs[FS_WG + sub] + to_double(om);
  }
}

// Per-cell sum of the S-weighted macro fluxes (Eq. macroscopicFlux summed
// over the faces); with level_n also the extensive level-n macro term
// TW = Omega^n W^n / dt - F^n / 2 (reading R4).
__global__ void k_cell_macro(Dev d, int level_n) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  double F[4] = {0, 0, 0, 0};
  for (int s = 0; s < 4; ++s) {
    int f = d.cell_faces[4 * c + s];
    double sg = (double)d.cell_sgn[4 * c + s];
    for (int m = 0; m < 4; ++m) F[m] += sg * d.fflux[4 * f + m];
  }
  for (int m = 0; m < 4; ++m) d.Fc[4 * c + m] = F[m];
  if (level_n)
    for (int m = 0; m < 4; ++m) d.TW[4 * c + m] = d.vol_old[c] / d.stepc[0] * d.W[4 * c + m] - 0.5 * F[m];
}

// Cell parameter record (prim, q, 1/tau) from W and q, and its Shakhov
// record in the arithmetic type (level n).
template <typename T> __global__ void k_cell_params(Dev d, const double *Wsrc, double *out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  Prim p = primitive(Wsrc + 4 * c, d.Keff);
  double *o = out + NCP * c;
  o[CP_RHO] = p.rho; o[CP_UX] = p.ux; o[CP_UY] = p.uy; o[CP_LAM] = p.lam;
  o[CP_QX] = d.q[2 * c]; o[CP_QY] = d.q[2 * c + 1];
  o[CP_ITAU] = 1.0 / collision_time(p.rho, p.lam, d.mu_ref, d.omega);
  o[CP_DBASE] = 0.0;
  write_shrec<T>(d, o, d.vol_old[c], reinterpret_cast<T *>(d.shn) + (size_t)NSH * c);
}

// ----------------------------------------------------- macro LU-SGS sweep
// Per-cell record of the macro sweep (gathered in parallel before it):
// R (4), 1/diag, then per face slot: neighbour W (4), outward normal (2),
// U.n, S/4, Gamma.
enum { MR_R = 0, MR_IDIAG = 4, MR_SLOT = 5, MR_SW = 9 };

// (1/4) S (dF_E,j - Gamma dW_j) across one face slot of the record.  FP64:
// the difference F_E(W + dW) - F_E(W) evaluated directly.  FP32 (mixed
// path): the same difference rewritten exactly in terms of dW (every term is
// O(dW)), so no cancellation occurs when dW << W.
// Off-diagonal coupling (1/4 S)(Delta F_E . n - Gamma dW) of a neighbour
// with state W (slot record r: W (4), n (2), U.n, S/4, Gamma) and increment
// dW, the flux variation written out as a difference (one division, no
// cancellation between the two fluxes): with d(ab/rho) = (da b rho + a db
// rho + da db rho - a b drho) / (rho (rho + drho)) and p = (gamma-1)(E -
// |m|^2/(2 rho)).
__device__ __forceinline__ void macro_off(const double *r, const double *dW, int Keff, double out[4]) {
  const double rho = r[0], m1 = r[1], m2 = r[2], E = r[3], nx = r[4], ny = r[5], un = r[6];
  const double dr = dW[0], d1 = dW[1], d2 = dW[2], dE = dW[3];
  const double g1 = 2.0 / (2.0 + (double)Keff);          // gamma - 1
  const double mn = m1 * nx + m2 * ny, dmn = d1 * nx + d2 * ny;
  const double den = 1.0 / (rho * (rho + dr));
  const double dq11 = (2.0 * (m1 * d1 + m2 * d2) * rho + (d1 * d1 + d2 * d2) * rho - (m1 * m1 + m2 * m2) * dr) * den;
  const double dp = g1 * (dE - 0.5 * dq11);
  const double p = g1 * (E - 0.5 * (m1 * m1 + m2 * m2) * ((rho + dr) * den));
  const double dv = (dmn * rho - mn * dr) * den;
  const double dF0 = dmn - dr * un;
  const double dF1 = (d1 * mn * rho + m1 * dmn * rho + d1 * dmn * rho - m1 * mn * dr) * den - d1 * un + dp * nx;
  const double dF2 = (d2 * mn * rho + m2 * dmn * rho + d2 * dmn * rho - m2 * mn * dr) * den - d2 * un + dp * ny;
  const double dF3 = (dE * mn * rho + E * dmn * rho + dE * dmn * rho - E * mn * dr) * den - dE * un +
                     dp * (mn + dmn) * (rho * den) + p * dv;
  const double q = r[7], g = r[8];
  out[0] = q * (dF0 - g * dr);
  out[1] = q * (dF1 - g * d1);
  out[2] = q * (dF2 - g * d2);
  out[3] = q * (dF3 - g * dE);
}

__device__ __forceinline__ void macro_off(const float *rr, const float *dWn, int Keff, float out[4]) {
  float4 s0 = reinterpret_cast<const float4 *>(rr)[0], s1 = reinterpret_cast<const float4 *>(rr)[1];
  float gam = rr[8];
  float4 dw = *reinterpret_cast<const float4 *>(dWn);
  float r = s0.x, m1 = s0.y, m2 = s0.z, E = s0.w;
  float nx = s1.x, ny = s1.y, un = s1.z;
  float dr = dw.x, d1 = dw.y, d2 = dw.z, dE = dw.w;
  float g1 = __fdividef(2.0f, 2.0f + (float)Keff);    // gamma - 1
  float mn = m1 * nx + m2 * ny, dmn = d1 * nx + d2 * ny;
  float den = __fdividef(1.0f, r * (r + dr));          // 1/(rho (rho + drho))
  // d(a b / rho) = [da b rho + a db rho + da db rho - a b drho] / (rho (rho + drho))
  float dq11 = (2.0f * (m1 * d1 + m2 * d2) * r + (d1 * d1 + d2 * d2) * r -
                (m1 * m1 + m2 * m2) * dr) * den;
  float dp = g1 * (dE - 0.5f * dq11);
  float p = g1 * (E - 0.5f * (m1 * m1 + m2 * m2) * ((r + dr) * den));
  float dv = (dmn * r - mn * dr) * den;               // d(mn / rho)
  float dF0 = dmn - dr * un;
  float dF1 = (d1 * mn * r + m1 * dmn * r + d1 * dmn * r - m1 * mn * dr) * den - d1 * un + dp * nx;
  float dF2 = (d2 * mn * r + m2 * dmn * r + d2 * dmn * r - m2 * mn * dr) * den - d2 * un + dp * ny;
  float dF3 = (dE * mn * r + E * dmn * r + dE * dmn * r - E * mn * dr) * den - dE * un +
              dp * (mn + dmn) * (r * den) + p * dv;
  float q = s1.w, g = gam;
  out[0] = q * (dF0 - g * dr);
  out[1] = q * (dF1 - g * d1);
  out[2] = q * (dF2 - g * d2);
  out[3] = q * (dF3 - g * dE);
}

// Gather the sweep record of every solved cell (parallel).  The FP64 record
// is the packed layout above.  The FP32 record (64 floats, 256 bytes) keeps
// every group 16-byte aligned for 128-bit shared-memory reads: R (4), 1/diag,
// the neighbour mask, then per face slot 12 values (neighbour W (4); normal
// (2), U.n, S/4; Gamma, 3 unused) and the increment of the sweep (4).
enum { M32_R = 0, M32_IDIAG = 4, M32_MASK = 5, M32_SLOT = 8, M32_SW = 12, M32_DWS = 56 };
template <typename MT> struct MacroRec;
template <> struct MacroRec<double> {
  static constexpr int R = MR_R, IDIAG = MR_IDIAG, SLOT = MR_SLOT, SW = MR_SW, STRIDE = NMR;
};
template <> struct MacroRec<float> {
  static constexpr int R = M32_R, IDIAG = M32_IDIAG, SLOT = M32_SLOT, SW = M32_SW, STRIDE = NMR32;
};

// FP32 records are diagonal-major per block: the record of cell (i, j) of
// block b is number mrec_off[b] + (i + j) nj + j, so the records of one
// diagonal are contiguous and a sweep step fetches them with one bulk copy.
__device__ __forceinline__ size_t mrec32_index(const Dev &d, int c) {
  int b = d.cell_block[c];
  int ni = d.blk_info[8 * b], nj = d.blk_info[8 * b + 1];
  int loc = c - d.cell_off[b];
  int i = loc % ni, j = loc / ni;
  return (size_t)d.mrec_off[b] + (size_t)(i + j) * nj + j;
}

template <typename MT> __global__ void k_macro_prep(Dev d, MT *rec) {
  typedef MacroRec<MT> L;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  MT *o = rec + (size_t)L::STRIDE * (sizeof(MT) == 4 ? mrec32_index(d, c) : (size_t)c);
  int mask = d.cmask[c];
  if (sizeof(MT) == 4) o[M32_MASK] = __int_as_float(mask);
  if (!(mask & 1)) return;
  double vol = d.vol_new[c], idt = 1.0 / d.stepc[0];
  for (int m = 0; m < 4; ++m)
    o[L::R + m] = (MT)(d.TW[4 * c + m] - vol * idt * d.W[4 * c + m] - 0.5 * d.Fc[4 * c + m]);
  double diag = vol * (d.cfl_s / (d.cfl_pseudo * d.dts[c]) + idt);
  for (int s = 0; s < 4; ++s) {
    int f = d.cell_faces[4 * c + s];
    diag += 0.25 * d.S[f] * d.gam[f];
    double sg = (double)d.cell_sgn[4 * c + s];
    int nb = (sg > 0) ? d.face_R[f] : d.face_L[f];
    MT *q = o + L::SLOT + L::SW * s;
    // missing neighbour: a harmless positive state (its increment is zero)
    for (int m = 0; m < 4; ++m) q[m] = nb >= 0 ? (MT)d.W[4 * nb + m] : (m == 0 || m == 3 ? MT(1) : MT(0));
    q[4] = (MT)(sg * d.nrm[2 * f]);
    q[5] = (MT)(sg * d.nrm[2 * f + 1]);
    q[6] = (MT)(sg * d.SUn[f] / d.S[f]);
    q[7] = (MT)(0.25 * d.S[f]);
    q[8] = (MT)d.gam[f];
  }
  o[L::IDIAG] = (MT)(1.0 / diag);
}

// shared memory of the FP32 macro sweep ahead of its buffers: the mbarriers
// of the ring stages (floats)
constexpr int MACRO_SMEM_HEAD = 16;

// FP32 macro sweep: as k_macro_sweep below, with TPR threads per row (each
// evaluates the couplings of face slots s = sub, sub + TPR, ...; a shuffle
// within the row's lanes sums them).  The records of the next NS-1 diagonals
// are in flight in a ring in shared memory, one bulk copy per diagonal
// completing on the stage's mbarrier (bounded waits), and the part of the
// next record a thread uses is moved into registers before the barrier that
// ends a diagonal, so after the barrier only the coupling arithmetic remains.
// The forward increment is stored into the record for the backward pass.
// NS = 0: no ring, records read from global memory (blocks too tall for a
// two-stage ring).
__device__ __forceinline__ void macro_off_v(float4 s0, float4 s1, float gam, float4 dw, int Keff,
                                            float out[4]) {
  __align__(16) float rr[12] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w, gam, 0.f, 0.f, 0.f};
  __align__(16) float dv[4] = {dw.x, dw.y, dw.z, dw.w};
  macro_off(rr, dv, Keff, out);
}

// PM (with TPR = 2): the two threads of a row take the two face slots that
// couple in this pass -- forward the lower neighbours (slots 0 and 2),
// backward the upper ones (1 and 3) -- and the first thread also the
// periodic wrap slot (1 forward at i = n_i - 1, 0 backward at i = 0) where it
// applies; couplings that are not evaluated are exact zeros in the TPR = 4
// form, so the sums are the same.
template <int NS, int TPR, bool PM = false>
__global__ void __launch_bounds__(512) k_macro_sweep_f32(Dev d, float *rec) {
  static_assert(!PM || TPR == 2, "pass-dependent slots pair two threads a row");
  constexpr int NSL = PM ? 1 : 4 / TPR;         // face slots per thread (PM: plus the wrap)
  constexpr int NSR_ = NS > 0 ? NS : 1;
  extern __shared__ __align__(16) float smf[];
  unsigned long long *mb = reinterpret_cast<unsigned long long *>(smf);   // one mbarrier per stage
  int rows = blockDim.x / TPR;
  float *buf0 = smf + MACRO_SMEM_HEAD, *buf1 = buf0 + 4 * rows;
  float *ring = buf1 + 4 * rows;                 // NS * rows * NMR32
  int b = blockIdx.x;
  const int *bi = d.blk_info + 8 * b;
  int ni = bi[0], nj = bi[1], per = bi[2];
  const float *rb = rec + (size_t)NMR32 * d.mrec_off[b];          // this block's records
  float *rbw = rec + (size_t)NMR32 * d.mrec_off[b];
  int row = threadIdx.x / TPR, sub = threadIdx.x % TPR;
  unsigned rmask = (TPR == 1 ? 1u : (1u << TPR) - 1u) << (threadIdx.x & 31 & ~(TPR - 1));
  int nd = ni + nj - 1;
  if (NS > 0 && threadIdx.x == 0) {
    for (int s = 0; s < NSR_; ++s) mbar_init(&mb[s], 1);
    mbar_fence_init();
  }
  if (sub == 0)
    for (int m = 0; m < 4; ++m) { buf0[4 * row + m] = 0.f; buf1[4 * row + m] = 0.f; }
  __syncthreads();
  const unsigned diag_bytes = (unsigned)nj * NMR32 * sizeof(float);
  bool to = false;                   // this thread's bounded wait ran out
  int issued = -1, waited = -1;      // thread 0: last stage copied into / waited for
  for (int pass = 0; pass < 2; ++pass) {
    float4 prev = make_float4(0.f, 0.f, 0.f, 0.f), first = prev;
    // face slot of this thread's q-th coupling
    auto slot_of = [&](int q) {
      if (!PM) return q * TPR + sub;
      return sub == 0 ? (pass == 0 ? 0 : 1) : (pass == 0 ? 2 : 3);
    };
    // diagonal of step it, and its position in the ring (g = steps so far)
    auto diag_of = [&](int it) { return pass == 0 ? it : nd - 1 - it; };
    auto gstep = [&](int it) { return pass * nd + it; };
    // thread 0 fetches the records of a whole diagonal with one bulk copy
    auto issue = [&](int it) {
      if (NS == 0 || threadIdx.x != 0 || it >= nd) return;
      int s = gstep(it) % NSR_;
      fence_proxy_async_shared();
      mbar_arrive_expect_tx(&mb[s], diag_bytes);
      bulk_g2s(ring + (size_t)s * rows * NMR32, rb + (size_t)diag_of(it) * nj * NMR32, diag_bytes, &mb[s]);
      issued = gstep(it);
    };
    // a bounded wait; a thread that gives up marks `to`, and the CTA stops
    // at the end of the diagonal (uniform decision at the barrier)
    auto wait_stage = [&](int it) {
      if (NS == 0 || it >= nd) return;
      int g = gstep(it);
      if (!mbar_wait(&mb[g % NSR_], (unsigned)(g / NSR_) & 1u, d.err, d.wait_polls)) to = true;
      else if (threadIdx.x == 0) waited = g;
    };
    // registers of the next diagonal: mask, this thread's slot records,
    // R (pass 0) or the forward increment (pass 1), 1/diag
    int nmask = 0;
    float4 nsa[NSL], nsb[NSL], nrv = make_float4(0.f, 0.f, 0.f, 0.f);
    float ngam[NSL], nidg = 0.f;
    auto fetch = [&](int it) {
      nmask = 0;
      if (it >= nd) return;
      int t = diag_of(it), i = t - row;
      if (!(row < nj && i >= 0 && i < ni)) return;
      const float *r = NS > 0 ? ring + ((size_t)(gstep(it) % NSR_) * rows + row) * NMR32
                              : rb + ((size_t)t * nj + row) * NMR32;
      nmask = __float_as_int(r[M32_MASK]);
#pragma unroll
      for (int q = 0; q < NSL; ++q) {
        const float *sr = r + M32_SLOT + M32_SW * slot_of(q);
        nsa[q] = *reinterpret_cast<const float4 *>(sr);
        nsb[q] = *reinterpret_cast<const float4 *>(sr + 4);
        ngam[q] = sr[8];
      }
      nrv = *reinterpret_cast<const float4 *>(r + (pass == 0 ? M32_R : M32_DWS));
      nidg = r[M32_IDIAG];
    };
#pragma unroll
    for (int q = 0; q < NS - 1; ++q) issue(q);
    wait_stage(0);
    fetch(0);
    int cur = 0;
    for (int it = 0; it < nd; ++it) {
      issue(it + NS - 1);
      int t = diag_of(it);
      int i = t - row;
      bool act = row < nj && i >= 0 && i < ni;
      int mask = nmask;
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
      if (mask & 1) {
        const float *prv = cur ? buf0 : buf1;
        float acc[4] = {0, 0, 0, 0};
#pragma unroll
        for (int q = 0; q < NSL; ++q) {
          int s = slot_of(q);
          float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
          bool use = !PM;                        // PM: only the couplings of this pass
          if (mask & (2 << s)) {
            if (pass == 0) {
              if (s == 0 && i > 0) { dv = prev; use = true; }
              else if (s == 1 && per && i == ni - 1) { dv = first; use = true; }
              else if (s == 2 && row > 0) { dv = *reinterpret_cast<const float4 *>(prv + 4 * (row - 1)); use = true; }
            } else {
              if (s == 1 && i < ni - 1) { dv = prev; use = true; }
              else if (s == 0 && per && i == 0) { dv = first; use = true; }
              else if (s == 3 && row < nj - 1) { dv = *reinterpret_cast<const float4 *>(prv + 4 * (row + 1)); use = true; }
            }
          }
          if (use) {
            float o[4];
            macro_off_v(nsa[q], nsb[q], ngam[q], dv, d.Keff, o);
            // a plain (never contracted) sum: the same bits as the lanes'
            // shuffle sums of the four-slot form
            for (int m = 0; m < 4; ++m) acc[m] = __fadd_rn(acc[m], o[m]);
          }
        }
        // PM: the periodic wrap (slot 1 forward at i = n_i - 1, slot 0
        // backward at i = 0), rare: its record is read where it lies (the
        // ring stage of this step is not reissued before the next step)
        if (PM && sub == 0 && per && i == (pass == 0 ? ni - 1 : 0) && (mask & (2 << (pass == 0 ? 1 : 0)))) {
          const float *r = NS > 0 ? ring + ((size_t)(gstep(it) % NSR_) * rows + row) * NMR32
                                  : rb + ((size_t)t * nj + row) * NMR32;
          const float *sr = r + M32_SLOT + M32_SW * (pass == 0 ? 1 : 0);
          float o[4];
          macro_off_v(*reinterpret_cast<const float4 *>(sr), *reinterpret_cast<const float4 *>(sr + 4), sr[8],
                      first, d.Keff, o);
          for (int m = 0; m < 4; ++m) acc[m] = __fadd_rn(acc[m], o[m]);
        }
#pragma unroll
        for (int w = 1; w < TPR; w <<= 1)
          for (int m = 0; m < 4; ++m) acc[m] += __shfl_xor_sync(rmask, acc[m], w);
        float4 rv = nrv;
        float idg = nidg;
        if (pass == 0)
          val = make_float4((rv.x - acc[0]) * idg, (rv.y - acc[1]) * idg, (rv.z - acc[2]) * idg,
                            (rv.w - acc[3]) * idg);
        else
          val = make_float4(rv.x - acc[0] * idg, rv.y - acc[1] * idg, rv.z - acc[2] * idg,
                            rv.w - acc[3] * idg);
        // forward: the increment d* for the backward pass; backward: the
        // final increment for the post-processing kernel
        if (sub == 0) *reinterpret_cast<float4 *>(rbw + ((size_t)t * nj + row) * NMR32 + M32_DWS) = val;
      }
      if (act) {
        prev = val;
        if (i == (pass == 0 ? 0 : ni - 1)) first = val;
      }
      float *dst = cur ? buf1 : buf0;
      if (sub == 0) *reinterpret_cast<float4 *>(dst + 4 * row) = val;
      // the next diagonal's records, read into registers before the barrier
      wait_stage(it + 1);
      fetch(it + 1);
      if (__syncthreads_or(to)) break;
      cur ^= 1;
    }
    if (__syncthreads_or(to)) break;
    // the increments stored above are read by the next pass's bulk copies
    fence_proxy_async_global();
    __threadfence_block();
    if (sub == 0)
      for (int m = 0; m < 4; ++m) { buf0[4 * row + m] = 0.f; buf1[4 * row + m] = 0.f; }
    __syncthreads();
  }
  // after a timeout: no copy of this CTA may still be in flight when it
  // exits, so thread 0 waits (default bound) for every stage it issued and
  // nobody waited for; the results of the step are invalid (EF_TIMEOUT)
  if (NS > 0 && threadIdx.x == 0 && issued > waited)
    for (int g = waited + 1; g <= issued; ++g) mbar_wait(&mb[g % NSR_], (unsigned)(g / NSR_) & 1u, d.err);
}

// LU-SGS of Eq. dualTimeStepping_macro (Sec. 2.2), one CTA per block,
// thread = row j; diagonals i + j in increasing (forward) then decreasing
// (backward) order reproduce the lexicographic Gauss-Seidel exactly.  The
// record of the next diagonal's cell is loaded before the barrier, so a
// diagonal step costs the arithmetic of its lower/upper couplings only.
template <typename MT> __global__ void __launch_bounds__(512) k_macro_sweep(Dev d, const MT *rec) {
  extern __shared__ double sm[];
  MT *buf0 = reinterpret_cast<MT *>(sm), *buf1 = buf0 + 4 * blockDim.x;
  int b = blockIdx.x;
  const int *bi = d.blk_info + 8 * b;
  int ni = bi[0], nj = bi[1], per = bi[2];
  int off = d.cell_off[b];
  int row = threadIdx.x;
  MT prev[4] = {0, 0, 0, 0}, first[4] = {0, 0, 0, 0};
  int nd = ni + nj - 1;
  for (int m = 0; m < 4; ++m) { buf0[4 * row + m] = 0; buf1[4 * row + m] = 0; }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    int cur = 0;
    // registers holding the record of the cell this thread handles next
    MT r[NMR];
    MT dws[4] = {0, 0, 0, 0};
    int mask = 0;
    auto load = [&](int it) {
      int step = pass == 0 ? it : nd - 1 - it;
      int i = step - row;
      mask = 0;
      if (it < nd && row < nj && i >= 0 && i < ni) {
        int c = off + row * ni + i;
        mask = d.cmask[c];
        if (mask & 1) {
          const MT *src = rec + (size_t)NMR * c;
#pragma unroll
          for (int m = 0; m < NMR; ++m) r[m] = src[m];
          if (pass == 1)
            for (int m = 0; m < 4; ++m) dws[m] = (MT)d.dW[4 * c + m];
        }
      }
    };
    // FP32: the next diagonal's record is loaded before the barrier; FP64
    // (reference path) loads at the start of the step to bound registers
    constexpr bool PF = sizeof(MT) == 4;
    if (PF) load(0);
    for (int it = 0; it < nd; ++it) {
      if (!PF) load(it);
      int step = pass == 0 ? it : nd - 1 - it;
      int i = step - row;
      bool act = row < nj && i >= 0 && i < ni;
      MT val[4] = {0, 0, 0, 0};
      if (act && (mask & 1)) {
        int c = off + row * ni + i;
        MT acc[4];
        if (pass == 0) for (int m = 0; m < 4; ++m) acc[m] = r[MR_R + m];
        else for (int m = 0; m < 4; ++m) acc[m] = 0;
        MT *prv = cur ? buf0 : buf1;
        const MT zero4[4] = {0, 0, 0, 0};
        MT o[4][4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const MT *dv = zero4;
          if (mask & (2 << s)) {
            if (pass == 0) {          // lower: i-1, wrap ni-1 -> 0, j-1
              if (s == 0 && i > 0) dv = prev;
              else if (s == 1 && per && i == ni - 1) dv = first;
              else if (s == 2 && row > 0) dv = prv + 4 * (row - 1);
            } else {                  // upper: i+1, wrap 0 -> ni-1, j+1
              if (s == 1 && i < ni - 1) dv = prev;
              else if (s == 0 && per && i == 0) dv = first;
              else if (s == 3 && row < nj - 1) dv = prv + 4 * (row + 1);
            }
          }
          // a zero increment couples to zero: only slots with a neighbour
          // increment are evaluated (the FP64 pipe is this kernel's bound)
          if (dv != zero4) macro_off(r + MR_SLOT + MR_SW * s, dv, d.Keff, o[s]);
          else o[s][0] = o[s][1] = o[s][2] = o[s][3] = MT(0);
        }
#pragma unroll
        for (int s = 0; s < 4; ++s)
          for (int m = 0; m < 4; ++m) acc[m] += pass == 0 ? -o[s][m] : o[s][m];
        MT idg = r[MR_IDIAG];
        if (pass == 0) for (int m = 0; m < 4; ++m) val[m] = acc[m] * idg;
        else for (int m = 0; m < 4; ++m) val[m] = dws[m] - acc[m] * idg;
        for (int m = 0; m < 4; ++m) d.dW[4 * c + m] = (double)val[m];
      }
      if (act) {
        for (int m = 0; m < 4; ++m) prev[m] = val[m];
        if (i == (pass == 0 ? 0 : ni - 1)) for (int m = 0; m < 4; ++m) first[m] = val[m];
      }
      MT *dst = cur ? buf1 : buf0;
      for (int m = 0; m < 4; ++m) dst[4 * row + m] = val[m];
      if (PF) load(it + 1);     // next diagonal's record, in flight across the barrier
      __syncthreads();
      cur ^= 1;
    }
    for (int m = 0; m < 4; ++m) { prev[m] = 0; first[m] = 0; }
    for (int m = 0; m < 4; ++m) { buf0[4 * row + m] = 0; buf1[4 * row + m] = 0; }
    __syncthreads();
  }
}

// W' = W + dW and the predictor cell record (Step 4 result) for Step 5.
template <typename T> __global__ void k_macro_post(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  T *sr = reinterpret_cast<T *>(d.srec) + (size_t)NSR * c;
  int mask = d.cmask[c];
  *reinterpret_cast<int *>(sr + SR_MASK) = mask;
  if (!(mask & 1)) {
    for (int m = 0; m < 4; ++m) d.Wp[4 * c + m] = d.W[4 * c + m];
    return;
  }
  if (sizeof(T) == 4) {
    const float *inc = reinterpret_cast<const float *>(d.mrec) + (size_t)NMR32 * mrec32_index(d, c) + M32_DWS;
    for (int m = 0; m < 4; ++m) d.Wp[4 * c + m] = d.W[4 * c + m] + (double)inc[m];
  } else {
    for (int m = 0; m < 4; ++m) d.Wp[4 * c + m] = d.W[4 * c + m] + d.dW[4 * c + m];
  }
  Prim p = primitive(d.Wp + 4 * c, d.Keff);
  double *o = d.cpar + NCP * c;
  o[CP_RHO] = p.rho; o[CP_UX] = p.ux; o[CP_UY] = p.uy; o[CP_LAM] = p.lam;
  o[CP_QX] = d.q[2 * c]; o[CP_QY] = d.q[2 * c + 1];
  o[CP_ITAU] = 1.0 / collision_time(p.rho, p.lam, d.mu_ref, d.omega);
  o[CP_DBASE] = d.vol_new[c] * (d.cfl_s / (d.cfl_pseudo * d.dts[c]) + 1.0 / d.stepc[0] + 0.5 * o[CP_ITAU]);
  sr[SR_DBASE] = (T)o[CP_DBASE];
  write_shrec<T>(d, o, d.vol_new[c], reinterpret_cast<T *>(d.shp) + (size_t)NSH * c);
}

// Step 7 (one warp per cell): W^{s+1} = W' + sum V Psi (f^{s+1} - g(W')),
// heat flux about V' (reading R7); flags non-physical states.
template <typename T, int FB> __global__ void k_moments(Dev d) {
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= d.nc) return;
  if (d.status[c] != ST_FIELD) return;
  const T *sr = reinterpret_cast<const T *>(d.shp) + (size_t)NSH * c;
  T hpre = sr[SH_HPRE], ux = sr[SH_UX], uy = sr[SH_UY], lam = sr[SH_LAM];
  T bfac = (T)d.Keff * sr[SH_IL];
  Acc<T> a[6];
  typedef typename Vec2<T>::type T2;
  constexpr int NB = 4;                     // loads of a lane in flight per batch
  for (int kb = lane; kb < d.nv; kb += 32 * NB) {
    T2 fb[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      int k = kb + 32 * u;
      fb[u] = k < d.nv ? ldF<T, FB>(d, (size_t)c * d.nvp + k) : T2{T(0), T(0)};
    }
    // the batch's terms are summed plainly, the batch sums compensated
    T p[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      int k = kb + 32 * u;
      if (k >= d.nv) break;
      T2 fv = fb[u];
      T vx = dvx<T>(d, k), vy = dvy<T>(d, k), w = dw<T>(d, k);
      V2<T> g = maxwellian_pre<T>(hpre, ux, uy, lam, bfac, vx, vy);
      T h = fv.x, b = fv.y;
      T dh = h - g.h, db = b - g.b;
      T v2 = T(0.5) * (vx * vx + vy * vy);
      p[0] += w * dh;
      p[1] += w * vx * dh;
      p[2] += w * vy * dh;
      p[3] += w * (v2 * dh + T(0.5) * db);
      T cx = vx - ux, cy = vy - uy;
      T e = (cx * cx + cy * cy) * h + b;
      p[4] += T(0.5) * w * cx * e;
      p[5] += T(0.5) * w * cy * e;
    }
#pragma unroll
    for (int m = 0; m < 6; ++m) a[m].add(p[m]);
  }
  // lane m < 6 stores component m (W' + sum for W, the sum for q); lane 0
  // then checks the new state for rho > 0 and a positive internal energy
  // (2 rho (rho E) - |rho V|^2 > 0), i.e. rho and lambda positive and finite
  auto tot = [&](int m) { return to_double(warp_total(a[m])); };
  double t0 = tot(0), t1 = tot(1), t2 = tot(2), t3 = tot(3), t4 = tot(4), t5 = tot(5);
  double mine = lane == 0 ? t0 : lane == 1 ? t1 : lane == 2 ? t2 : lane == 3 ? t3 : lane == 4 ? t4 : t5;
  if (d.shard) {        // this shard's sums; k_moments_finish completes them after the exchange
    if (lane < 6) d.msum[6 * c + lane] = mine;
    return;
  }
  double wn = 0.0;
  if (lane < 4) {
    wn = d.Wp[4 * c + lane] + mine;
    d.W[4 * c + lane] = wn;
  } else if (lane < 6) {
    d.q[2 * c + lane - 4] = mine;
  }
  double w0 = __shfl_sync(0xffffffffu, wn, 0), w1 = __shfl_sync(0xffffffffu, wn, 1);
  double w2 = __shfl_sync(0xffffffffu, wn, 2), w3 = __shfl_sync(0xffffffffu, wn, 3);
  if (lane == 0) {
    double ei2 = 2.0 * w0 * w3 - (w1 * w1 + w2 * w2);
    if (!(w0 > 0.0) || !(ei2 > 0.0) || !isfinite(w0) || !isfinite(ei2))
      atomicOr(d.err, EF_NONPHYSICAL);
  }
}

// Step 7 of a sharded step after the exchange: msum holds the sums over the
// whole velocity grid; W = W' + the fix, q the heat flux, checked as above.
__global__ void k_moments_finish(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc || d.status[c] != ST_FIELD) return;
  const double *m = d.msum + 6 * (size_t)c;
  double w[4];
  for (int i = 0; i < 4; ++i) {
    w[i] = d.Wp[4 * c + i] + m[i];
    d.W[4 * c + i] = w[i];
  }
  d.q[2 * c] = m[4];
  d.q[2 * c + 1] = m[5];
  double ei2 = 2.0 * w[0] * w[3] - (w[1] * w[1] + w[2] * w[2]);
  if (!(w[0] > 0.0) || !(ei2 > 0.0) || !isfinite(w[0]) || !isfinite(ei2)) atomicOr(d.err, EF_NONPHYSICAL);
}

// Initial state: f = reduced Maxwellian of the primitive field, W, and q from f.
template <typename T> __global__ void k_init_state(Dev d, const double *prim) {
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= d.nc) return;
  double rho = prim[4 * c], ux = prim[4 * c + 1], uy = prim[4 * c + 2], T0 = prim[4 * c + 3];
  double lam = 1.0 / (2.0 * T0);
  for (int k = lane; k < d.nvp; k += 32) {
    if (k >= d.nv) { stF<T>(d, (size_t)c * d.nvp + k, T(0), T(0)); continue; }
    V2<double> g = maxwellian<double>(rho, ux, uy, lam, d.vx[k], d.vy[k], (double)d.Keff);
    stF<T>(d, (size_t)c * d.nvp + k, (T)g.h, (T)g.b);
  }
  // q from the stored values over the whole grid (a shard recomputes the
  // other shards' Maxwellian values, so no exchange is needed)
  double qx = 0, qy = 0;
  for (int k = lane; k < d.nv_all; k += 32) {
    V2<double> g = maxwellian<double>(rho, ux, uy, lam, d.vxa[k], d.vya[k], (double)d.Keff);
    T h = (T)g.h, b = (T)g.b;
    double cx = d.vxa[k] - ux, cy = d.vya[k] - uy;
    double e = (cx * cx + cy * cy) * (double)h + (double)b;
    qx += 0.5 * d.wa[k] * cx * e;
    qy += 0.5 * d.wa[k] * cy * e;
  }
  qx = warp_sum(qx);
  qy = warp_sum(qy);
  if (lane == 0) {
    double W[4];
    conservative(rho, ux, uy, lam, d.Keff, W);
    for (int m = 0; m < 4; ++m) d.W[4 * c + m] = W[m];
    d.q[2 * c] = qx;
    d.q[2 * c + 1] = qy;
  }
}

// Diagnostic: D_ik for every (cell, velocity), written as FP64.
template <typename T> __global__ void k_flux_div_all(Dev d, double *D) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t n = (size_t)d.nc * d.nv;
  if (t >= n) return;
  int c = (int)(t / d.nv), k = (int)(t % d.nv);
  V2<T> r = {0, 0};
  if (d.status[c] == ST_FIELD) r = flux_div<T>(d, c, k);
  D[2 * t] = (double)r.h;
  D[2 * t + 1] = (double)r.b;
}

// Sum of S * wall macro flux per block: one CTA per block, a strided partial
// sum per thread and a fixed-shape tree, so the order (and the result) is
// the same on every call.
constexpr int WL_THREADS = 256;
__global__ void __launch_bounds__(WL_THREADS) k_wall_loads(Dev d) {
  __shared__ double part[4][WL_THREADS];
  int b = blockIdx.x;
  double s[4] = {0, 0, 0, 0};
  for (int f = threadIdx.x; f < d.nf; f += WL_THREADS) {
    if (d.face_block[f] != b || d.face_kind[f] != BC_WALL) continue;
    for (int m = 0; m < 4; ++m) s[m] += d.fflux[4 * f + m];
  }
  for (int m = 0; m < 4; ++m) part[m][threadIdx.x] = s[m];
  __syncthreads();
  for (int w = WL_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int m = 0; m < 4; ++m) part[m][threadIdx.x] += part[m][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) d.wall_loads[4 * b + threadIdx.x] = part[threadIdx.x][0];
}

// Torque about the point ctr[b] of each block's wall force: sum over its
// wall faces of (x_f - ctr) x (S F_x, S F_y) of the last flux evaluation
// (mid-time face centres), same fixed reduction shape as k_wall_loads.
__global__ void __launch_bounds__(WL_THREADS) k_wall_torque(Dev d, const double *ctr, double *out) {
  __shared__ double part[WL_THREADS];
  int b = blockIdx.x;
  double cx = ctr[2 * b], cy = ctr[2 * b + 1], s = 0.0;
  for (int f = threadIdx.x; f < d.nf; f += WL_THREADS) {
    if (d.face_block[f] != b || d.face_kind[f] != BC_WALL) continue;
    double rx = d.xf[2 * f] - cx, ry = d.xf[2 * f + 1] - cy;
    s += rx * d.fflux[4 * f + 2] - ry * d.fflux[4 * f + 1];
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = WL_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = part[0];
}

// Copy f between the storage type and FP64 (get/set state).
template <typename T> __global__ void k_f_to_double(Dev d, double *out) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t n = (size_t)d.nc * d.nv;
  if (t >= n) return;
  int c = (int)(t / d.nv), k = (int)(t % d.nv);
  auto v = ldF<T>(d, (size_t)c * d.nvp + k);
  out[2 * t] = (double)v.x;
  out[2 * t + 1] = (double)v.y;
}
template <typename T> __global__ void k_f_from_double(Dev d, const double *in) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t n = (size_t)d.nc * d.nv;
  if (t >= n) return;
  int c = (int)(t / d.nv), k = (int)(t % d.nv);
  stF<T>(d, (size_t)c * d.nvp + k, (T)in[2 * t], (T)in[2 * t + 1]);
}

// ------------------------------------------------------- launch wrappers
static inline int nblk(size_t n, int b) { return (int)((n + b - 1) / b); }

// ---------------------------------------------------------------- metrics
// Per-block sums in a fixed order (each thread strides over its items, then
// a shared-memory tree), finished by one block in the same way: the metrics
// are the same bits on every run of a given mesh and launch shape.
__device__ __forceinline__ void met_block_sum(double *sh, double v, double *out) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int h = MET_THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
  __syncthreads();
}

// |R|^2 of Step 4: R = T_W - Omega^{n+1} W / dt - F / 2 (the right-hand side
// of the macro LU-SGS, before W changes in this iteration)
__global__ void __launch_bounds__(MET_THREADS) k_met_macro(Dev d) {
  __shared__ double sh[MET_THREADS];
  double idt = 1.0 / d.stepc[0], acc = 0.0;
  for (int c = blockIdx.x * MET_THREADS + threadIdx.x; c < d.nc; c += MET_BLOCKS * MET_THREADS) {
    if (!(d.cmask[c] & 1)) continue;
    double vol = d.vol_new[c];
    for (int m = 0; m < 4; ++m) {
      double r = d.TW[4 * c + m] - vol * idt * d.W[4 * c + m] - 0.5 * d.Fc[4 * c + m];
      acc += r * r;
    }
  }
  met_block_sum(sh, acc, d.mpart + MET_R2 * MET_BLOCKS + blockIdx.x);
}

// |r|^2 of Step 5 over the solved cells and this context's velocities
template <typename T> __global__ void __launch_bounds__(MET_THREADS) k_met_micro(Dev d) {
  __shared__ double sh[MET_THREADS];
  double acc = 0.0;
  size_t n = (size_t)d.nc * d.nvp;
  for (size_t t = (size_t)blockIdx.x * MET_THREADS + threadIdx.x; t < n; t += (size_t)MET_BLOCKS * MET_THREADS) {
    int c = (int)(t / d.nvp), k = (int)(t - (size_t)c * d.nvp);
    if (k >= d.nv || !(d.cmask[c] & 1)) continue;
    typename Vec2<T>::type r = ldf<T>(d.dfs, t);
    acc += (double)r.x * (double)r.x + (double)r.y * (double)r.y;
  }
  met_block_sum(sh, acc, d.mpart + MET_RMICRO2 * MET_BLOCKS + blockIdx.x);
}

// |W^{s+1} - W'|^2 (Step 7) and the totals of Omega^{n+1} W over the field
__global__ void __launch_bounds__(MET_THREADS) k_met_fix(Dev d) {
  __shared__ double sh[MET_THREADS];
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int c = blockIdx.x * MET_THREADS + threadIdx.x; c < d.nc; c += MET_BLOCKS * MET_THREADS) {
    if (d.status[c] != ST_FIELD) continue;
    double vol = d.vol_new[c];
    for (int m = 0; m < 4; ++m) {
      double w = d.W[4 * c + m], e = w - d.Wp[4 * c + m];
      acc[0] += e * e;
      acc[1 + m] += vol * w;
    }
  }
  for (int q = 0; q < 5; ++q) met_block_sum(sh, acc[q], d.mpart + (MET_FIX2 + q) * MET_BLOCKS + blockIdx.x);
}

__global__ void __launch_bounds__(MET_THREADS) k_met_final(Dev d) {
  __shared__ double sh[MET_THREADS];
  for (int q = 0; q < MET_NQ; ++q) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < MET_BLOCKS; b += MET_THREADS) acc += d.mpart[q * MET_BLOCKS + b];
    met_block_sum(sh, acc, d.mout + q);
  }
}

void launch_metrics(const Dev &d, cudaStream_t s, int stage, int fp32) {
  if (stage == 0) k_met_macro<<<MET_BLOCKS, MET_THREADS, 0, s>>>(d);
  else if (stage == 1) {
    if (fp32) k_met_micro<float><<<MET_BLOCKS, MET_THREADS, 0, s>>>(d);
    else k_met_micro<double><<<MET_BLOCKS, MET_THREADS, 0, s>>>(d);
  } else {
    k_met_fix<<<MET_BLOCKS, MET_THREADS, 0, s>>>(d);
    k_met_final<<<1, MET_THREADS, 0, s>>>(d);
  }
}

void launch_move_nodes(const Dev &d, cudaStream_t s) { k_move_nodes<<<nblk(d.nn, 256), 256, 0, s>>>(d); }

// Small host->device uploads (motion maps, search-bin boxes) travel as kernel
// arguments: the bytes are captured when the launch is issued, so the upload
// neither waits on the stream nor needs pinned staging, and it can be
// captured in a graph.
struct UploadBlob {
  unsigned char b[2048];
};
__global__ void k_upload(unsigned char *dst, UploadBlob blob, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = blob.b[i];
}
int launch_upload(void *dst, const void *src, size_t n, cudaStream_t s) {
  const unsigned char *p = static_cast<const unsigned char *>(src);
  unsigned char *q = static_cast<unsigned char *>(dst);
  int launches = 0;
  while (n > 0) {
    size_t m = n < sizeof(UploadBlob) ? n : sizeof(UploadBlob);
    UploadBlob blob;
    memcpy(blob.b, p, m);
    k_upload<<<1, 256, 0, s>>>(q, blob, (int)m);
    p += m;
    q += m;
    n -= m;
    ++launches;
  }
  return launches;
}
void launch_geometry(const Dev &d, cudaStream_t s, int fp32) {
  k_cell_geom<<<nblk(d.nc, 256), 256, 0, s>>>(d);
  k_face_geom<<<nblk(d.nf, 256), 256, 0, s>>>(d);
  k_dts<<<nblk(d.nc, 256), 256, 0, s>>>(d, d.vbox[0], d.vbox[1], d.vbox[2], d.vbox[3]);
  int n = d.nf > d.nc ? d.nf : d.nc;
  if (fp32) k_geo_records<float><<<nblk(n, 256), 256, 0, s>>>(d);
  else k_geo_records<double><<<nblk(n, 256), 256, 0, s>>>(d);
}
void launch_slope_geo(const Dev &d, cudaStream_t s) { k_slope_geo<<<nblk(d.nc, 256), 256, 0, s>>>(d); }

void launch_ghost_gradW(const Dev &d, cudaStream_t s) {
  k_ghost<<<nblk(d.nf, 256), 256, 0, s>>>(d);
  k_gradW<<<nblk(d.nc, 256), 256, 0, s>>>(d);
}
void launch_gradW(const Dev &d, cudaStream_t s) { k_gradW<<<nblk(d.nc, 256), 256, 0, s>>>(d); }
void launch_face_coef(const Dev &d, cudaStream_t s, int fp32) {
  if (fp32) {
    k_face_scalar<float><<<nblk(d.nf, 128), 128, 0, s>>>(d);
    k_face_coef_sep<float><<<nblk((size_t)d.nf * FCG, 256), 256, 0, s>>>(d);
    if (d.nwall > 0)
      k_face_coef<float><<<nblk((size_t)d.nwall * 32 * FCW, 256), 256, 0, s>>>(d, d.wall_faces, d.nwall);
  } else {
    k_face_scalar<double><<<nblk(d.nf, 128), 128, 0, s>>>(d);
    k_face_coef_sep<double><<<nblk((size_t)d.nf * FCG, 256), 256, 0, s>>>(d);
    if (d.nwall > 0)
      k_face_coef<double><<<nblk((size_t)d.nwall * 32 * FCW, 256), 256, 0, s>>>(d, d.wall_faces, d.nwall);
  }
}
void launch_cell_macro(const Dev &d, cudaStream_t s, int level_n) {
  k_cell_macro<<<nblk(d.nc, 256), 256, 0, s>>>(d, level_n);
}
void launch_cell_params(const Dev &d, cudaStream_t s, const double *W, double *out, int fp32) {
  if (fp32) k_cell_params<float><<<nblk(d.nc, 256), 256, 0, s>>>(d, W, out);
  else k_cell_params<double><<<nblk(d.nc, 256), 256, 0, s>>>(d, W, out);
}
// dynamic shared memory of the sweeps: up to the 227 KB a CTA may use
constexpr size_t kMacroSmem = 227 * 1024;
// The sweep records are gathered on the caller's stream before the fork, so
// the sweep kernel is the first work of the side stream: it then takes its
// empty SMs before the flux kernel launched beside it fills the GPU.
void launch_macro_prep(const Dev &d, cudaStream_t s, int fp32) {
  if (fp32) k_macro_prep<float><<<nblk(d.nc, 256), 256, 0, s>>>(d, reinterpret_cast<float *>(d.mrec));
  else k_macro_prep<double><<<nblk(d.nc, 256), 256, 0, s>>>(d, reinterpret_cast<double *>(d.mrec));
}

void launch_macro_sweep(const Dev &d, cudaStream_t s, int rows, int fp32) {
  if (fp32) {
    float *rec = reinterpret_cast<float *>(d.mrec);
    size_t per = (size_t)rows * NMR32 * sizeof(float);
    size_t base = (MACRO_SMEM_HEAD + 8 * (size_t)rows) * sizeof(float);
    int NS = (int)((kMacroSmem - base) / per);
    NS = NS > 4 ? 4 : (NS < 2 ? 0 : NS);
    // two threads a row on the slots of the pass (PM) where the rows fit
    int tpr = rows <= 256 ? 2 : 1;
    bool pm = tpr == 2;
    if (const char *env = getenv("UGKS_MACRO_TPR")) {   // tuning: threads per row (1, 2 or 4; plain slots)
      int t = atoi(env);
      if ((t == 1 || t == 2 || t == 4) && t * rows <= 512) { tpr = t; pm = false; }
    }
    // the whole shared memory of an SM: the sweep's SMs take no CTA of the
    // kernels running beside it on the main stream
    size_t sm = kMacroSmem;
    int th = tpr * rows;
#define UGKS_MACRO_F32(ns, tp) k_macro_sweep_f32<ns, tp><<<d.nblocks, th, sm, s>>>(d, rec)
#define UGKS_MACRO_PM(ns) k_macro_sweep_f32<ns, 2, true><<<d.nblocks, th, sm, s>>>(d, rec)
    if (pm) {
      if (NS == 4) UGKS_MACRO_PM(4); else if (NS == 3) UGKS_MACRO_PM(3);
      else if (NS == 2) UGKS_MACRO_PM(2); else UGKS_MACRO_PM(0);
    } else if (tpr == 4) {
      if (NS == 4) UGKS_MACRO_F32(4, 4); else if (NS == 3) UGKS_MACRO_F32(3, 4);
      else if (NS == 2) UGKS_MACRO_F32(2, 4); else UGKS_MACRO_F32(0, 4);
    } else if (tpr == 2) {
      if (NS == 4) UGKS_MACRO_F32(4, 2); else if (NS == 3) UGKS_MACRO_F32(3, 2);
      else if (NS == 2) UGKS_MACRO_F32(2, 2); else UGKS_MACRO_F32(0, 2);
    } else {
      if (NS == 4) UGKS_MACRO_F32(4, 1); else if (NS == 3) UGKS_MACRO_F32(3, 1);
      else if (NS == 2) UGKS_MACRO_F32(2, 1); else UGKS_MACRO_F32(0, 1);
    }
#undef UGKS_MACRO_F32
#undef UGKS_MACRO_PM
  } else {
    double *rec = reinterpret_cast<double *>(d.mrec);
    k_macro_sweep<double><<<d.nblocks, rows, kMacroSmem, s>>>(d, rec);
  }
  if (fp32) k_macro_post<float><<<nblk(d.nc, 256), 256, 0, s>>>(d);
  else k_macro_post<double><<<nblk(d.nc, 256), 256, 0, s>>>(d);
}
// shared memory of the macro sweeps exceeds the default 48 KB
void sweep_setup() {
  int ms = (int)kMacroSmem;
  cudaFuncSetAttribute(k_macro_sweep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, ms);
#define UGKS_MACRO_ATTR(ns, tp) \
  cudaFuncSetAttribute(k_macro_sweep_f32<ns, tp>, cudaFuncAttributeMaxDynamicSharedMemorySize, ms)
  UGKS_MACRO_ATTR(4, 4); UGKS_MACRO_ATTR(3, 4); UGKS_MACRO_ATTR(2, 4); UGKS_MACRO_ATTR(0, 4);
  UGKS_MACRO_ATTR(4, 2); UGKS_MACRO_ATTR(3, 2); UGKS_MACRO_ATTR(2, 2); UGKS_MACRO_ATTR(0, 2);
  UGKS_MACRO_ATTR(4, 1); UGKS_MACRO_ATTR(3, 1); UGKS_MACRO_ATTR(2, 1); UGKS_MACRO_ATTR(0, 1);
#undef UGKS_MACRO_ATTR
#define UGKS_MACRO_ATTR_PM(ns) \
  cudaFuncSetAttribute(k_macro_sweep_f32<ns, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ms)
  UGKS_MACRO_ATTR_PM(4); UGKS_MACRO_ATTR_PM(3); UGKS_MACRO_ATTR_PM(2); UGKS_MACRO_ATTR_PM(0);
#undef UGKS_MACRO_ATTR_PM
}

void launch_moments_finish(const Dev &d, cudaStream_t s) { k_moments_finish<<<nblk(d.nc, 256), 256, 0, s>>>(d); }
// Two cells (warps) a CTA: small CTAs fit beside the velocity reduction's
// two CTAs an SM, with which this Step 7 runs concurrently.
constexpr int MOM_THREADS = 64;
void launch_moments(const Dev &d, cudaStream_t s, int fp32) {
  int g = nblk((size_t)d.nc * 32, MOM_THREADS);
  if (fp32 && d.fbf) k_moments<float, 1><<<g, MOM_THREADS, 0, s>>>(d);
  else if (fp32) k_moments<float, 0><<<g, MOM_THREADS, 0, s>>>(d);
  else k_moments<double, 0><<<g, MOM_THREADS, 0, s>>>(d);
}
void launch_init_state(const Dev &d, cudaStream_t s, const double *prim, int fp32) {
  if (fp32) k_init_state<float><<<nblk((size_t)d.nc * 32, 256), 256, 0, s>>>(d, prim);
  else k_init_state<double><<<nblk((size_t)d.nc * 32, 256), 256, 0, s>>>(d, prim);
}
void launch_flux_div_all(const Dev &d, cudaStream_t s, double *D, int fp32) {
  size_t n = (size_t)d.nc * d.nv;
  if (fp32) k_flux_div_all<float><<<nblk(n, 256), 256, 0, s>>>(d, D);
  else k_flux_div_all<double><<<nblk(n, 256), 256, 0, s>>>(d, D);
}
void launch_wall_loads(const Dev &d, cudaStream_t s) { k_wall_loads<<<d.nblocks, WL_THREADS, 0, s>>>(d); }
void launch_wall_torque(const Dev &d, cudaStream_t s, const double *ctr, double *out) {
  k_wall_torque<<<d.nblocks, WL_THREADS, 0, s>>>(d, ctr, out);
}
void launch_f_convert(const Dev &d, cudaStream_t s, double *out, const double *in, int fp32) {
  size_t n = (size_t)d.nc * d.nv;
  if (out) {
    if (fp32) k_f_to_double<float><<<nblk(n, 256), 256, 0, s>>>(d, out);
    else k_f_to_double<double><<<nblk(n, 256), 256, 0, s>>>(d, out);
  } else {
    if (fp32) k_f_from_double<float><<<nblk(n, 256), 256, 0, s>>>(d, in);
    else k_f_from_double<double><<<nblk(n, 256), 256, 0, s>>>(d, in);
  }
}

}  // namespace ugks
