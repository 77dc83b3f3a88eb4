// ugks_tile.cu -- the two velocity-resolved passes over f of every inner
// iteration (arXiv 2604.09984 Sec. 2.2, Steps 3 and 5) and the micro residual:
//   k_face_reduce  per face, the velocity sums of W0 (the interface
//                  equilibrium's moments) and of the f-dependent parts of the
//                  macro flux (Eq. macroscopicFlux);
//   k_flux         flux divergence D = sum_faces S F_hat per (cell, velocity)
//                  (Eqs. microscopicFlux, fullSolution, wall condition) from
//                  the face reconstruction the reduction stored; it does not
//                  depend on the macro predictor, so it runs while the macro
//                  LU-SGS sweep runs on another stream;
//   k_residual     the micro residual r from D (reading R4).
//
// One CTA per 8x8 cell tile of a block walks all velocity chunks of VK
// velocities.  In the reduction, per chunk, f of the tile plus a two-cell
// halo (ghost cells hold the Maxwellian of their ghost state) is staged in
// shared memory with asynchronous copies, double-buffered so the next chunk
// arrives while the current one is reconstructed.  A thread owns one face
// slot of the tile and one half of every chunk's velocities: everything that
// does not depend on the velocity -- the face geometry, which region cells
// are its two sides, their slope cases and inverse Jacobians, and for the
// flux the interface record of Eq. fullSolution -- is loaded once and kept
// in registers for the whole velocity loop.  The reduction accumulates its
// 12 face sums in registers across all chunks (per-chunk partial sums added
// with an error-free transformation on the FP32 path) and writes them once,
// with no atomics: the result does not depend on scheduling.  It also stores
// the reconstruction of every (face, velocity), so the flux pass reads one
// 4-vector per (face, velocity) instead of re-staging f and recomputing the
// limited gradients.
#include "ugks_internal.cuh"
#include "ugks_launch.h"

namespace ugks {

constexpr int TX = 8, TY = 8, RW = TX + 4, RH = TY + 4, NR = RW * RH;
constexpr int NSI = (TX + 1) * TY;          // i-face slots: tile row w, column x = 0..TX
constexpr int NSLOT = NSI + TX * (TY + 1);  // + j-face slots: tile column w, row y = 0..TY
// Tile shape of the two face kernels (the autotuner's choice): VK velocities
// per chunk, NH threads per face slot, NT threads a CTA.  The NH threads of a
// slot are adjacent lanes and take interleaved velocities (kk = part + NH q),
// so the NH of them store NH consecutive reconstructions -- whole 32-byte
// sectors for NH = 2.  Row strides (in elements) of the staged region (VKP:
// rows of whole 16-byte copies), of the gradient rows and face-flux rows
// (VKG) and of the staged face reconstructions (VKF), chosen so that the
// lanes of a quarter warp -- NH velocities of 8 / NH neighbouring cells or
// faces -- fall in different banks.
template <typename T, int VK_, int NH_> struct FCfg {
  static constexpr int VK = VK_, NH = NH_, NT = NSLOT * NH_, VH = VK_ / NH_;
  static constexpr int VKP = sizeof(T) == 4 ? VK_ + 2 : VK_, VKG = VK_ + 2, VKF = VK_ + 2;
  static_assert(NT % VK == 0 && VK % NH == 0 && NH == 2, "tile shape");
};

// region cell (i, j) of block b -> cell id (>= 0), ghost (-2 - face id) or
// none (-1).  Periodic blocks wrap in i.
__device__ __forceinline__ int region_gid(const Dev &d, const int *bi, int off, int i, int j) {
  int ni = bi[0], nj = bi[1], per = bi[2];
  if (per) i = ((i % ni) + ni) % ni;
  bool iin = i >= 0 && i < ni, jin = j >= 0 && j < nj;
  if (iin && jin) return off + j * ni + i;
  int c = -1, s = -1;
  if (jin && !iin) {
    if (i == -1) { c = off + j * ni; s = 0; }
    else if (i == ni) { c = off + j * ni + ni - 1; s = 1; }
  } else if (iin && !jin) {
    if (j == -1) { c = off + i; s = 2; }
    else if (j == nj) { c = off + (nj - 1) * ni + i; s = 3; }
  }
  if (c < 0) return -1;
  if (d.nb_kind[4 * c + s] == NB_GHOST) return -2 - d.nb_id[4 * c + s];
  return -1;
}

// Face id of slot (dir, w, x): dir 0 the i-face left of tile column x of tile
// row w (x = TX: right of the last column), dir 1 the j-face below tile row
// x of tile column w; -1 where the face lies outside the block.
__device__ __forceinline__ int tile_face_id(const Dev &d, int dir, int off, int ni, int nj, int i0, int j0,
                                            int w, int x) {
  if (dir == 0) {
    int i = i0 + x, j = j0 + w;
    if (j >= nj || i > ni) return -1;
    return (i < ni) ? d.cell_faces[4 * (off + j * ni + i) + 0] : d.cell_faces[4 * (off + j * ni + ni - 1) + 1];
  }
  int i = i0 + w, j = j0 + x;
  if (i >= ni || j > nj) return -1;
  return (j < nj) ? d.cell_faces[4 * (off + j * ni + i) + 2] : d.cell_faces[4 * (off + (nj - 1) * ni + i) + 3];
}

// Gradient cells: the 10x10 block of region cells (rows and columns 1..10)
// that can be the upwind side of a tile face; g = (ry - 1) * GW + rx - 1.
constexpr int GW = TX + 2, NG = GW * (TY + 2);
__device__ __forceinline__ int region_of_g(int g) {
  int gy = g / GW;
  return (gy + 1) * RW + (g - gy * GW) + 1;
}
__device__ __forceinline__ int g_of_region(int r) {
  int ry = r / RW;
  return (ry - 1) * GW + (r - ry * RW) - 1;
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4 type; };

// Shared memory of both kernels: the double-buffered region of f, the limited
// Cartesian gradients of the chunk, the velocity table of both buffered
// chunks, and per region cell its id, slope cases and inverse Jacobian (the
// ghost Maxwellian's parameters for ghost cells).
template <typename T, typename C> struct FaceSmem {
  typedef typename Vec2<T>::type T2;
  typedef typename Vec4<T>::type T4;
  static constexpr int VK = C::VK, VKP = C::VKP, VKG = C::VKG;
  T2 *F;         // [2][NR][VKP]
  T4 *G;         // [NG][VKG]: (d_x h, d_x b, d_y h, d_y b)
  T4 *vt;        // [2][VK]: vx, vy, weight, |v|^2 / 2
  T4 *J;         // [NR]: inverse Jacobian (real cells), ghost state rho lam / pi, Vx, Vy, lam (ghosts)
  int *gid;      // [NR]
  int *fl;       // [NR]: slope cases, 0 for ghost / missing cells
  __host__ __device__ static constexpr size_t bytes() {
    return sizeof(T2) * 2 * NR * VKP + sizeof(T4) * NG * VKG + sizeof(T4) * 2 * VK + sizeof(T4) * NR +
           sizeof(int) * 2 * NR;
  }
  __device__ void carve(unsigned char *p) {
    F = reinterpret_cast<T2 *>(p);
    p += sizeof(T2) * 2 * NR * VKP;
    G = reinterpret_cast<T4 *>(p);
    p += sizeof(T4) * NG * VKG;
    vt = reinterpret_cast<T4 *>(p);
    p += sizeof(T4) * 2 * VK;
    J = reinterpret_cast<T4 *>(p);
    p += sizeof(T4) * NR;
    gid = reinterpret_cast<int *>(p);
    p += sizeof(int) * NR;
    fl = reinterpret_cast<int *>(p);
  }
};

// region ids, slope cases, inverse Jacobians and ghost states (once per CTA)
template <typename T, typename C>
__device__ __forceinline__ void region_meta(const Dev &d, FaceSmem<T, C> &S, const int *bi, int off, int i0, int j0) {
  typedef typename Vec4<T>::type T4;
  for (int r = threadIdx.x; r < NR; r += blockDim.x) {
    int rx = r % RW, ry = r / RW;
    int g = region_gid(d, bi, off, i0 - 2 + rx, j0 - 2 + ry);
    S.gid[r] = g;
    T4 J = {T(0), T(0), T(0), T(0)};
    int fl = 0;
    if (g >= 0) {
      fl = d.slope_flags[g];
      if (sizeof(T) == 4) {
        float4 j = d.jinvf[g];
        J.x = (T)j.x; J.y = (T)j.y; J.z = (T)j.z; J.w = (T)j.w;
      } else {
        J.x = (T)d.jinv[4 * g]; J.y = (T)d.jinv[4 * g + 1]; J.z = (T)d.jinv[4 * g + 2]; J.w = (T)d.jinv[4 * g + 3];
      }
    } else if (g <= -2) {
      Prim p = primitive(d.ghostW + 4 * (-2 - g), d.Keff);
      J.x = (T)(p.rho * p.lam * M_1_PI); J.y = (T)p.ux; J.z = (T)p.uy; J.w = (T)p.lam;
    }
    S.J[r] = J;
    S.fl[r] = fl;
  }
}

// Issue the copies of velocity chunk `ch` into buffer `buf`: real cells by
// asynchronous 16-byte copies (bf16 storage: load and widen), ghost cells the
// Maxwellian of their ghost state, no cell / padding velocities zero; and the
// chunk's velocity table.  EP velocities per copy.
template <typename T, int FB, typename C>
__device__ __forceinline__ void stage_chunk(const Dev &d, FaceSmem<T, C> &S, int ch, int buf) {
  typedef typename Vec2<T>::type T2;
  typedef typename Vec4<T>::type T4;
  constexpr int VK = C::VK, VKP = C::VKP, EP = 16 / (int)sizeof(T2), NP = VK / EP;
  const int kb = ch * VK;
  T2 *Fb = S.F + (size_t)buf * NR * VKP;
  for (int it = threadIdx.x; it < NR * NP; it += blockDim.x) {
    int r = it / NP, kp = it - (it / NP) * NP;
    int kk = kp * EP, k = kb + kk;
    int g = S.gid[r];
    T2 *dst = Fb + r * VKP + kk;
    if (k < d.nv && g >= 0) {
      if (FB) {
#pragma unroll
        for (int e = 0; e < EP; ++e) {
          auto v = ldF<T, 1>(d, (size_t)g * d.nvp + k + e);
          dst[e] = T2{v.x, v.y};
        }
      } else {
        // k < nv <= nvp, nvp a multiple of 4 and k even: the pair stays in
        // the cell's row (padding velocities hold zero)
        cp_async<16>(dst, reinterpret_cast<const T2 *>(d.f) + (size_t)g * d.nvp + k);
      }
      continue;
    }
#pragma unroll
    for (int e = 0; e < EP; ++e) {
      T2 v = {T(0), T(0)};
      if (k + e < d.nv && g <= -2) {
        T4 p = S.J[r];
        V2<T> m = maxwellian_pre<T>(p.x, p.y, p.z, p.w, (T)d.Keff / (T(2) * p.w), dvx<T>(d, k + e), dvy<T>(d, k + e));
        v.x = m.h;
        v.y = m.b;
      }
      dst[e] = v;
    }
  }
  for (int kk = threadIdx.x; kk < VK; kk += blockDim.x) {
    int k = kb + kk;
    T vx = k < d.nv ? dvx<T>(d, k) : T(0), vy = k < d.nv ? dvy<T>(d, k) : T(0);
    T4 t = {vx, vy, k < d.nv ? dw<T>(d, k) : T(0), T(0.5) * (vx * vx + vy * vy)};
    S.vt[buf * VK + kk] = t;
  }
  cp_async_commit();
}

// limited slope of one logical direction from the backward / forward
// differences a, b (reading R1: van Leer where both neighbours exist,
// one-sided where one does)
template <typename T> __device__ __forceinline__ T lim_slope(T a, T b, bool hm, bool hp) {
  T v = vanleer<T>(a, b);
  return hm ? (hp ? v : a) : (hp ? b : T(0));
}

// Phase A of a chunk: the limited Cartesian gradient of (h, b) of every
// gradient cell and chunk velocity (lanes run over velocities; ghost and
// missing cells carry none).  A thread keeps one chunk velocity and walks
// the gradient cells with a fixed stride; cells with all four neighbours take
// the two-sided limiter without the one-sided selections.
template <typename T, typename C>
__device__ __forceinline__ void chunk_gradients(FaceSmem<T, C> &S, int buf) {
  typedef typename Vec2<T>::type T2;
  typedef typename Vec4<T>::type T4;
  constexpr int VK = C::VK, VKP = C::VKP, VKG = C::VKG, GS = C::NT / VK;
  const T2 *Fb = S.F + (size_t)buf * NR * VKP;
  const int kk = threadIdx.x % VK;
  for (int g = threadIdx.x / VK; g < NG; g += GS) {
    int r = region_of_g(g);
    int fl = S.fl[r];
    T4 G = {T(0), T(0), T(0), T(0)};
    if (fl) {
      T4 J = S.J[r];
      const T2 *c = Fb + r * VKP + kk;
      T2 fc = c[0], im = c[-VKP], ip = c[VKP], jm = c[-RW * VKP], jp = c[RW * VKP];
      T sih, sib, sjh, sjb;
      if (fl == 15) {
        sih = vanleer<T>(fc.x - im.x, ip.x - fc.x);
        sib = vanleer<T>(fc.y - im.y, ip.y - fc.y);
        sjh = vanleer<T>(fc.x - jm.x, jp.x - fc.x);
        sjb = vanleer<T>(fc.y - jm.y, jp.y - fc.y);
      } else {
        bool him = fl & 1, hip = fl & 2, hjm = fl & 4, hjp = fl & 8;
        sih = lim_slope<T>(fc.x - im.x, ip.x - fc.x, him, hip);
        sib = lim_slope<T>(fc.y - im.y, ip.y - fc.y, him, hip);
        sjh = lim_slope<T>(fc.x - jm.x, jp.x - fc.x, hjm, hjp);
        sjb = lim_slope<T>(fc.y - jm.y, jp.y - fc.y, hjm, hjp);
      }
      G.x = J.x * sih + J.y * sjh;
      G.y = J.x * sib + J.y * sjb;
      G.z = J.z * sih + J.w * sjh;
      G.w = J.z * sib + J.w * sjb;
    }
    S.G[g * VKG + kk] = G;
  }
}

// One side of a face: its region cell, its gradient cell, and the vector
// from its centre to the face centre.
template <typename T> struct Side {
  int r, g;
  T dx, dy;
};

template <typename T> __device__ __forceinline__ Side<T> make_side(int r, T dx, T dy) {
  Side<T> s;
  s.r = r;
  s.g = g_of_region(r);
  s.dx = dx;
  s.dy = dy;
  return s;
}

// Reconstructed face value f + dx.grad f and w.grad f of side s at chunk
// velocity kk.
template <typename T, typename C>
__device__ __forceinline__ void side_value(const FaceSmem<T, C> &S, const typename Vec2<T>::type *Fb, int r, int g,
                                           T dx, T dy, int kk, T wx, T wy, V2<T> &ff, V2<T> &wg) {
  constexpr int VKP = C::VKP, VKG = C::VKG;
  auto fc = Fb[r * VKP + kk];
  auto G = S.G[g * VKG + kk];
  ff.h = fc.x + dx * G.x + dy * G.z;
  ff.b = fc.y + dx * G.y + dy * G.w;
  wg.h = wx * G.x + wy * G.z;
  wg.b = wx * G.y + wy * G.w;
}

// Upwind face value and w.grad f (walls: the interior side L only); only
// w.S = 0 exactly averages the two sides.
template <typename T, typename C>
__device__ __forceinline__ void upwind(const FaceSmem<T, C> &S, const typename Vec2<T>::type *Fb, const Side<T> &L,
                                       const Side<T> &R, bool wall, int kk, T wS, T wx, T wy, V2<T> &ff,
                                       V2<T> &wg) {
  if (!wall && wS == T(0)) {
    V2<T> f1, g1, f2, g2;
    side_value<T, C>(S, Fb, L.r, L.g, L.dx, L.dy, kk, wx, wy, f1, g1);
    side_value<T, C>(S, Fb, R.r, R.g, R.dx, R.dy, kk, wx, wy, f2, g2);
    ff = {T(0.5) * (f1.h + f2.h), T(0.5) * (f1.b + f2.b)};
    wg = {T(0.5) * (g1.h + g2.h), T(0.5) * (g1.b + g2.b)};
    return;
  }
  bool useR = !wall && wS < T(0);
  side_value<T, C>(S, Fb, useR ? R.r : L.r, useR ? R.g : L.g, useR ? R.dx : L.dx, useR ? R.dy : L.dy, kk, wx, wy,
                   ff, wg);
}

// Slot -> (direction, tile row / column w, position x) and the region cells
// A (lower logical side) and B of the face.
__device__ __forceinline__ void slot_geom(int slot, int &dir, int &w, int &x, int &A, int &B) {
  if (slot < NSI) {
    dir = 0;
    w = slot / (TX + 1);
    x = slot - w * (TX + 1);
    A = (x + 1) + (w + 2) * RW;
    B = A + 1;
  } else {
    int s = slot - NSI;
    dir = 1;
    w = s / (TY + 1);
    x = s - w * (TY + 1);
    A = (w + 2) + (x + 1) * RW;
    B = A + RW;
  }
}

// The stored reconstruction of one (face, velocity): (f_face h, f_face b,
// w.grad f h, w.grad f b).
template <typename T>
__device__ __forceinline__ void st_fval(typename Vec4<T>::type *p, const V2<T> &ff, const V2<T> &wg) {
  typename Vec4<T>::type v;
  v.x = ff.h; v.y = ff.b; v.z = wg.h; v.w = wg.b;
  *p = v;
}

// bytes of the flux pass's face-flux rows (a multiple of 32)
template <typename T, typename C> __host__ __device__ constexpr size_t flux_fs_bytes() {
  return (sizeof(typename Vec2<T>::type) * NSLOT * C::VKG + 31) / 32 * 32;
}

// error-free sum (Knuth): s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// ------------------------------------------------------------ face reduction
// Per owned face (the i- and j-faces on the low side of the tile's cells, and
// the closing faces at a non-periodic block end) the 12 sums over all
// velocities: W0 = sum V Psi f_face (interior faces), and the incident-part
// sums sum V Psi w.S f_face and sum V Psi w.S (w.grad f) (Eq. macroscopicFlux
// with the time integrals q1, q2 applied afterwards).  Per chunk: staging of
// the next chunk, gradients (phase A), face sums (phase B); FP32 partial sums
// of two chunks are folded into a (sum, error) pair by an error-free sum.
// The reconstruction of every (face, velocity) -- the upwind face value and
// w.grad f of Eq. fullSolution -- is stored for the flux pass, which then
// needs neither f nor its gradients.
template <typename T, int FB, int VKT, int NHT>
__global__ void __launch_bounds__(NSLOT * NHT) k_face_reduce(Dev d) {
  typedef typename Vec2<T>::type T2;
  typedef typename Vec4<T>::type T4;
  typedef FCfg<T, VKT, NHT> C;
  constexpr int VK = C::VK, VKP = C::VKP, NH = C::NH, VH = VK / NH;
  extern __shared__ __align__(16) unsigned char smraw[];
  FaceSmem<T, C> S;
  S.carve(smraw);
  int tile = blockIdx.x;
  int b = d.tiles[3 * tile], i0 = d.tiles[3 * tile + 1], j0 = d.tiles[3 * tile + 2];
  const int *bi = d.blk_info + 8 * b;
  int ni = bi[0], nj = bi[1], per = bi[2], off = d.cell_off[b];
  region_meta<T, C>(d, S, bi, off, i0, j0);
  __syncthreads();
  const int nch = (d.nv + VK - 1) / VK;
  stage_chunk<T, FB, C>(d, S, 0, 0);
  // this thread's face (the NH threads of a slot are adjacent lanes)
  int slot = threadIdx.x / NH, half = threadIdx.x % NH;
  int dir, w, x, A, B;
  slot_geom(slot, dir, w, x, A, B);
  int fid = tile_face_id(d, dir, off, ni, nj, i0, j0, w, x);
  bool act = false;
  if (fid >= 0) {
    int i = dir == 0 ? i0 + x : i0 + w, j = dir == 0 ? j0 + w : j0 + x;
    bool own = dir == 0 ? ((i < ni && x < TX) || (!per && i == ni)) : ((j < nj && x < TY) || j == nj);
    act = own && d.face_kind[fid] != BC_OVERSET;
    if (act) {
      int Lg = d.face_L[fid], Rg = d.face_R[fid];
      act = d.status[Lg] == ST_FIELD || (Rg >= 0 && d.status[Rg] == ST_FIELD);
    }
  }
  bool wall = false;
  T snx = T(0), sny = T(0), sun = T(0), ufx = T(0), ufy = T(0);
  Side<T> L = make_side<T>(A, T(0), T(0)), R = L;
  if (act) {
    wall = d.face_kind[fid] == BC_WALL;
    __align__(16) T Gr[NFG];
    load_rec<T, NFG>(reinterpret_cast<const T *>(d.fgeo) + (size_t)fid * NFG, Gr);
    snx = Gr[FG_SNX]; sny = Gr[FG_SNY]; sun = Gr[FG_SUN]; ufx = Gr[FG_UFX]; ufy = Gr[FG_UFY];
    int Lr = (S.gid[A] == d.face_L[fid]) ? A : B, Rr = (Lr == A) ? B : A;
    L = make_side<T>(Lr, Gr[FG_DXLX], Gr[FG_DXLY]);
    R = make_side<T>(Rr, Gr[FG_DXRX], Gr[FG_DXRY]);
  }
  T hi[NFS], lo[NFS], acc[NFS];
#pragma unroll
  for (int m = 0; m < NFS; ++m) { hi[m] = T(0); lo[m] = T(0); acc[m] = T(0); }
  for (int ch = 0; ch < nch; ++ch) {
    int buf = ch & 1;
    cp_async_wait<0>();
    __syncthreads();                       // chunk ch visible; phase B of ch-1 done everywhere
    if (ch + 1 < nch) stage_chunk<T, FB, C>(d, S, ch + 1, buf ^ 1);
    chunk_gradients<T, C>(S, buf);
    __syncthreads();
    if (act) {
      const T2 *Fb = S.F + (size_t)buf * NR * VKP;
      const T4 *vt = S.vt + buf * VK;
      const int kb = ch * VK;
      T4 *fv = reinterpret_cast<T4 *>(d.fval) + (size_t)fid * d.nvp + kb;
#pragma unroll 4
      for (int q = 0; q < VH; ++q) {
        int kk = half + NH * q;
        T4 v = vt[kk];
        T vx = v.x, vy = v.y, v2 = v.w;
        T wS = vx * snx + vy * sny - sun;
        // reflected velocities of a wall carry no f (zero weight, no branch)
        T wk = (wall && !(wS > T(0))) ? T(0) : v.z;
        V2<T> ff, wg;
        upwind<T, C>(S, Fb, L, R, wall, kk, wS, vx - ufx, vy - ufy, ff, wg);
        // the flux pass reads the reconstruction from here
        if (kb + kk < d.nv) st_fval<T>(fv + kk, ff, wg);
        T a = wk * ff.h, bb = T(0.5) * wk * ff.b;
        T p0 = a, p1 = vx * a, p2 = vy * a, p3 = v2 * a + bb;
        T ga = wk * wg.h, gb = T(0.5) * wk * wg.b;
        T g0 = ga, g1 = vx * ga, g2 = vy * ga, g3 = v2 * ga + gb;
        acc[FS_W0 + 0] += p0; acc[FS_W0 + 1] += p1; acc[FS_W0 + 2] += p2; acc[FS_W0 + 3] += p3;
        acc[FS_FF + 0] += wS * p0; acc[FS_FF + 1] += wS * p1; acc[FS_FF + 2] += wS * p2; acc[FS_FF + 3] += wS * p3;
        acc[FS_WG + 0] += wS * g0; acc[FS_WG + 1] += wS * g1; acc[FS_WG + 2] += wS * g2; acc[FS_WG + 3] += wS * g3;
      }
      if ((ch & 1) || ch + 1 == nch) {
        if (sizeof(T) == 4) {
#pragma unroll
          for (int m = 0; m < NFS; ++m) {
            float s, e;
            two_sum((float)hi[m], (float)acc[m], s, e);
            hi[m] = (T)s;
            lo[m] += (T)e;
            acc[m] = T(0);
          }
        } else {
#pragma unroll
          for (int m = 0; m < NFS; ++m) { hi[m] += acc[m]; acc[m] = T(0); }
        }
      }
    }
  }
  // the NH parts of a face meet in shared memory (the region buffers are
  // free once every thread has passed the barrier), summed in part order
  __syncthreads();
  T *xs = reinterpret_cast<T *>(S.F);
  if (half > 0) {
    T *o = xs + (size_t)(half - 1) * 2 * NFS * NSLOT;
#pragma unroll
    for (int m = 0; m < NFS; ++m) { o[(2 * m) * NSLOT + slot] = hi[m]; o[(2 * m + 1) * NSLOT + slot] = lo[m]; }
  }
  __syncthreads();
  if (half == 0 && act) {
    double *out = d.fsum + (size_t)NFS * fid;
#pragma unroll
    for (int m = 0; m < NFS; ++m) {
      double v;
      if (sizeof(T) == 4) {
        float h = (float)hi[m], l = (float)lo[m];
        for (int p = 1; p < NH; ++p) {
          const T *o = xs + (size_t)(p - 1) * 2 * NFS * NSLOT;
          float s, e;
          two_sum(h, (float)o[(2 * m) * NSLOT + slot], s, e);
          h = s;
          l = (l + e) + (float)o[(2 * m + 1) * NSLOT + slot];
        }
        v = to_double(h) + to_double(l);
      } else {
        v = (double)hi[m];
        for (int p = 1; p < NH; ++p) v += (double)xs[(size_t)(p - 1) * 2 * NFS * NSLOT + (2 * m) * NSLOT + slot];
      }
      out[m] = (wall && m < FS_FF) ? 0.0 : v;     // walls take W0 from the interior cell
    }
  }
}

// -------------------------------------------------------- flux divergence
// Every face slot of the tile (faces shared with a neighbouring tile are
// evaluated by both) computes S F_hat per velocity into shared memory from
// the reconstruction the reduction pass stored; then each (tile cell,
// velocity) sums its four faces with the cell's orientation signs and stores
// D.  A streaming pass: the reconstructions of a chunk arrive in shared
// memory as one bulk copy per face row (VK 4-vectors, issued by the face's
// own thread, completing on the buffer's mbarrier; double-buffered), each
// (face, velocity) adds the equilibrium part from the face's cubics, and each
// (cell, velocity) makes one store.  ROW: the chunk lies in one row of the
// velocity grid (VK divides N_vx), so c_y is fixed over it: the cubics
// become cubics in c_x with coefficients formed once per chunk, and the
// c_y factor of the Maxwellian is one exponential per chunk.
template <typename T, typename C> __host__ __device__ constexpr size_t flux_fv_bytes() {
  return sizeof(typename Vec4<T>::type) * 2 * NSLOT * C::VKF;
}

template <typename T, int VKT, int NHT, bool ROW> __global__ void __launch_bounds__(NSLOT * NHT) k_flux(Dev d) {
  typedef typename Vec2<T>::type T2;
  typedef typename Vec4<T>::type T4;
  typedef FCfg<T, VKT, NHT> C;
  constexpr int VK = C::VK, VKG = C::VKG, VKF = C::VKF, NH = C::NH, VH = C::VH;
  extern __shared__ __align__(16) unsigned char smraw[];
  T4 *FV = reinterpret_cast<T4 *>(smraw);                                    // [2][NSLOT][VKF]
  T2 *Fs = reinterpret_cast<T2 *>(smraw + flux_fv_bytes<T, C>());            // [NSLOT][VKG]
  T4 *sgn = reinterpret_cast<T4 *>(smraw + flux_fv_bytes<T, C>() + flux_fs_bytes<T, C>());  // [TX*TY]
  T2 *vt = reinterpret_cast<T2 *>(sgn + TX * TY);                           // [2][VK]: vx, vy
  unsigned long long *mb = reinterpret_cast<unsigned long long *>(vt + 2 * VK);  // [2]
  int *cinf = reinterpret_cast<int *>(mb + 2);                              // [TX*TY]: cell id or -1
  int tile = blockIdx.x;
  int b = d.tiles[3 * tile], i0 = d.tiles[3 * tile + 1], j0 = d.tiles[3 * tile + 2];
  const int *bi = d.blk_info + 8 * b;
  int ni = bi[0], nj = bi[1], off = d.cell_off[b];
  if (threadIdx.x == 0) {
    mbar_init(&mb[0], 1);
    mbar_init(&mb[1], 1);
    mbar_fence_init();
  }
  for (int c = threadIdx.x; c < TX * TY; c += blockDim.x) {
    int tx = c % TX, ty = c / TX, i = i0 + tx, j = j0 + ty;
    int g = (i < ni && j < nj) ? off + j * ni + i : -1;
    if (g >= 0 && d.status[g] != ST_FIELD) g = -1;
    cinf[c] = g;
    char4 sc = g >= 0 ? reinterpret_cast<const char4 *>(d.cell_sgn)[g] : make_char4(0, 0, 0, 0);
    sgn[c] = T4{(T)sc.x, (T)sc.y, (T)sc.z, (T)sc.w};
  }
  const int nv = d.nv, nch = (nv + VK - 1) / VK;
  int slot = threadIdx.x / NH, half = threadIdx.x % NH;
  bool act = false;
  int fid;
  {
    int dir, w, x, A, B;
    slot_geom(slot, dir, w, x, A, B);
    fid = tile_face_id(d, dir, off, ni, nj, i0, j0, w, x);
    if (fid >= 0 && d.face_kind[fid] != BC_OVERSET) {
      int Lg = d.face_L[fid], Rg = d.face_R[fid];
      act = d.status[Lg] == ST_FIELD || (Rg >= 0 && d.status[Rg] == ST_FIELD);
    }
  }
  const T4 *frow = reinterpret_cast<const T4 *>(d.fval) + (size_t)(act ? fid : 0) * d.nvp;
  // velocity table of chunk ch into buffer ch & 1
  auto stage_v = [&](int ch) {
    for (int kk = threadIdx.x; kk < VK; kk += blockDim.x) {
      int k = ch * VK + kk;
      T2 t = {T(0), T(0)};
      if (k < nv) { t.x = dvx<T>(d, k); t.y = dvy<T>(d, k); }
      vt[(ch & 1) * VK + kk] = t;
    }
  };
  // this face's row of chunk ch into buffer ch & 1 (the slot's first thread)
  auto stage_row = [&](int ch) {
    if (act && half == 0) {
      int kb = ch * VK;
      unsigned bytes = (unsigned)(sizeof(T4) * (nv - kb < VK ? nv - kb : VK));
      unsigned long long *m = &mb[ch & 1];
      mbar_expect_tx(m, bytes);
      bulk_g2s(FV + ((ch & 1) * NSLOT + slot) * VKF, frow + kb, bytes, m);
    }
  };
  bool wall = false;
  __align__(16) T P[NFP];
  if (act) {
    wall = d.face_kind[fid] == BC_WALL;
    load_rec<T, NFP>(reinterpret_cast<const T *>(d.fparT) + (size_t)fid * NFP, P);
  } else {
#pragma unroll
    for (int m = 0; m < NFP; ++m) P[m] = T(0);
  }
  stage_v(0);
  __syncthreads();                 // mbarriers initialised; cinf, sgn, vt of chunk 0 visible
  stage_row(0);
  __syncthreads();                 // every expectation of chunk 0 registered
  if (threadIdx.x == 0) mbar_arrive(&mb[0]);
  const T Keff = (T)d.Keff;
  for (int ch = 0; ch < nch; ++ch) {
    const int buf = ch & 1, kb = ch * VK;
    // one warp polls the chunk's mbarrier (bounded; after a timeout, flagged,
    // a second wait drains the copies), the others wait at the barrier
    // without taking issue slots
    if (threadIdx.x < 32)
      if (!mbar_wait(&mb[buf], (ch >> 1) & 1, d.err)) mbar_wait(&mb[buf], (ch >> 1) & 1, d.err);
    __syncthreads();               // chunk ch visible; the face fluxes of ch-1 consumed
    if (ch + 1 < nch) {            // buffer buf ^ 1 was last read before the previous combine
      stage_row(ch + 1);
      stage_v(ch + 1);
    }
    const T4 *fvb = FV + (buf * NSLOT + slot) * VKF;
    const T2 *vtb = vt + buf * VK;
    T2 *fso = Fs + slot * VKG;
    // the loops below are uniform per thread: walls (reflected part for
    // w.n <= 0), interior faces of a chunk inside one velocity row (ROW, no
    // ragged tail: N_v is a multiple of VK), other interior faces
    if (act && !wall && ROW) {
      // per-chunk factors: the c_y parts of the cubics and of the Maxwellian
      const T vy = vtb[0].y, cy = vy - P[FP_UY];
      const T *ch3 = P + FP_IH, *cb3 = P + FP_IB;
      const T ah0 = ch3[0] + cy * (ch3[2] + cy * (ch3[5] + cy * ch3[9]));
      const T ah1 = ch3[1] + cy * (ch3[4] + cy * ch3[8]);
      const T ah2 = ch3[3] + cy * ch3[7], ah3 = ch3[6];
      const T ab0 = cb3[0] + cy * (cb3[2] + cy * (cb3[5] + cy * cb3[9]));
      const T ab1 = cb3[1] + cy * (cb3[4] + cy * cb3[8]);
      const T ab2 = cb3[3] + cy * cb3[7], ab3 = cb3[6];
      const T ey = P[FP_HPRE] * r_exp<T>(-P[FP_LAM] * (cy * cy));
      const T wsy = vy * P[FP_SNY] - P[FP_SUN];
      const T snx = P[FP_SNX], ux = P[FP_UX], nlam = -P[FP_LAM], q1 = P[FP_Q1], q2 = P[FP_Q2];
#pragma unroll
      for (int q = 0; q < VH; ++q) {
        const int kk = half + NH * q;
        const T4 fv = fvb[kk];
        const T vx = vtb[kk].x;
        // Eq. fullSolution averaged over dt_s: q1 f + q2 w.grad f + H ih(c)
        // (and b), the equilibrium factors as per-face cubics in c = v - U0
        const T wS = vx * snx + wsy, cx = vx - ux;
        const T H = ey * r_exp<T>(nlam * (cx * cx));
        const T ph = ah0 + cx * (ah1 + cx * (ah2 + cx * ah3));
        const T pb = ab0 + cx * (ab1 + cx * (ab2 + cx * ab3));
        T2 Fo;
        Fo.x = wS * (q1 * fv.x + q2 * fv.z + H * ph);
        Fo.y = wS * (q1 * fv.y + q2 * fv.w + H * pb);
        fso[kk] = Fo;
      }
    } else if (act) {
#pragma unroll 4
      for (int q = 0; q < VH; ++q) {
        const int kk = half + NH * q, k = kb + kk;
        T2 Fo = {T(0), T(0)};
        if (k < nv) {
          const T4 fv = fvb[kk];
          const T2 v = vtb[kk];
          const T vx = v.x, vy = v.y;
          const T wS = vx * P[FP_SNX] + vy * P[FP_SNY] - P[FP_SUN];
          if (wall && !(wS > T(0))) {
            // reflected part: wall Maxwellian at the face velocity (Eq. maxWalldes)
            T wx = vx - P[FP_UFX], wy = vy - P[FP_UFY];
            T lw = P[FP_LAMW];
            T Hw = P[FP_RHOW] * (lw * T(M_1_PI)) * r_exp<T>(-lw * (wx * wx + wy * wy));
            Fo.x = wS * Hw;
            Fo.y = wS * Keff / (T(2) * lw) * Hw;
          } else {
            T cx = vx - P[FP_UX], cy = vy - P[FP_UY];
            T H = P[FP_HPRE] * r_exp<T>(-P[FP_LAM] * (cx * cx + cy * cy));
            T Ih = P[FP_Q1] * fv.x + P[FP_Q2] * fv.z + H * poly3_at<T>(P + FP_IH, cx, cy);
            T Ib = P[FP_Q1] * fv.y + P[FP_Q2] * fv.w + H * poly3_at<T>(P + FP_IB, cx, cy);
            Fo.x = wS * Ih;
            Fo.y = wS * Ib;
          }
        }
        fso[kk] = Fo;
      }
    } else {
#pragma unroll 4
      for (int q = 0; q < VH; ++q) fso[half + NH * q] = T2{T(0), T(0)};
    }
    __syncthreads();               // face fluxes complete; expectations of chunk ch + 1 registered
    if (threadIdx.x == 0 && ch + 1 < nch) mbar_arrive(&mb[buf ^ 1]);
    for (int it = threadIdx.x; it < TX * TY * VK; it += blockDim.x) {
      int c = it / VK, kk = it - (it / VK) * VK;
      int g = cinf[c];
      if (g < 0 || kb + kk >= nv) continue;
      int tx = c % TX, ty = c / TX;
      T4 sg = sgn[c];
      T2 a = Fs[(ty * (TX + 1) + tx) * VKG + kk], bq = Fs[(ty * (TX + 1) + tx + 1) * VKG + kk];
      T2 cq = Fs[(NSI + tx * (TY + 1) + ty) * VKG + kk], dq = Fs[(NSI + tx * (TY + 1) + ty + 1) * VKG + kk];
      T Dh = sg.x * a.x + sg.y * bq.x + sg.z * cq.x + sg.w * dq.x;
      T Db = sg.x * a.y + sg.y * bq.y + sg.z * cq.y + sg.w * dq.y;
      stf<T>(d.Dbuf, (size_t)g * d.nvp + kb + kk, Dh, Db);
    }
  }
}

// Micro residual (Steps 3, 5; reading R4), elementwise over (cell, velocity):
//   r = T - Omega^{n+1} f / dt + (Omega^{n+1} (f+(W') - f)/tau' - D) / 2,
// with the level-n term T = Omega^n f^n / dt + (Omega^n (f+(W^n) - f^n)/tau^n
// - D^n) / 2 formed on the first inner iteration.  r goes to the sweep buffer.
template <typename T, int FB> __global__ void k_residual(Dev d, int first_iter) {
  typedef typename Vec2<T>::type T2;
  // grid: cells x velocity chunks; a thread takes two adjacent velocities
  // (nvp is a multiple of 4, so the pair stays inside the cell's row)
  int c = blockIdx.x, k0 = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
  if (k0 >= d.nv || !(d.cmask[c] & 1)) return;
  const T *cp = reinterpret_cast<const T *>(d.shp) + (size_t)NSH * c;
  T itau = cp[SH_ITAU];
  T vol1 = cp[SH_VOL];
  T idt = sizeof(T) == 4 ? (T)(float)d.stepc[2] : (T)d.stepc[1];
  const T *cn = reinterpret_cast<const T *>(d.shn) + (size_t)NSH * c;
  T2 fv[2], D[2], tn[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    size_t t = (size_t)c * d.nvp + k0 + u;
    fv[u] = ldF<T, FB>(d, t);
    D[u] = ldf<T>(d.Dbuf, t);
    if (!first_iter) tn[u] = ldf<T>(d.Tn, t);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int k = k0 + u;
    if (k >= d.nv) break;
    size_t t = (size_t)c * d.nvp + k;
    T vx = dvx<T>(d, k), vy = dvy<T>(d, k);
    V2<T> fp = shakhov_rec<T>(cp, vx, vy, (T)d.Keff, (T)d.Kint);
    if (first_iter) {
      T itn = cn[SH_ITAU];
      V2<T> fn = shakhov_rec<T>(cn, vx, vy, (T)d.Keff, (T)d.Kint);
      T vol0 = cn[SH_VOL];
      tn[u].x = vol0 * idt * fv[u].x + T(0.5) * (vol0 * (fn.h - fv[u].x) * itn - D[u].x);
      tn[u].y = vol0 * idt * fv[u].y + T(0.5) * (vol0 * (fn.b - fv[u].y) * itn - D[u].y);
      stf<T>(d.Tn, t, tn[u].x, tn[u].y);
    }
    T rh = tn[u].x - vol1 * idt * fv[u].x + T(0.5) * (vol1 * (fp.h - fv[u].x) * itau - D[u].x);
    T rb = tn[u].y - vol1 * idt * fv[u].y + T(0.5) * (vol1 * (fp.b - fv[u].y) * itau - D[u].y);
    stf<T>(d.dfs, t, rh, rb);
  }
}

// The residual in two passes (FP32 path): the part without the predictor W'
// of Step 4, P = T_n - Omega^{n+1} f / dt - D / 2, runs right after the flux
// divergence, beside the macro LU-SGS (the level-n term T_n is formed and
// stored on the first inner iteration); after the macro sweep the second
// pass adds the collision term at W': r = P + Omega^{n+1} (f+(W') - f) / (2 tau').
template <typename T, int FB> __global__ void k_residual_pre(Dev d, int first_iter) {
  typedef typename Vec2<T>::type T2;
  int c = blockIdx.x, k0 = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
  if (k0 >= d.nv || !(d.cmask[c] & 1)) return;
  T vol1 = (T)d.vol_new[c];                 // the value the cell record holds
  T idt = sizeof(T) == 4 ? (T)(float)d.stepc[2] : (T)d.stepc[1];
  const T *cn = reinterpret_cast<const T *>(d.shn) + (size_t)NSH * c;
  T2 fv[2], D[2], tn[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    size_t t = (size_t)c * d.nvp + k0 + u;
    fv[u] = ldF<T, FB>(d, t);
    D[u] = ldf<T>(d.Dbuf, t);
    if (!first_iter) tn[u] = ldf<T>(d.Tn, t);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int k = k0 + u;
    if (k >= d.nv) break;
    size_t t = (size_t)c * d.nvp + k;
    if (first_iter) {
      T vx = dvx<T>(d, k), vy = dvy<T>(d, k);
      T itn = cn[SH_ITAU];
      V2<T> fn = shakhov_rec<T>(cn, vx, vy, (T)d.Keff, (T)d.Kint);
      T vol0 = cn[SH_VOL];
      tn[u].x = vol0 * idt * fv[u].x + T(0.5) * (vol0 * (fn.h - fv[u].x) * itn - D[u].x);
      tn[u].y = vol0 * idt * fv[u].y + T(0.5) * (vol0 * (fn.b - fv[u].y) * itn - D[u].y);
      stf<T>(d.Tn, t, tn[u].x, tn[u].y);
    }
    stf<T>(d.dfs, t, tn[u].x - vol1 * idt * fv[u].x - T(0.5) * D[u].x,
           tn[u].y - vol1 * idt * fv[u].y - T(0.5) * D[u].y);
  }
}

template <typename T, int FB> __global__ void k_residual_post(Dev d) {
  typedef typename Vec2<T>::type T2;
  int c = blockIdx.x, k0 = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
  if (k0 >= d.nv || !(d.cmask[c] & 1)) return;
  const T *cp = reinterpret_cast<const T *>(d.shp) + (size_t)NSH * c;
  T itau = cp[SH_ITAU];
  T hv = T(0.5) * cp[SH_VOL];
  T2 fv[2], P[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    size_t t = (size_t)c * d.nvp + k0 + u;
    fv[u] = ldF<T, FB>(d, t);
    P[u] = ldf<T>(d.dfs, t);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int k = k0 + u;
    if (k >= d.nv) break;
    T vx = dvx<T>(d, k), vy = dvy<T>(d, k);
    V2<T> fp = shakhov_rec<T>(cp, vx, vy, (T)d.Keff, (T)d.Kint);
    stf<T>(d.dfs, (size_t)c * d.nvp + k, P[u].x + hv * (fp.h - fv[u].x) * itau,
           P[u].y + hv * (fp.b - fv[u].y) * itau);
  }
}

template <typename T, typename C> static size_t flux_smem() {
  return flux_fv_bytes<T, C>() + flux_fs_bytes<T, C>() + sizeof(typename Vec4<T>::type) * TX * TY +
         sizeof(typename Vec2<T>::type) * 2 * C::VK + 2 * sizeof(unsigned long long) + sizeof(int) * TX * TY;
}
template <typename T, typename C> static size_t reduce_smem() {
  size_t a = FaceSmem<T, C>::bytes(), b = sizeof(T) * 2 * NFS * NSLOT * (C::NH > 1 ? C::NH - 1 : 1);
  return a > b ? a : b;
}

// Candidate tile shapes of the FP32 face kernels (velocities per chunk,
// threads per face slot); the FP64 path keeps (8, 2).
constexpr int kFaceVK[] = {8, 16, 32};
constexpr int kFaceNH[] = {2, 2, 2};
constexpr int kFaceDefault = 1;     // (16, 2)
int face_tile_count() { return 3; }
void face_tile_shape(int v, int *vk, int *nh) {
  if (v < 0 || v >= face_tile_count()) v = kFaceDefault;
  *vk = kFaceVK[v];
  *nh = kFaceNH[v];
}
int face_tile_default() { return kFaceDefault; }

template <typename T, int FB, int VK, int NH> static void face_attr() {
  typedef FCfg<T, VK, NH> C;
  cudaFuncSetAttribute(k_flux<T, VK, NH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)flux_smem<T, C>());
  cudaFuncSetAttribute(k_flux<T, VK, NH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)flux_smem<T, C>());
  cudaFuncSetAttribute(k_face_reduce<T, FB, VK, NH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)reduce_smem<T, C>());
}
template <int FB> static void face_attr_f32() {
  face_attr<float, FB, 8, 2>();
  face_attr<float, FB, 16, 2>();
  face_attr<float, FB, 32, 2>();
}

void tile_setup() {
  face_attr_f32<0>();
  face_attr_f32<1>();
  face_attr<double, 0, 8, 2>();
}

int tile_count(int ni, int nj) { return ((ni + TX - 1) / TX) * ((nj + TY - 1) / TY); }
void tile_origins(int ni, int nj, int *out) {   // (i0, j0) pairs
  int q = 0;
  for (int tj = 0; tj < (nj + TY - 1) / TY; ++tj)
    for (int ti = 0; ti < (ni + TX - 1) / TX; ++ti) { out[q++] = ti * TX; out[q++] = tj * TY; }
}

template <typename T, int FB, int VK, int NH> static void face_launch(const Dev &d, cudaStream_t s, int which) {
  typedef FCfg<T, VK, NH> C;
  if (which == 0) k_face_reduce<T, FB, VK, NH><<<d.ntiles, C::NT, reduce_smem<T, C>(), s>>>(d);
  else if (d.nvx % VK == 0) k_flux<T, VK, NH, true><<<d.ntiles, C::NT, flux_smem<T, C>(), s>>>(d);
  else k_flux<T, VK, NH, false><<<d.ntiles, C::NT, flux_smem<T, C>(), s>>>(d);
}
template <int FB> static void face_launch_f32(const Dev &d, cudaStream_t s, int which, int v) {
  switch (v) {
    case 0: face_launch<float, FB, 8, 2>(d, s, which); break;
    case 2: face_launch<float, FB, 32, 2>(d, s, which); break;
    default: face_launch<float, FB, 16, 2>(d, s, which); break;
  }
}
static void face_dispatch(const Dev &d, cudaStream_t s, int which, int fp32, int v) {
  if (!fp32) face_launch<double, 0, 8, 2>(d, s, which);
  else if (d.fbf) face_launch_f32<1>(d, s, which, v);
  else face_launch_f32<0>(d, s, which, v);
}

void launch_flux_tile(const Dev &d, cudaStream_t s, int fp32, int tile) { face_dispatch(d, s, 1, fp32, tile); }
void launch_face_reduce_tile(const Dev &d, cudaStream_t s, int fp32, int tile) {
  face_dispatch(d, s, 0, fp32, tile);
}
void launch_residual(const Dev &d, cudaStream_t s, int first_iter, int fp32, int part) {
  int pairs = (d.nv + 1) / 2;
  int bt = pairs >= 256 ? 256 : ((pairs + 31) / 32) * 32;
  dim3 grid(d.nc, (pairs + bt - 1) / bt);
  if (part == 1) {
    if (fp32 && d.fbf) k_residual_pre<float, 1><<<grid, bt, 0, s>>>(d, first_iter);
    else if (fp32) k_residual_pre<float, 0><<<grid, bt, 0, s>>>(d, first_iter);
    else k_residual_pre<double, 0><<<grid, bt, 0, s>>>(d, first_iter);
  } else if (part == 2) {
    if (fp32 && d.fbf) k_residual_post<float, 1><<<grid, bt, 0, s>>>(d);
    else if (fp32) k_residual_post<float, 0><<<grid, bt, 0, s>>>(d);
    else k_residual_post<double, 0><<<grid, bt, 0, s>>>(d);
  } else if (fp32 && d.fbf) k_residual<float, 1><<<grid, bt, 0, s>>>(d, first_iter);
  else if (fp32) k_residual<float, 0><<<grid, bt, 0, s>>>(d, first_iter);
  else k_residual<double, 0><<<grid, bt, 0, s>>>(d, first_iter);
}

}  // namespace ugks
