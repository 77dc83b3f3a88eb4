// ugks_tile.cu -- shared-memory tiled kernels for the two velocity-resolved
// passes over f of every inner iteration (arXiv 2604.09984 Sec. 2.2, Steps 3
// and 5):
//   k_face_reduce_tile  velocity sums per face: W0 of the interface
//                       equilibrium and the f-dependent parts of the macro
//                       flux (Eq. macroscopicFlux);
//   k_flux_tile         flux divergence D = sum_faces S F_hat (Eqs.
//                       microscopicFlux, fullSolution, wall condition), which
//                       does not depend on the macro predictor, so it runs
//                       while the macro LU-SGS sweep runs on another stream;
//   k_residual          the micro residual r from D (reading R4).
// A CTA stages f of an 8x8 cell tile plus a two-cell halo (ghost cells hold
// the Maxwellian of their ghost state) for 32 velocities in shared memory,
// reconstructs from there and evaluates each face of the tile once (one warp
// per tile row for i-faces, per tile column for j-faces).  Lane = velocity.
#include "ugks_internal.cuh"
#include "ugks_launch.h"

namespace ugks {

constexpr int TX = 8, TY = 8, RW = TX + 4, RH = TY + 4, NR = RW * RH, VK = 32;
constexpr int TTHREADS = 256;   // 8 warps: one per tile row / column

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

template <typename T> struct TileSmem {
  typedef typename Vec2<T>::type T2;
  T2 *F;        // NR * VK
  int *gid;     // NR
  int *flags;   // NR: slope flags | status << 8
  T *jinv;      // NR * 4
  T *gprim;     // NR * 4 ghost (rho, ux, uy, lam)
  __host__ __device__ static constexpr size_t bytes() {
    return sizeof(T2) * NR * VK + sizeof(int) * 2 * NR + sizeof(T) * 8 * NR;
  }
  __device__ void carve(unsigned char *p) {
    F = reinterpret_cast<T2 *>(p);
    p += sizeof(T2) * NR * VK;
    jinv = reinterpret_cast<T *>(p);
    p += sizeof(T) * 4 * NR;
    gprim = reinterpret_cast<T *>(p);
    p += sizeof(T) * 4 * NR;
    gid = reinterpret_cast<int *>(p);
    p += sizeof(int) * NR;
    flags = reinterpret_cast<int *>(p);
  }
};

// metadata of the region cells (all threads)
template <typename T>
__device__ __forceinline__ void tile_meta(const Dev &d, TileSmem<T> &S, const int *bi, int off, int i0,
                                          int j0) {
  for (int r = threadIdx.x; r < NR; r += blockDim.x) {
    int rx = r % RW, ry = r / RW;
    int g = region_gid(d, bi, off, i0 - 2 + rx, j0 - 2 + ry);
    S.gid[r] = g;
    if (g >= 0) {
      S.flags[r] = d.slope_flags[g] | (d.status[g] << 8);
      if (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(S.jinv + 4 * r) = d.jinvf[g];
      } else {
        for (int m = 0; m < 4; ++m) S.jinv[4 * r + m] = (T)d.jinv[4 * g + m];
      }
    } else {
      S.flags[r] = ST_HOLE << 8;
      if (g <= -2) {
        Prim p = primitive(d.ghostW + 4 * (-2 - g), d.Keff);
        S.gprim[4 * r] = (T)(p.rho * p.lam * M_1_PI); S.gprim[4 * r + 1] = (T)p.ux;
        S.gprim[4 * r + 2] = (T)p.uy; S.gprim[4 * r + 3] = (T)p.lam;
      }
    }
  }
}

// f of the region for velocity chunk kbase (warp w loads cells w, w+8, ...)
template <typename T, int FB>
__device__ __forceinline__ void tile_load_f(const Dev &d, TileSmem<T> &S, int k, bool kv, T vx, T vy) {
  typedef typename Vec2<T>::type T2;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // real cells: asynchronous copies, all of a lane's in flight at once;
  // ghost cells: the Maxwellian of their ghost state; no cell: zero
  for (int r = w; r < NR; r += nw) {
    int g = S.gid[r];
    T2 *dst = &S.F[r * VK + lane];
    if (kv && g >= 0) {
      if (FB) {                                // bf16 storage: widen on the way in
        auto v = ldF<T, 1>(d, (size_t)g * d.nvp + k);
        *dst = T2{v.x, v.y};
      } else {
        cp_async<(int)sizeof(T2)>(dst, reinterpret_cast<const T2 *>(d.f) + (size_t)g * d.nvp + k);
      }
      continue;
    }
    T2 v = {T(0), T(0)};
    if (kv && g <= -2) {
      const T *p = S.gprim + 4 * r;
      V2<T> m = maxwellian_pre<T>(p[0], p[1], p[2], p[3], (T)d.Keff / (T(2) * p[3]), vx, vy);
      v.x = m.h;
      v.y = m.b;
    }
    *dst = v;
  }
  cp_async_commit();
  cp_async_wait<0>();
}

// limited gradient of region cell r (a real cell) at this lane (reading R1)
template <typename T>
__device__ __forceinline__ void tile_grad(const TileSmem<T> &S, int r, int lane, V2<T> fc, V2<T> &gx,
                                          V2<T> &gy) {
  int fl = S.flags[r];
  V2<T> s[2];
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    int cs = (fl >> (2 * dir)) & 3;
    int st = dir == 0 ? 1 : RW;
    V2<T> o = {T(0), T(0)};
    if (cs == SL_BOTH) {
      auto m = S.F[(r - st) * VK + lane], p = S.F[(r + st) * VK + lane];
      o.h = vanleer<T>(fc.h - m.x, p.x - fc.h);
      o.b = vanleer<T>(fc.b - m.y, p.y - fc.b);
    } else if (cs == SL_P) {
      auto p = S.F[(r + st) * VK + lane];
      o.h = p.x - fc.h;
      o.b = p.y - fc.b;
    } else if (cs == SL_M) {
      auto m = S.F[(r - st) * VK + lane];
      o.h = fc.h - m.x;
      o.b = fc.b - m.y;
    }
    s[dir] = o;
  }
  const T *J = S.jinv + 4 * r;
  gx.h = J[0] * s[0].h + J[1] * s[1].h;
  gx.b = J[0] * s[0].b + J[1] * s[1].b;
  gy.h = J[2] * s[0].h + J[3] * s[1].h;
  gy.b = J[2] * s[0].b + J[3] * s[1].b;
}

// Reconstructed value of region cell r at the face (offset dx, dy from its
// centre) and w.grad f; ghost or missing cells carry no gradient.
template <typename T>
__device__ __forceinline__ void tile_side(const TileSmem<T> &S, int r, int lane, T dx, T dy, T wx, T wy,
                                          V2<T> &f, V2<T> &g) {
  auto v = S.F[r * VK + lane];
  V2<T> fc = {v.x, v.y};
  if (S.gid[r] >= 0) {
    V2<T> gx, gy;
    tile_grad<T>(S, r, lane, fc, gx, gy);
    f = {fc.h + dx * gx.h + dy * gy.h, fc.b + dx * gx.b + dy * gy.b};
    g = {wx * gx.h + wy * gy.h, wx * gx.b + wy * gy.b};
  } else {
    f = fc;       // ghost Maxwellian, no gradient
    g = {T(0), T(0)};
  }
}

// upwind face value and w.grad f for face fid between region cells Lr and Rr
// (walls: interior side, incident velocities only).  Each lane reconstructs
// its own upwind cell, so lanes of one face with opposite signs of w.S do not
// run both sides; only w.S = 0 exactly averages the two sides.
template <typename T>
__device__ __forceinline__ void tile_upwind(const Dev &d, const TileSmem<T> &S, const T *P, int kind,
                                            int Lr, int Rr, int lane, T vx, T vy, T wS, V2<T> &ff,
                                            V2<T> &wg) {
  (void)d;
  T wx = vx - P[FP_UFX], wy = vy - P[FP_UFY];
  bool wall = kind == BC_WALL;
  bool useR = !wall && wS < T(0);
  int U = useR ? Rr : Lr;
  T dx = useR ? P[FP_DXRX] : P[FP_DXLX], dy = useR ? P[FP_DXRY] : P[FP_DXLY];
  tile_side<T>(S, U, lane, dx, dy, wx, wy, ff, wg);
  if (!wall && wS == T(0)) {
    V2<T> f2, g2;
    tile_side<T>(S, Rr, lane, P[FP_DXRX], P[FP_DXRY], wx, wy, f2, g2);
    ff = {T(0.5) * (ff.h + f2.h), T(0.5) * (ff.b + f2.b)};
    wg = {T(0.5) * (wg.h + g2.h), T(0.5) * (wg.b + g2.b)};
  }
}

// S * F_hat of a face at this lane (oriented along the face normal) from its
// staged record Ps (shared memory), kind and left cell Lg.
template <typename T>
__device__ __forceinline__ V2<T> tile_face_flux(const Dev &d, const TileSmem<T> &S, const T *Ps, int kind,
                                                int Lg, int A, int B, int lane, T vx, T vy) {
  if (kind == BC_OVERSET) return {T(0), T(0)};
  __align__(16) T P[NFP];
#pragma unroll
  for (int q = 0; q < (int)(NFP * sizeof(T) / 16); ++q)
    reinterpret_cast<float4 *>(P)[q] = reinterpret_cast<const float4 *>(Ps)[q];
  int Lr = (S.gid[A] == Lg) ? A : B;
  int Rr = (Lr == A) ? B : A;
  T wS = vx * P[FP_SNX] + vy * P[FP_SNY] - P[FP_SUN];
  if (kind == BC_WALL && !(wS > T(0))) {
    T wx = vx - P[FP_UFX], wy = vy - P[FP_UFY];
    T lw = P[FP_LAMW];
    T Hw = P[FP_RHOW] * (lw * T(M_1_PI)) * r_exp<T>(-lw * (wx * wx + wy * wy));
    return {wS * Hw, wS * (T)d.Keff / (T(2) * lw) * Hw};
  }
  V2<T> ff, wg;
  tile_upwind<T>(d, S, P, kind, Lr, Rr, lane, vx, vy, wS, ff, wg);
  V2<T> I = interface_integral<T>(P, vx, vy, ff, wg, (T)d.Keff, (T)d.Kint, (T)d.Pr);
  return {wS * I.h, wS * I.b};
}

// Face id, kind and left cell of face `x` of a tile row (dir 0: the i-face
// left of region column x + 2) or column (dir 1: the j-face below region row
// x + 2); -1 where the face lies outside the block.
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

// Stage per warp the scalars and the records (N values each, from `src`) of
// the up to 9 faces a warp walks: lane x keeps face x's id, kind and left
// cell (read back with shuffles), the records go to the warp's buffer `buf`.
// Every global load of the walk is issued here, side by side, instead of one
// dependent chain per face.
template <typename T, int N>
__device__ __forceinline__ void tile_stage_faces(const Dev &d, const T *src, int my_fid, int &my_kind,
                                                 int &my_L, T *buf, int lane) {
  my_kind = BC_OVERSET;
  my_L = -1;
  if (my_fid >= 0) {
    my_kind = d.face_kind[my_fid];
    my_L = d.face_L[my_fid];
  }
  constexpr int NQ = (int)(N * sizeof(T) / 16);
  constexpr int ROUNDS = ((TX + 1) * NQ + 31) / 32;
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    int q = r * 32 + lane;
    int x = q / NQ, ch = q - (q / NQ) * NQ;
    bool in = x <= TX;
    int f = __shfl_sync(0xffffffffu, my_fid, in ? x : 0);
    int kd = __shfl_sync(0xffffffffu, my_kind, in ? x : 0);
    if (in && f >= 0 && kd != BC_OVERSET)
      reinterpret_cast<float4 *>(buf + (size_t)x * N)[ch] =
          __ldg(reinterpret_cast<const float4 *>(src + (size_t)f * N) + ch);
  }
  __syncwarp();
}

__device__ __forceinline__ int cell_status(const TileSmem<float> &S, int r) { return S.flags[r] >> 8; }
__device__ __forceinline__ int cell_status(const TileSmem<double> &S, int r) { return S.flags[r] >> 8; }

// ------------------------------------------------------- flux divergence
template <typename T, int FB> __global__ void __launch_bounds__(TTHREADS) k_flux_tile(Dev d) {
  typedef typename Vec2<T>::type T2;
  extern __shared__ __align__(16) unsigned char smraw[];
  TileSmem<T> S;
  S.carve(smraw);
  T2 *Ds = reinterpret_cast<T2 *>(smraw + TileSmem<T>::bytes());   // TX*TY*VK
  int tile = blockIdx.x % d.ntiles, vc = blockIdx.x / d.ntiles;
  int b = d.tiles[3 * tile], i0 = d.tiles[3 * tile + 1], j0 = d.tiles[3 * tile + 2];
  const int *bi = d.blk_info + 8 * b;
  int ni = bi[0], nj = bi[1], off = d.cell_off[b];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int k = vc * VK + lane;
  bool kv = k < d.nv;
  T vx = kv ? dvx<T>(d, k) : T(0), vy = kv ? dvy<T>(d, k) : T(0);
  tile_meta<T>(d, S, bi, off, i0, j0);
  __syncthreads();
  tile_load_f<T, FB>(d, S, k, kv, vx, vy);
  __syncthreads();
  T *Pw = reinterpret_cast<T *>(smraw + TileSmem<T>::bytes() + sizeof(T2) * TX * TY * VK) +
          (size_t)w * (TX + 1) * NFP;
  const T *fparT_base = reinterpret_cast<const T *>(d.fparT);
  int my_kind, my_L;
  // i-faces of tile row w
  {
    int ty = w, j = j0 + ty;
    int my_fid = lane <= TX ? tile_face_id(d, 0, off, ni, nj, i0, j0, w, lane) : -1;
    tile_stage_faces<T, NFP>(d, fparT_base, my_fid, my_kind, my_L, Pw, lane);
    T2 carry = {T(0), T(0)};
    if (j < nj) {
      for (int x = 0; x <= TX; ++x) {
        int i = i0 + x;
        if (i > ni) break;
        int kind = __shfl_sync(0xffffffffu, my_kind, x);
        int Lg = __shfl_sync(0xffffffffu, my_L, x);
        int A = (x + 1) + (ty + 2) * RW, B = A + 1;
        bool lin = x >= 1, rin = x < TX && i < ni;
        bool need = (lin && cell_status(S, A) == ST_FIELD) || (rin && cell_status(S, B) == ST_FIELD);
        V2<T> F = {T(0), T(0)};
        if (need && kv) {
          F = tile_face_flux<T>(d, S, Pw + (size_t)x * NFP, kind, Lg, A, B, lane, vx, vy);
          T sA = (S.gid[A] == Lg) ? T(1) : T(-1);
          if (lin) { carry.x += sA * F.h; carry.y += sA * F.b; }
          if (lin) Ds[(ty * TX + x - 1) * VK + lane] = carry;
          carry.x = -sA * F.h;     // the other side sees the opposite orientation
          carry.y = -sA * F.b;
        } else {
          if (lin) Ds[(ty * TX + x - 1) * VK + lane] = carry;
          carry.x = T(0);
          carry.y = T(0);
        }
      }
    }
  }
  __syncthreads();
  // j-faces of tile column w
  {
    int tx = w, i = i0 + tx;
    int my_fid = lane <= TY ? tile_face_id(d, 1, off, ni, nj, i0, j0, w, lane) : -1;
    tile_stage_faces<T, NFP>(d, fparT_base, my_fid, my_kind, my_L, Pw, lane);
    if (i < ni) {
      for (int y = 0; y <= TY; ++y) {
        int j = j0 + y;
        if (j > nj) break;
        int kind = __shfl_sync(0xffffffffu, my_kind, y);
        int Lg = __shfl_sync(0xffffffffu, my_L, y);
        int A = (tx + 2) + (y + 1) * RW, B = A + RW;
        bool lin = y >= 1, rin = y < TY && j < nj;
        bool need = (lin && cell_status(S, A) == ST_FIELD) || (rin && cell_status(S, B) == ST_FIELD);
        if (!(need && kv)) continue;
        V2<T> F = tile_face_flux<T>(d, S, Pw + (size_t)y * NFP, kind, Lg, A, B, lane, vx, vy);
        T sA = (S.gid[A] == Lg) ? T(1) : T(-1);
        if (lin) {
          T2 &q = Ds[((y - 1) * TX + tx) * VK + lane];
          q.x += sA * F.h;
          q.y += sA * F.b;
        }
        if (rin) {
          T2 &q = Ds[(y * TX + tx) * VK + lane];
          q.x -= sA * F.h;
          q.y -= sA * F.b;
        }
      }
    }
  }
  __syncthreads();
  // flux divergence of the tile cells of row w
  if (!kv) return;
  int ty = w, j = j0 + ty;
  if (j >= nj) return;
  for (int x = 0; x < TX; ++x) {
    int i = i0 + x;
    if (i >= ni) break;
    int r = (x + 2) + (ty + 2) * RW;
    if (cell_status(S, r) != ST_FIELD) continue;
    T2 D = Ds[(ty * TX + x) * VK + lane];
    stf<T>(d.Dbuf, (size_t)S.gid[r] * d.nvp + k, D.x, D.y);
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
  T idt = sizeof(T) == 4 ? (T)d.idt_f : (T)d.idt;
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

// --------------------------------------------------------- face reduction
// One CTA per (tile, 32-velocity chunk), like the residual kernel.  Each tile
// owns the i-faces on the low side of its cells (plus the block's closing
// face of a non-periodic block when the tile reaches it) and the j-faces on
// the low side of its cells (plus the closing face).  Per owned face the 12
// velocity sums of the chunk are reduced across the warp in the arithmetic
// type (butterfly, every lane ends with the totals) and lane m adds total m
// to the FP64 face sums with an atomic.
template <typename T, int FB> __global__ void __launch_bounds__(TTHREADS) k_face_reduce_tile(Dev d) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TileSmem<T> S;
  S.carve(smraw);
  int tile = blockIdx.x % d.ntiles, vc = blockIdx.x / d.ntiles;
  int b = d.tiles[3 * tile], i0 = d.tiles[3 * tile + 1], j0 = d.tiles[3 * tile + 2];
  const int *bi = d.blk_info + 8 * b;
  int ni = bi[0], nj = bi[1], per = bi[2], off = d.cell_off[b];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int k = vc * VK + lane;
  bool kv = k < d.nv;
  T vx = kv ? dvx<T>(d, k) : T(0), vy = kv ? dvy<T>(d, k) : T(0);
  tile_meta<T>(d, S, bi, off, i0, j0);
  __syncthreads();
  tile_load_f<T, FB>(d, S, k, kv, vx, vy);
  __syncthreads();
  T wk = kv ? dw<T>(d, k) : T(0);
  T v2 = T(0.5) * (vx * vx + vy * vy);
  T *Gw = reinterpret_cast<T *>(smraw + TileSmem<T>::bytes()) + (size_t)w * (TX + 1) * NFG;
  const T *fgeo = reinterpret_cast<const T *>(d.fgeo);
  for (int dir = 0; dir < 2; ++dir) {
    // dir 0: i-faces of tile row w; dir 1: j-faces of tile column w.  Lane x
    // stages face x: id, kind, left cell, whether a field cell touches it,
    // and its geometry record.
    int my_fid = lane <= TX ? tile_face_id(d, dir, off, ni, nj, i0, j0, w, lane) : -1;
    if (my_fid >= 0) {
      int i = dir == 0 ? i0 + lane : i0 + w, j = dir == 0 ? j0 + w : j0 + lane;
      bool own = dir == 0 ? ((i < ni && lane < TX) || (!per && i == ni))   // closing face of a ragged tile too
                          : ((j < nj && lane < TY) || j == nj);
      if (!own) my_fid = -1;
    }
    int my_need = 0;
    if (my_fid >= 0) {
      int Lg = d.face_L[my_fid], Rg = d.face_R[my_fid];
      my_need = d.status[Lg] == ST_FIELD || (Rg >= 0 && d.status[Rg] == ST_FIELD);
      if (!my_need) my_fid = -1;
    }
    int my_kind, my_L;
    tile_stage_faces<T, NFG>(d, fgeo, my_fid, my_kind, my_L, Gw, lane);
    for (int x = 0; x <= (dir == 0 ? TX : TY); ++x) {
      int fid = __shfl_sync(0xffffffffu, my_fid, x);
      int kind = __shfl_sync(0xffffffffu, my_kind, x);
      int Lg = __shfl_sync(0xffffffffu, my_L, x);
      if (fid < 0 || kind == BC_OVERSET) continue;
      int A, B;
      if (dir == 0) { A = (x + 1) + (w + 2) * RW; B = A + 1; }
      else { A = (w + 2) + (x + 1) * RW; B = A + RW; }
      T sums[NFS];
#pragma unroll
      for (int m = 0; m < NFS; ++m) sums[m] = T(0);
      bool wall = kind == BC_WALL;
      if (kv) {
        __align__(16) T G[NFG];
#pragma unroll
        for (int q = 0; q < (int)(NFG * sizeof(T) / 16); ++q)
          reinterpret_cast<float4 *>(G)[q] = reinterpret_cast<const float4 *>(Gw + (size_t)x * NFG)[q];
        T wS = vx * G[FG_SNX] + vy * G[FG_SNY] - G[FG_SUN];
        if (!wall || wS > T(0)) {
          T Pg[NFP];
          Pg[FP_UFX] = G[FG_UFX];
          Pg[FP_UFY] = G[FG_UFY];
          Pg[FP_DXLX] = G[FG_DXLX];
          Pg[FP_DXLY] = G[FG_DXLY];
          Pg[FP_DXRX] = G[FG_DXRX];
          Pg[FP_DXRY] = G[FG_DXRY];
          int Lr = (S.gid[A] == Lg) ? A : B;
          int Rr = (Lr == A) ? B : A;
          V2<T> ff, wg;
          tile_upwind<T>(d, S, Pg, kind, Lr, Rr, lane, vx, vy, wS, ff, wg);
          T p[4] = {wk * ff.h, wk * vx * ff.h, wk * vy * ff.h, wk * (v2 * ff.h + T(0.5) * ff.b)};
          T g[4] = {wk * wg.h, wk * vx * wg.h, wk * vy * wg.h, wk * (v2 * wg.h + T(0.5) * wg.b)};
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            sums[FS_W0 + m] = wall ? T(0) : p[m];
            sums[FS_FF + m] = wS * p[m];
            sums[FS_WG + m] = wS * g[m];
          }
        }
      }
      // transposed butterfly: 16 slots (12 used) halve at every level, so
      // 16 shuffles replace 12 x 5; lane pairs end with the total of slot
      // 8 b4 + 4 b3 + 2 b2 + b1 (b_n = bit n of the lane)
      T v16[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) v16[m] = m < NFS ? sums[m] : T(0);
#pragma unroll
      for (int half = 8; half >= 1; half >>= 1) {
        bool up = lane & (2 * half);
#pragma unroll
        for (int q = 0; q < half; ++q) {
          T send = up ? v16[q] : v16[q + half];
          T keep = up ? v16[q + half] : v16[q];
          v16[q] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * half);
        }
      }
      v16[0] += __shfl_xor_sync(0xffffffffu, v16[0], 1);
      int slotm = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
      if (!(lane & 1) && slotm < NFS) atomicAdd(&d.fsum[NFS * fid + slotm], to_double(v16[0]));
    }
  }
}

template <typename T> static size_t rhs_smem() {
  return TileSmem<T>::bytes() + sizeof(typename Vec2<T>::type) * TX * TY * VK +
         sizeof(T) * (TTHREADS / 32) * (TX + 1) * NFP;
}
template <typename T> static size_t reduce_smem() {
  return TileSmem<T>::bytes() + sizeof(T) * (TTHREADS / 32) * (TX + 1) * NFG;
}

void tile_setup() {
  cudaFuncSetAttribute(k_flux_tile<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<float>());
  cudaFuncSetAttribute(k_flux_tile<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<float>());
  cudaFuncSetAttribute(k_flux_tile<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_smem<double>());
  cudaFuncSetAttribute(k_face_reduce_tile<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)reduce_smem<float>());
  cudaFuncSetAttribute(k_face_reduce_tile<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)reduce_smem<float>());
  cudaFuncSetAttribute(k_face_reduce_tile<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)reduce_smem<double>());
}

int tile_count(int ni, int nj) { return ((ni + TX - 1) / TX) * ((nj + TY - 1) / TY); }
void tile_origins(int ni, int nj, int *out) {   // (i0, j0) pairs
  int q = 0;
  for (int tj = 0; tj < (nj + TY - 1) / TY; ++tj)
    for (int ti = 0; ti < (ni + TX - 1) / TX; ++ti) { out[q++] = ti * TX; out[q++] = tj * TY; }
}

void launch_flux_tile(const Dev &d, cudaStream_t s, int fp32) {
  int nchunks = (d.nv + VK - 1) / VK;
  int grid = d.ntiles * nchunks;
  if (fp32 && d.fbf) k_flux_tile<float, 1><<<grid, TTHREADS, rhs_smem<float>(), s>>>(d);
  else if (fp32) k_flux_tile<float, 0><<<grid, TTHREADS, rhs_smem<float>(), s>>>(d);
  else k_flux_tile<double, 0><<<grid, TTHREADS, rhs_smem<double>(), s>>>(d);
}
void launch_residual(const Dev &d, cudaStream_t s, int first_iter, int fp32) {
  int pairs = (d.nv + 1) / 2;
  int bt = pairs >= 256 ? 256 : ((pairs + 31) / 32) * 32;
  dim3 grid(d.nc, (pairs + bt - 1) / bt);
  if (fp32 && d.fbf) k_residual<float, 1><<<grid, bt, 0, s>>>(d, first_iter);
  else if (fp32) k_residual<float, 0><<<grid, bt, 0, s>>>(d, first_iter);
  else k_residual<double, 0><<<grid, bt, 0, s>>>(d, first_iter);
}

void launch_face_reduce_tile(const Dev &d, cudaStream_t s, int fp32) {
  int nchunks = (d.nv + VK - 1) / VK;
  cudaMemsetAsync(d.fsum, 0, sizeof(double) * NFS * (size_t)d.nf, s);
  int grid = d.ntiles * nchunks;
  if (fp32 && d.fbf) k_face_reduce_tile<float, 1><<<grid, TTHREADS, reduce_smem<float>(), s>>>(d);
  else if (fp32) k_face_reduce_tile<float, 0><<<grid, TTHREADS, reduce_smem<float>(), s>>>(d);
  else k_face_reduce_tile<double, 0><<<grid, TTHREADS, reduce_smem<double>(), s>>>(d);
}

}  // namespace ugks
