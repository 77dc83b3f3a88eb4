// ugks_overset.cu -- overset assembly (arXiv 2604.09984 Sec. 3.1) and
// inverse-distance interpolation (Sec. 3.2) on the device.
//
// Every geometric predicate uses explicit round-to-nearest FP64 operations
// (__dadd_rn, __dmul_rn, ...) so no multiply-add is contracted: the result is
// bit-identical to a plain FP64 evaluation of the same expressions in the
// same order.  Readings of the garbled classification sentence of Sec. 3.1:
//   * wall distance of a node to a zone: min squared distance to the zone's
//     wall segments (+inf without walls);
//   * a node of zone Z is inactive if it lies inside another zone's body
//     polygon, or inside a core cell (not within n_fringe + n_gap layers of an
//     overset edge) of a zone D with a smaller wall distance (ties: higher
//     priority wins);
//   * cells: all nodes inactive -> hole, mixed -> boundary, fringe layers ->
//     receptor; active face neighbours of boundary or hole cells form the
//     buffer layer (receptors); the rest are field cells;
//   * donor: the containing cell of another zone, field cells before
//     receptor cells, then (priority desc, block, cell index); stencil =
//     donor + its non-hole face neighbours (order i-1, i+1, j-1, j+1),
//     weights d^-2 normalised in that order (Sec. 3.2).
//
// The FP64 predicates decide everything; float filters in front of them only
// skip work whose outcome they already know exactly: with rn() the
// round-to-nearest map to float (monotone), rn(a) > rn(b) implies a > b.
#include <algorithm>

#include "ugks_internal.cuh"
#include "ugks_launch.h"

namespace ugks {

enum { CL_ACTIVE = 0, CL_MIXED = 1, CL_HOLE = 2, CL_FRINGE = 3 };

__device__ __forceinline__ double ad(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sb(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ml(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dv(double a, double b) { return __ddiv_rn(a, b); }

// squared distance of (x, y) to wall segment s (exact FP64 expression)
__device__ __forceinline__ double seg_dist2(const Dev &d, int s, double x, double y) {
  int a = d.wall_seg[2 * s], b = d.wall_seg[2 * s + 1];
  double ax = d.X_new[2 * a], ay = d.X_new[2 * a + 1];
  double ex = sb(d.X_new[2 * b], ax), ey = sb(d.X_new[2 * b + 1], ay);
  double px = sb(x, ax), py = sb(y, ay);
  double t = dv(ad(ml(px, ex), ml(py, ey)), ad(ml(ex, ex), ml(ey, ey)));
  t = fmin(fmax(t, 0.0), 1.0);
  double dx = sb(px, ml(t, ex)), dy = sb(py, ml(t, ey));
  return ad(ml(dx, dx), ml(dy, dy));
}

// Minimum squared distance to the zone's wall segments (+inf without).
// A float pass picks a near segment, whose exact distance bounds the
// minimum; then only segments whose float lower bound (distance to their
// bounding box, shrunk by the float rounding of the coordinates and
// scaled down) does not exceed that bound are evaluated exactly.  The
// skipped ones are farther than the minimum, so the result is the exact
// minimum over all segments.
// `seg` holds the float endpoints (A.x, A.y, B.x, B.y) of every segment
// (shared memory, or the global copy when they do not fit there).
__device__ double wall_dist2(const Dev &d, const float4 *seg, int blk, double x, double y) {
  double best = __longlong_as_double(0x7ff0000000000000LL);   // +inf
  int s0 = d.wall_seg_off[blk], s1 = d.wall_seg_off[blk + 1];
  if (s1 <= s0) return best;
  float xf = __double2float_rn(x), yf = __double2float_rn(y);
  int sg = s0;
  float gbest = __int_as_float(0x7f800000);
  for (int s = s0; s < s1; ++s) {
    float4 AB = seg[s];
    float2 A = make_float2(AB.x, AB.y), B = make_float2(AB.z, AB.w);
    float ex = B.x - A.x, ey = B.y - A.y, px = xf - A.x, py = yf - A.y;
    float ee = ex * ex + ey * ey;
    float t = ee > 0.f ? fminf(fmaxf((px * ex + py * ey) / ee, 0.f), 1.f) : 0.f;
    float dx = px - t * ex, dy = py - t * ey, g = dx * dx + dy * dy;
    if (g < gbest) { gbest = g; sg = s; }
  }
  best = seg_dist2(d, sg, x, y);
  float bestf = __double2float_ru(best);
  for (int s = s0; s < s1; ++s) {
    if (s == sg) continue;
    float4 AB = seg[s];
    float2 A = make_float2(AB.x, AB.y), B = make_float2(AB.z, AB.w);
    float lx = fminf(A.x, B.x), hx = fmaxf(A.x, B.x), ly = fminf(A.y, B.y), hy = fmaxf(A.y, B.y);
    float tol = 2.4e-7f * (fabsf(xf) + fabsf(yf) + fabsf(lx) + fabsf(hx) + fabsf(ly) + fabsf(hy));
    float gx = fmaxf(fmaxf(lx - xf, xf - hx) - tol, 0.f);
    float gy = fmaxf(fmaxf(ly - yf, yf - hy) - tol, 0.f);
    float lb = (gx * gx + gy * gy) * 0.99999f;
    if (lb > bestf) continue;
    double d2 = seg_dist2(d, s, x, y);
    if (d2 < best) { best = d2; bestf = __double2float_ru(best); }
  }
  return best;
}

// Bracket of the same minimum without its exact evaluation over every
// candidate: hi = the exact distance of the float-nearest segment (an upper
// bound), lo = the smallest float lower bound over all segments (rounded
// so that lo <= every exact segment distance).  Both +inf without walls.
__device__ void wall_dist2_bounds(const Dev &d, const float4 *seg, int blk, double x, double y,
                                  double &lo, double &hi) {
  lo = hi = __longlong_as_double(0x7ff0000000000000LL);
  int s0 = d.wall_seg_off[blk], s1 = d.wall_seg_off[blk + 1];
  if (s1 <= s0) return;
  float xf = __double2float_rn(x), yf = __double2float_rn(y);
  int sg = s0;
  float gbest = __int_as_float(0x7f800000), lbmin = __int_as_float(0x7f800000);
  for (int s = s0; s < s1; ++s) {
    float4 AB = seg[s];
    float ex = AB.z - AB.x, ey = AB.w - AB.y, px = xf - AB.x, py = yf - AB.y;
    float ee = ex * ex + ey * ey;
    float t = ee > 0.f ? fminf(fmaxf((px * ex + py * ey) / ee, 0.f), 1.f) : 0.f;
    float dx = px - t * ex, dy = py - t * ey, g = dx * dx + dy * dy;
    if (g < gbest) { gbest = g; sg = s; }
    float lx = fminf(AB.x, AB.z), hx = fmaxf(AB.x, AB.z), ly = fminf(AB.y, AB.w), hy = fmaxf(AB.y, AB.w);
    float tol = 2.4e-7f * (fabsf(xf) + fabsf(yf) + fabsf(lx) + fabsf(hx) + fabsf(ly) + fabsf(hy));
    float gx = fmaxf(fmaxf(lx - xf, xf - hx) - tol, 0.f);
    float gy = fmaxf(fmaxf(ly - yf, yf - hy) - tol, 0.f);
    lbmin = fminf(lbmin, (gx * gx + gy * gy) * 0.99999f);
  }
  hi = seg_dist2(d, sg, x, y);
  lo = (double)lbmin;
}

__device__ bool inside_quad(const Dev &d, int c, double x, double y) {
  const int *nd = d.cell_nodes + 4 * c;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int a = nd[e], b = nd[(e + 1) & 3];
    double ax = d.X_new[2 * a], ay = d.X_new[2 * a + 1];
    double bx = d.X_new[2 * b], by = d.X_new[2 * b + 1];
    double cr = sb(ml(sb(bx, ax), sb(y, ay)), ml(sb(by, ay), sb(x, ax)));
    if (!(cr >= 0.0)) return false;
  }
  return true;
}

// Float box of each block's body polygon, rounded outward (one warp per
// block): a point outside it is outside the polygon.
__global__ void k_body_box(Dev d) {
  int b = blockIdx.x, lane = threadIdx.x;
  int r0 = d.body_ring_off[b], r1 = d.body_ring_off[b + 1];
  double xl = 1e300, xh = -1e300, yl = 1e300, yh = -1e300;
  for (int i = r0 + lane; i < r1; i += 32) {
    int a = d.body_ring[i];
    double x = d.X_new[2 * a], y = d.X_new[2 * a + 1];
    xl = fmin(xl, x); xh = fmax(xh, x); yl = fmin(yl, y); yh = fmax(yh, y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    xl = fmin(xl, __shfl_xor_sync(0xffffffffu, xl, o));
    xh = fmax(xh, __shfl_xor_sync(0xffffffffu, xh, o));
    yl = fmin(yl, __shfl_xor_sync(0xffffffffu, yl, o));
    yh = fmax(yh, __shfl_xor_sync(0xffffffffu, yh, o));
  }
  if (lane == 0)
    d.body_bb[b] = make_float4(__double2float_rd(xl), __double2float_rd(yl), __double2float_ru(xh),
                               __double2float_ru(yh));
}

__device__ bool inside_body(const Dev &d, int blk, double x, double y) {
  float4 bb = d.body_bb[blk];
  if (x < (double)bb.x || x > (double)bb.z || y < (double)bb.y || y > (double)bb.w) return false;
  int r0 = d.body_ring_off[blk], r1 = d.body_ring_off[blk + 1];
  int M = r1 - r0;
  bool in = false;
  float yf = __double2float_rn(y);
  for (int i = 0; i < M; ++i) {
    int a = d.body_ring[r0 + i], b = d.body_ring[r0 + (i + 1 < M ? i + 1 : 0)];
    // side of y for each end from the floats where they differ, else exactly
    float af = d.Xf[a].y, bf = d.Xf[b].y;
    int sa = af > yf ? 1 : (af < yf ? -1 : 0), sbv = bf > yf ? 1 : (bf < yf ? -1 : 0);
    if (sa != 0 && sa == sbv) continue;                   // both above or both below
    double ax = d.X_new[2 * a], ay = d.X_new[2 * a + 1];
    double bx = d.X_new[2 * b], by = d.X_new[2 * b + 1];
    bool crosses = (ay > y) != (by > y);
    if (crosses) {
      double xint = ad(ax, dv(ml(sb(y, ay), sb(bx, ax)), sb(by, ay)));
      if (x < xint) in = !in;
    }
  }
  return in;
}

__device__ __forceinline__ bool in_layer(const int *bi, int i, int j, int L) {
  int ni = bi[0], nj = bi[1], mask = bi[6];
  if ((mask & 1) && i < L) return true;
  if ((mask & 2) && i >= ni - L) return true;
  if ((mask & 4) && j < L) return true;
  if ((mask & 8) && j >= nj - L) return true;
  return false;
}

// ---------------------------------------------------------------- bins
// Per block a uniform grid of bins over a box containing the block at
// t^{n+1}; every cell is registered in the bins its bounding box overlaps.
// A point lies in the bin (floor((x-x0)/hx), floor((y-y0)/hy)); a cell that
// contains the point overlaps that bin (floor is monotone), so the minimum
// index among the bin's candidates that contain the point equals the minimum
// over all cells: same result as a scan of the whole block.
__device__ __forceinline__ void bin_range(const Dev &d, int b, double lo, double hi, int axis,
                                          int &i0, int &i1) {
  const double *g = d.bin_geo + 4 * b;
  int n = d.bin_dim[3 * b + axis];
  double x0 = g[axis], ih = g[2 + axis];
  double a = floor((lo - x0) * ih), c = floor((hi - x0) * ih);
  i0 = a < 0.0 ? 0 : (a > n - 1 ? n - 1 : (int)a);
  i1 = c < 0.0 ? 0 : (c > n - 1 ? n - 1 : (int)c);
}

__device__ __forceinline__ int bin_of(const Dev &d, int b, double x, double y) {
  const double *g = d.bin_geo + 4 * b;
  int nx = d.bin_dim[3 * b], ny = d.bin_dim[3 * b + 1];
  double a = floor((x - g[0]) * g[2]), c = floor((y - g[1]) * g[3]);
  if (a < 0.0 || c < 0.0 || a > nx - 1 || c > ny - 1) return -1;
  return d.bin_dim[3 * b + 2] + (int)c * nx + (int)a;
}

__global__ void k_node_f(Dev d) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < d.nn)
    d.Xf[n] = make_float2(__double2float_rn(d.X_new[2 * n]), __double2float_rn(d.X_new[2 * n + 1]));
  if (n < d.nseg) {      // float endpoints of wall segment n, one record each
    int a = d.wall_seg[2 * n], b = d.wall_seg[2 * n + 1];
    d.segf[n] = make_float4(__double2float_rn(d.X_new[2 * a]), __double2float_rn(d.X_new[2 * a + 1]),
                            __double2float_rn(d.X_new[2 * b]), __double2float_rn(d.X_new[2 * b + 1]));
  }
}

__global__ void k_bin_count(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  int b = d.cell_block[c];
  const int *nd = d.cell_nodes + 4 * c;
  double xl = d.X_new[2 * nd[0]], xh = xl, yl = d.X_new[2 * nd[0] + 1], yh = yl;
  for (int v = 1; v < 4; ++v) {
    double x = d.X_new[2 * nd[v]], y = d.X_new[2 * nd[v] + 1];
    xl = fmin(xl, x); xh = fmax(xh, x); yl = fmin(yl, y); yh = fmax(yh, y);
  }
  d.cbb[c] = make_float4(__double2float_rd(xl), __double2float_rd(yl), __double2float_ru(xh),
                         __double2float_ru(yh));
  int ix0, ix1, iy0, iy1;
  bin_range(d, b, xl, xh, 0, ix0, ix1);
  bin_range(d, b, yl, yh, 1, iy0, iy1);
  int nx = d.bin_dim[3 * b], base = d.bin_dim[3 * b + 2];
  for (int iy = iy0; iy <= iy1; ++iy)
    for (int ix = ix0; ix <= ix1; ++ix) atomicAdd(&d.bin_cnt[base + iy * nx + ix], 1);
}

// exclusive scan of the bin counts (one CTA), cursor = start
__global__ void k_bin_scan(Dev d) {
  __shared__ int part[1024];
  int n = d.nbins;
  int per = (n + blockDim.x - 1) / blockDim.x;
  int lo = threadIdx.x * per, hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += d.bin_cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) { int v = part[t]; part[t] = run; run += v; }
    d.bin_start[n] = run;
    if (run > d.bin_cap) atomicOr(d.err, EF_BINS);
  }
  __syncthreads();
  int run = part[threadIdx.x];
  for (int i = lo; i < hi; ++i) {
    int v = d.bin_cnt[i];
    d.bin_start[i] = run;
    d.bin_cnt[i] = run;            // reused as the fill cursor
    run += v;
  }
}

__global__ void k_bin_fill(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  int b = d.cell_block[c];
  const int *nd = d.cell_nodes + 4 * c;
  double xl = d.X_new[2 * nd[0]], xh = xl, yl = d.X_new[2 * nd[0] + 1], yh = yl;
  for (int v = 1; v < 4; ++v) {
    double x = d.X_new[2 * nd[v]], y = d.X_new[2 * nd[v] + 1];
    xl = fmin(xl, x); xh = fmax(xh, x); yl = fmin(yl, y); yh = fmax(yh, y);
  }
  int ix0, ix1, iy0, iy1;
  bin_range(d, b, xl, xh, 0, ix0, ix1);
  bin_range(d, b, yl, yh, 1, iy0, iy1);
  int nx = d.bin_dim[3 * b], base = d.bin_dim[3 * b + 2];
  for (int iy = iy0; iy <= iy1; ++iy)
    for (int ix = ix0; ix <= ix1; ++ix) {
      int pos = atomicAdd(&d.bin_cnt[base + iy * nx + ix], 1);
      if (pos < d.bin_cap) d.bin_items[pos] = c;
    }
}

// lowest-index cell of block b containing (x, y) among the cells accepted by
// `ok` (bins guarantee the same answer as a scan of the block)
template <typename Pred>
__device__ int first_containing(const Dev &d, int b, double x, double y, Pred ok) {
  int bin = bin_of(d, b, x, y);
  if (bin < 0) return -1;
  int best = 0x7fffffff;
  float xf = __double2float_rn(x), yf = __double2float_rn(y);
  int q1 = min(d.bin_start[bin + 1], d.bin_cap);
  for (int q = d.bin_start[bin]; q < q1; ++q) {
    int c = d.bin_items[q];
    if (c >= best) continue;
    float4 bb = d.cbb[c];                       // the cell lies inside its box
    if (xf < bb.x || xf > bb.z || yf < bb.y || yf > bb.w) continue;
    if (ok(c) && inside_quad(d, c, x, y)) best = c;
  }
  return best == 0x7fffffff ? -1 : best;
}

// node classification (one thread per node); the wall segments' float
// records are staged in shared memory when they fit (STAGE)
template <bool STAGE> __global__ void k_node_classify(Dev d) {
  extern __shared__ float4 seg_s[];
  if (STAGE) {
    for (int q = threadIdx.x; q < d.nseg; q += blockDim.x) seg_s[q] = d.segf[q];
    __syncthreads();
  }
  const float4 *seg = STAGE ? seg_s : d.segf;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.nn) return;
  int z = d.node_block[n];
  double x = d.X_new[2 * n], y = d.X_new[2 * n + 1];
  // the node's own wall distance is needed only where another zone's core
  // contains it (most background nodes lie in no other zone), and exactly
  // only where the brackets of the two distances overlap: elsewhere the
  // brackets already decide db < dz (or db > dz) as the exact values would
  double dz = 0.0, zlo = 0.0, zhi = 0.0;
  bool have_z = false, have_dz = false;
  bool inact = false;
  for (int b = 0; b < d.nblocks && !inact; ++b) {
    if (b == z) continue;
    if (d.body_ring_off[b + 1] > d.body_ring_off[b] && inside_body(d, b, x, y)) {
      inact = true;
      break;
    }
    const int *bi = d.blk_info + 8 * b;
    int ni = bi[0], L = bi[4] + bi[5];
    int c0 = d.cell_off[b];
    bool hit = first_containing(d, b, x, y, [&](int c) {
      int loc = c - c0;
      return !in_layer(bi, loc % ni, loc / ni, L);
    }) >= 0;
    if (hit) {
      if (!have_z) {
        wall_dist2_bounds(d, seg, z, x, y, zlo, zhi);
        have_z = true;
      }
      double blo, bhi;
      wall_dist2_bounds(d, seg, b, x, y, blo, bhi);
      if (bhi < zlo) {                  // db <= bhi < zlo <= dz
        inact = true;
      } else if (!(blo > zhi)) {        // brackets overlap: exact values
        if (!have_dz) {
          dz = wall_dist2(d, seg, z, x, y);
          have_dz = true;
        }
        double db = wall_dist2(d, seg, b, x, y);
        const int *bz = d.blk_info + 8 * z;
        if (db < dz || (db == dz && bi[3] > bz[3])) inact = true;
      }                                 // else db >= blo > zhi >= dz: stays active
    }
  }
  d.node_active[n] = inact ? 0 : 1;
}

__global__ void k_cell_classify(Dev d) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  const int *nd = d.cell_nodes + 4 * c;
  int na = d.node_active[nd[0]] + d.node_active[nd[1]] + d.node_active[nd[2]] + d.node_active[nd[3]];
  int b = d.cell_block[c];
  const int *bi = d.blk_info + 8 * b;
  int loc = c - d.cell_off[b];
  int i = loc % bi[0], j = loc / bi[0];
  int cl;
  if (na == 0) cl = CL_HOLE;
  else if (na < 4) cl = CL_MIXED;
  else if (in_layer(bi, i, j, bi[4])) cl = CL_FRINGE;
  else cl = CL_ACTIVE;
  d.cls[c] = cl;
}

// status from the classes; buffer layer; fresh cells (hole -> field) flagged
// with bit 8 of prev_status scratch
__global__ void k_cell_buffer(Dev d, int *prev_status) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  int cl = d.cls[c];
  int st;
  if (cl == CL_HOLE) st = ST_HOLE;
  else if (cl == CL_MIXED || cl == CL_FRINGE) st = ST_RECEPTOR;
  else {
    st = ST_FIELD;
    for (int s = 0; s < 4; ++s) {
      if (d.nb_kind[4 * c + s] != NB_CELL) continue;
      int nc2 = d.cls[d.nb_id[4 * c + s]];
      if (nc2 == CL_MIXED || nc2 == CL_HOLE) st = ST_RECEPTOR;
    }
  }
  int prev = prev_status[c];
  prev_status[c] = (prev == ST_HOLE && st == ST_FIELD) ? 1 : 0;   // fresh flag
  d.status[c] = st;
}

// donor search and IDW weights for receptor / fresh cells
__global__ void k_donor(Dev d, const int *fresh_flag, const int *blk_order, int *n_orphan) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.nc) return;
  int st = d.status[c];
  for (int m = 0; m < 5; ++m) { d.donors[5 * c + m] = -1; d.dwgt[5 * c + m] = 0.0; }
  if (st != ST_RECEPTOR && !fresh_flag[c]) return;
  double x = d.xc_new[2 * c], y = d.xc_new[2 * c + 1];
  int own = d.cell_block[c];
  int found = -1;
  for (int cls = ST_FIELD; cls <= ST_RECEPTOR && found < 0; ++cls) {
    for (int o = 0; o < d.nblocks && found < 0; ++o) {
      int b = blk_order[o];
      if (b == own) continue;
      int e = first_containing(d, b, x, y, [&](int q) { return d.status[q] == cls; });
      if (e >= 0) found = e;
    }
  }
  if (found < 0) {
    atomicAdd(n_orphan, 1);
    return;
  }
  int stn[5];
  int ns = 0;
  stn[ns++] = found;
  for (int s = 0; s < 4; ++s) {
    if (d.nb_kind[4 * found + s] != NB_CELL) continue;
    int e = d.nb_id[4 * found + s];
    if (d.status[e] != ST_HOLE) stn[ns++] = e;
  }
  double d2[5];
  int zero = -1;
  for (int m = 0; m < ns; ++m) {
    double ex = sb(x, d.xc_new[2 * stn[m]]), ey = sb(y, d.xc_new[2 * stn[m] + 1]);
    d2[m] = ad(ml(ex, ex), ml(ey, ey));
    if (d2[m] == 0.0 && zero < 0) zero = m;
  }
  for (int m = 0; m < ns; ++m) d.donors[5 * c + m] = stn[m];
  if (zero >= 0) {
    d.dwgt[5 * c + zero] = 1.0;
    return;
  }
  double inv[5], tot = 0.0;
  for (int m = 0; m < ns; ++m) inv[m] = dv(1.0, d2[m]);
  for (int m = 0; m < ns; ++m) tot = ad(tot, inv[m]);
  for (int m = 0; m < ns; ++m) d.dwgt[5 * c + m] = dv(inv[m], tot);
}

// Receptor and fresh-cell lists, compacted on the device in ascending cell
// order (two passes over 1024-cell chunks: count, then scan and write), so
// that no host round trip sits between the assembly and the step.
constexpr int LCHUNK = 1024;

__global__ void __launch_bounds__(LCHUNK) k_list_count(Dev d, const int *fresh_flag) {
  int c = blockIdx.x * LCHUNK + threadIdx.x;
  bool in = c < d.nc;
  int st = in ? d.status[c] : -1;
  int nr = __syncthreads_count(in && st == ST_RECEPTOR);
  int nfr = __syncthreads_count(in && fresh_flag[c] != 0);
  int nfd = __syncthreads_count(in && st == ST_FIELD);
  int no = __syncthreads_count(in && st != ST_FIELD && st != ST_RECEPTOR);
  if (threadIdx.x == 0) d.conn_chunk[blockIdx.x] = make_int4(nr, nfr, nfd, no);
}

__global__ void __launch_bounds__(LCHUNK) k_list_write(Dev d, const int *fresh_flag, const int *n_orphan) {
  __shared__ int base[2];
  __shared__ int wcnt[2][LCHUNK / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w == 0) {   // offsets of this chunk: totals of the earlier chunks
    int a = 0, b = 0;
    for (int q = lane; q < (int)blockIdx.x; q += 32) {
      int4 v = d.conn_chunk[q];
      a += v.x;
      b += v.y;
    }
    for (int o = 16; o >= 1; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { base[0] = a; base[1] = b; }
  }
  int c = blockIdx.x * LCHUNK + threadIdx.x;
  bool in = c < d.nc;
  bool isr = in && d.status[c] == ST_RECEPTOR;
  bool isf = in && fresh_flag[c] != 0;
  unsigned mr = __ballot_sync(0xffffffffu, isr), mf = __ballot_sync(0xffffffffu, isf);
  if (lane == 0) { wcnt[0][w] = __popc(mr); wcnt[1][w] = __popc(mf); }
  __syncthreads();
  int orr = base[0], off = base[1];
  for (int q = 0; q < w; ++q) { orr += wcnt[0][q]; off += wcnt[1][q]; }
  unsigned below = (1u << lane) - 1u;
  int ir = orr + __popc(mr & below), jf = off + __popc(mf & below);
  if (isr && ir < d.cap_interp) d.rec_list[ir] = c;
  if (isf && jf < d.cap_interp) d.fresh_list[jf] = c;
  if (blockIdx.x == gridDim.x - 1 && w == 0) {   // totals and their checks
    int t[4] = {0, 0, 0, 0};
    for (int q = lane; q < (int)gridDim.x; q += 32) {
      int4 v = d.conn_chunk[q];
      t[0] += v.x; t[1] += v.y; t[2] += v.z; t[3] += v.w;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
      for (int o = 16; o >= 1; o >>= 1) t[m] += __shfl_xor_sync(0xffffffffu, t[m], o);
    if (lane == 0) {
      int no = *n_orphan;
      d.conn_cnt[0] = t[0]; d.conn_cnt[1] = t[1]; d.conn_cnt[2] = t[2]; d.conn_cnt[3] = t[3];
      d.conn_cnt[4] = no;
      if (t[0] > d.cap_interp || t[1] > d.cap_interp) atomicOr(d.err, EF_CAPACITY);
      if (no > 0) atomicOr(d.err, EF_ORPHAN);
    }
  }
}

// Jacobi interpolation: gather into staging, then scatter.  The list length
// is read on the device (*cnt, clamped to the staging capacity); a fixed grid
// strides over it.
// parts: bit 0 the distributions, bit 1 W and q (the two may run apart: the
// distributions right after the micro sweep, W and q after Step 7)
template <typename T> __global__ void k_interp_gather(Dev d, const int *list, const int *cnt, int parts) {
  int n = min(*cnt, d.cap_interp);
  size_t nk = (parts & 1) ? (size_t)d.nvp : 1;
  size_t tot = (size_t)n * nk;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(t / nk), k = (int)(t % nk);
    int c = list[r];
    if (parts & 1) {
      // f in the arithmetic type (its storage type): FP32 weights and sums on
      // the mixed path keep the FP64 pipe out of the per-velocity loop
      T ah = T(0), ab = T(0);
      for (int m = 0; m < 5; ++m) {
        int e = d.donors[5 * c + m];
        if (e < 0) continue;
        T w = (T)d.dwgt[5 * c + m];
        auto v = ldF<T>(d, (size_t)e * d.nvp + k);
        ah = ah + w * v.x;
        ab = ab + w * v.y;
      }
      stf<T>(d.itmp, (size_t)r * d.nvp + k, ah, ab);
    }
    if ((parts & 2) && k == 0) {
      double acc[6] = {0, 0, 0, 0, 0, 0};
      for (int m = 0; m < 5; ++m) {
        int e = d.donors[5 * c + m];
        if (e < 0) continue;
        double w = d.dwgt[5 * c + m];
        for (int q = 0; q < 4; ++q) acc[q] = acc[q] + w * d.W[4 * e + q];
        acc[4] = acc[4] + w * d.q[2 * e];
        acc[5] = acc[5] + w * d.q[2 * e + 1];
      }
      for (int q = 0; q < 6; ++q) d.itmpW[6 * r + q] = acc[q];
    }
  }
}

template <typename T> __global__ void k_interp_scatter(Dev d, const int *list, const int *cnt, int parts) {
  int n = min(*cnt, d.cap_interp);
  size_t nk = (parts & 1) ? (size_t)d.nvp : 1;
  size_t tot = (size_t)n * nk;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(t / nk), k = (int)(t % nk);
    int c = list[r];
    if (d.donors[5 * c] < 0) continue;          // orphan: keep its values
    if (parts & 1) {
      auto v = ldf<T>(d.itmp, (size_t)r * d.nvp + k);
      stF<T>(d, (size_t)c * d.nvp + k, v.x, v.y);
    }
    if ((parts & 2) && k == 0) {
      for (int q = 0; q < 4; ++q) d.W[4 * c + q] = d.itmpW[6 * r + q];
      d.q[2 * c] = d.itmpW[6 * r + 4];
      d.q[2 * c + 1] = d.itmpW[6 * r + 5];
    }
  }
}

static inline int nblk(size_t n, int b) { return (int)((n + b - 1) / b); }

void launch_connect(const Dev &d, cudaStream_t s, int *prev_status, const int *blk_order,
                    int *n_orphan) {
  cudaMemsetAsync(d.bin_cnt, 0, sizeof(int) * d.nbins, s);
  k_node_f<<<nblk(d.nn > d.nseg ? d.nn : d.nseg, 256), 256, 0, s>>>(d);
  k_body_box<<<d.nblocks, 32, 0, s>>>(d);
  k_bin_count<<<nblk(d.nc, 256), 256, 0, s>>>(d);
  k_bin_scan<<<1, 1024, 0, s>>>(d);
  k_bin_fill<<<nblk(d.nc, 256), 256, 0, s>>>(d);
  size_t segb = sizeof(float4) * (size_t)d.nseg;
  if (segb <= 48 * 1024) k_node_classify<true><<<nblk(d.nn, 128), 128, segb, s>>>(d);
  else k_node_classify<false><<<nblk(d.nn, 128), 128, 0, s>>>(d);
  k_cell_classify<<<nblk(d.nc, 256), 256, 0, s>>>(d);
  k_cell_buffer<<<nblk(d.nc, 256), 256, 0, s>>>(d, prev_status);
  k_donor<<<nblk(d.nc, 128), 128, 0, s>>>(d, prev_status, blk_order, n_orphan);
}

void launch_lists(const Dev &d, cudaStream_t s, const int *fresh_flag, const int *n_orphan) {
  int nch = nblk(d.nc, LCHUNK);
  k_list_count<<<nch, LCHUNK, 0, s>>>(d, fresh_flag);
  k_list_write<<<nch, LCHUNK, 0, s>>>(d, fresh_flag, n_orphan);
}

void launch_interp(const Dev &d, cudaStream_t s, const int *list, const int *cnt, int nsm, int fp32, int parts) {
  size_t tot = (size_t)d.cap_interp * ((parts & 1) ? d.nvp : 1);
  int grid = std::max(1, std::min(nblk(tot, 256), 8 * std::max(nsm, 1)));
  if (fp32) {
    k_interp_gather<float><<<grid, 256, 0, s>>>(d, list, cnt, parts);
    k_interp_scatter<float><<<grid, 256, 0, s>>>(d, list, cnt, parts);
  } else {
    k_interp_gather<double><<<grid, 256, 0, s>>>(d, list, cnt, parts);
    k_interp_scatter<double><<<grid, 256, 0, s>>>(d, list, cnt, parts);
  }
}

}  // namespace ugks
