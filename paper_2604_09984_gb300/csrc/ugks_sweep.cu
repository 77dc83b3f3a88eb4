// ugks_sweep.cu -- micro LU-SGS (arXiv 2604.09984 Sec. 2.2, Eq.
// dualTimeStepping_micro with the upwind flux variation): the forward sweep
// d* = (r - sum_lower c d*) / D and the backward sweep d = d* - sum_upper c d
// / D, f += d, over every block in lexicographic order (i fastest), for
// every discrete velocity independently.
//
// The sweep runs as a skewed wavefront.  A warp owns a band of ROWS rows of a
// block (QL lanes a row, VPT consecutive velocities a lane); row j of the
// band takes cell i = s - j of its row at step s, so its lower neighbour
// along the row is its own result of step s - 1 and its lower neighbour
// across rows is row j-1's result of step s - 1, fetched with a warp shuffle:
// no barrier inside a band.  Bands of one block (warps of one CTA) pass the
// last row's values to the next band through a ring in shared memory with
// progress counters (bounded waits); the next band trails by ROWS steps.  The
// QL lanes of a row prefetch the inputs of their cell (the residual / forward
// result, f, the cell's sweep record) NS - 1 steps ahead with asynchronous
// copies of consecutive 16-byte chunks into the warp's ring.  Cells of one diagonal i + j are
// independent, and lower (upper) neighbours always come from earlier steps,
// so the result is the lexicographic Gauss-Seidel exactly.
#include <cstdlib>
#include "ugks_internal.cuh"
#include "ugks_launch.h"

namespace ugks {

constexpr int WS_LR = 64;            // most ring entries between two bands (cells): the next band
                                     // trails by ROWS steps, the rest of the ring is slack; fewer
                                     // (a power of two >= 2) where shared memory is short

// A warp: ROWS = 32 / QL rows of a block, QL lanes per row, VPT velocities a
// lane (QL * VPT consecutive velocities a warp).
template <typename T, int PASS, int VPT, int FB, int QL> struct WsCfg {
  typedef typename Vec2<T>::type T2;
  static constexpr int ROWS = 32 / QL;
  static constexpr bool BF = PASS == 1 && FB == 1;                 // bf16 f in the backward pass
  static constexpr int RV = QL * VPT * (int)sizeof(T2) / 16;        // chunks of a row's values
  static constexpr int RF = PASS == 1 ? (BF ? QL * VPT * 4 / 16 : RV) : 0;   // chunks of a row's f
  static constexpr int RR = NSR * (int)sizeof(T) / 16;              // chunks of the cell record
  static constexpr int RUSED = RV + RF + RR;
  static constexpr int RS = RUSED | 1;        // row stride in the ring (odd: rows in distinct banks)
  static_assert(RV * 16 == QL * VPT * (int)sizeof(T2), "whole chunks of a row's values");
  static_assert(!BF || (QL * VPT * 4) % 16 == 0, "whole chunks of a row's bf16 values");
};

// Shared memory of a sweep CTA with nw warps and ring depth ns.
template <typename T, int PASS, int VPT, int FB, int QL>
__host__ __device__ constexpr size_t ws_smem(int nw, int ns, int lr = WS_LR) {
  typedef WsCfg<T, PASS, VPT, FB, QL> C;
  return (size_t)nw * ns * C::ROWS * C::RS * 16 +
         (size_t)nw * lr * QL * VPT * sizeof(typename Vec2<T>::type) + (size_t)nw * 2 * sizeof(int);
}

// work item: block, first velocity, velocity groups in this CTA
template <typename T, int PASS, int NS, int VPT, int FB, int QL>
__global__ void __launch_bounds__(1024) k_wsweep(Dev d, const int *work, int lr) {
  typedef typename Vec2<T>::type T2;
  typedef WsCfg<T, PASS, VPT, FB, QL> C;
  constexpr int ROWS = C::ROWS, VW = QL * VPT, EPC = 16 / (int)sizeof(T2);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jl = lane / QL, q = lane - jl * QL;          // row of the band, lane of the row
  int b = work[3 * blockIdx.x], k0 = work[3 * blockIdx.x + 1], gpc = work[3 * blockIdx.x + 2];
  const int *bi = d.blk_info + 8 * b;
  const int ni = bi[0], nj = bi[1], per = bi[2], off = d.cell_off[b];
  const int nb = (nj + ROWS - 1) / ROWS;          // bands of the block
  const int gw = w / nb, band = w - gw * nb;     // velocity group, band
  unsigned char *ring = smraw + (size_t)w * NS * ROWS * C::RS * 16;
  T2 *links = reinterpret_cast<T2 *>(smraw + (size_t)nw * NS * ROWS * C::RS * 16);
  volatile int *prog = reinterpret_cast<volatile int *>(links + (size_t)nw * lr * VW);
  volatile int *cons = prog + nw;
  if (lane == 0) { prog[w] = 0; cons[w] = 0; }
  __syncthreads();
  const int kw = k0 + gw * VW;                   // first velocity of the warp
  if (gw >= gpc || kw >= d.nvp) return;          // idle warp (no later CTA-wide barrier)
  const int kb = kw + q * VPT;                   // first velocity of the lane
  const int jb = ROWS * band + jl;
  const int row = PASS == 0 ? jb : nj - 1 - jb;
  const bool rowv = jb < nj;
  T vx[VPT], vy[VPT];
  bool kok[VPT];
#pragma unroll
  for (int u = 0; u < VPT; ++u) {
    kok[u] = kb + u < d.nv;
    vx[u] = kok[u] ? dvx<T>(d, kb + u) : T(0);
    vy[u] = kok[u] ? dvy<T>(d, kb + u) : T(0);
  }
  const unsigned char *gin = reinterpret_cast<const unsigned char *>(d.dfs);
  const unsigned char *gf = reinterpret_cast<const unsigned char *>(d.f);
  const unsigned char *grec = reinterpret_cast<const unsigned char *>(d.srec);
  // copies of step st into ring slot sl: the QL lanes of a row copy
  // consecutive 16-byte chunks of the row's cell (coalesced per row)
  auto issue = [&](int st, int sl) {
    int il = st - jl;
    if (rowv && il >= 0 && il < ni) {
      int i = PASS == 0 ? il : ni - 1 - il;
      size_t c = (size_t)off + (size_t)row * ni + i;
      unsigned char *dst = ring + ((size_t)sl * ROWS + jl) * C::RS * 16;
      size_t gb = (c * d.nvp + kw) * sizeof(T2);
#pragma unroll
      for (int ch = q; ch < C::RV; ch += QL)
        if (kw + ch * EPC < d.nvp) cp_async<16>(dst + 16 * ch, gin + gb + 16 * ch);
      if (PASS == 1) {
#pragma unroll
        for (int ch = q; ch < C::RF; ch += QL) {
          if (C::BF) {
            if (kw + 4 * ch < d.nvp) cp_async<16>(dst + 16 * (C::RV + ch), gf + (c * d.nvp + kw) * 4 + 16 * ch);
          } else {
            if (kw + ch * EPC < d.nvp) cp_async<16>(dst + 16 * (C::RV + ch), gf + gb + 16 * ch);
          }
        }
      }
#pragma unroll
      for (int ch = q; ch < C::RR; ch += QL)
        cp_async<16>(dst + 16 * (C::RV + C::RF + ch), grec + c * NSR * sizeof(T) + 16 * ch);
    }
    cp_async_commit();
  };
  const int nsteps = ni + ROWS - 1;
#pragma unroll
  for (int m = 0; m < NS - 1; ++m) issue(m, m);
  T2 valp[VPT], first[VPT];
#pragma unroll
  for (int u = 0; u < VPT; ++u) { valp[u] = T2{T(0), T(0)}; first[u] = T2{T(0), T(0)}; }
  const int srow = PASS == 0 ? 0 : 1, scol = PASS == 0 ? 2 : 3, sseam = PASS == 0 ? 1 : 0;
  const bool has_below = PASS == 0 ? row > 0 : row < nj - 1;
  const T2 *lin = links + (size_t)(w - 1) * lr * VW + q * VPT;   // previous band's last row
  T2 *lout = links + (size_t)w * lr * VW + q * VPT;
  bool ok = true;
  int slot = 0;
  for (int s = 0; s < nsteps; ++s) {
    issue(s + NS - 1, (slot + NS - 1) % NS);
    cp_async_wait<NS - 1>();
    __syncwarp();                                // the row's chunks, copied by its QL lanes
    const int il = s - jl;
    const bool act = rowv && il >= 0 && il < ni;
    // lower (upper) neighbour across rows: the row below's result of step
    // s - 1 (QL lanes down), or for the band's first row the previous band's
    // last row through the link ring
    T2 up[VPT];
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
      up[u].x = __shfl_up_sync(0xffffffffu, valp[u].x, QL);
      up[u].y = __shfl_up_sync(0xffffffffu, valp[u].y, QL);
    }
    const bool rd = jl == 0 && band > 0 && act;
    if (rd) {
      int n = 0;
      while (prog[w - 1] <= il && ok) {
        __nanosleep(32);                 // leave the issue slots to the other warps
        if (++n > d.wait_polls) { ok = false; atomicOr(d.err, EF_TIMEOUT); }
      }
      __threadfence_block();
      const T2 *src = lin + (size_t)(il & (lr - 1)) * VW;
#pragma unroll
      for (int u = 0; u < VPT; ++u) up[u] = src[u];
    }
    __syncwarp();
    if (rd && q == 0) {
      __threadfence_block();
      cons[w - 1] = il + 1;
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) break;
    const unsigned char *st = ring + ((size_t)slot * ROWS + jl) * C::RS * 16;
    T2 val[VPT];
#pragma unroll
    for (int u = 0; u < VPT; ++u) val[u] = T2{T(0), T(0)};
    if (act) {
      T rec[NSR];
#pragma unroll
      for (int m = 0; m < C::RR; ++m)
        reinterpret_cast<float4 *>(rec)[m] = reinterpret_cast<const float4 *>(st + 16 * (C::RV + C::RF))[m];
      int mask = *reinterpret_cast<const int *>(rec + SR_MASK);
      if (mask & 1) {
        bool urow = il > 0 && (mask & (2 << srow));
        bool ucol = has_below && (mask & (2 << scol));
        bool useam = per && il == ni - 1 && (mask & (2 << sseam));
        const T2 *rv = reinterpret_cast<const T2 *>(st) + q * VPT;
#pragma unroll
        for (int u = 0; u < VPT; ++u) {
          T w0 = vx[u] * rec[0] + vy[u] * rec[1] - rec[2];
          T w1 = vx[u] * rec[3] + vy[u] * rec[4] - rec[5];
          T w2 = vx[u] * rec[6] + vy[u] * rec[7] - rec[8];
          T w3 = vx[u] * rec[9] + vy[u] * rec[10] - rec[11];
          T dg = rec[SR_DBASE];
          dg += w0 > T(0) ? w0 : T(0);
          dg += w1 > T(0) ? w1 : T(0);
          dg += w2 > T(0) ? w2 : T(0);
          dg += w3 > T(0) ? w3 : T(0);
          T wr = PASS == 0 ? w0 : w1, wc = PASS == 0 ? w2 : w3;
          T cr = (urow && wr < T(0)) ? wr : T(0), cc = (ucol && wc < T(0)) ? wc : T(0);
          T ah = cr * valp[u].x + cc * up[u].x, ab = cr * valp[u].y + cc * up[u].y;
          if (useam) {
            T ws = PASS == 0 ? w1 : w0;
            T cs = ws < T(0) ? ws : T(0);
            ah += cs * first[u].x;
            ab += cs * first[u].y;
          }
          T idg = qdiv<T>(T(1), dg);       // FP32: the fast approximate quotient
          T2 r = rv[u];
          if (PASS == 0) {
            val[u].x = (r.x - ah) * idg;
            val[u].y = (r.y - ab) * idg;
          } else {
            val[u].x = r.x - ah * idg;
            val[u].y = r.y - ab * idg;
          }
          if (!kok[u]) val[u] = T2{T(0), T(0)};
        }
        int i = PASS == 0 ? il : ni - 1 - il;
        size_t idx = ((size_t)off + (size_t)row * ni + i) * d.nvp + kb;
        if (PASS == 0) {
          T2 *out = reinterpret_cast<T2 *>(d.dfs) + idx;
#pragma unroll
          for (int u = 0; u < VPT; ++u)
            if (kok[u]) out[u] = val[u];
        } else {
#pragma unroll
          for (int u = 0; u < VPT; ++u) {
            if (!kok[u]) continue;
            T2 fv;
            if (C::BF) {
              float2 x = __bfloat1622float2(
                  reinterpret_cast<const __nv_bfloat162 *>(st + 16 * C::RV)[q * VPT + u]);
              fv = T2{(T)x.x, (T)x.y};
            } else {
              fv = reinterpret_cast<const T2 *>(st + 16 * C::RV)[q * VPT + u];
            }
            stF<T, FB>(d, idx + u, fv.x + val[u].x, fv.y + val[u].y);
          }
        }
      }
    }
    if (act && il == 0) {
#pragma unroll
      for (int u = 0; u < VPT; ++u) first[u] = val[u];
    }
    // the band's last row feeds the next band
    const bool wr_link = jl == ROWS - 1 && act && band + 1 < nb;
    if (wr_link) {
      int n = 0;
      while (cons[w] + lr <= il && ok) {
        __nanosleep(32);
        if (++n > d.wait_polls) { ok = false; atomicOr(d.err, EF_TIMEOUT); }
      }
      T2 *dst = lout + (size_t)(il & (lr - 1)) * VW;
#pragma unroll
      for (int u = 0; u < VPT; ++u) dst[u] = val[u];
      __threadfence_block();
    }
    __syncwarp();
    if (wr_link && q == 0) prog[w] = il + 1;
#pragma unroll
    for (int u = 0; u < VPT; ++u) valp[u] = val[u];
    slot = slot + 1 == NS ? 0 : slot + 1;
  }
  cp_async_wait<0>();
}

template <typename T, int PASS, int VPT, int FB, int QL>
static void ws_launch(const Dev &d, cudaStream_t s, const int *work, int nwork, int nw, int ns) {
  size_t lim = 227 * 1024;
  // deepest ring that fits (6, 4, 2 or 1 steps; 1 = no prefetch), no deeper
  // than asked; then the longest link ring that fits
  int n = ns >= 6 ? 6 : (ns >= 4 ? 4 : (ns >= 2 ? 2 : 1));
  while (n > 1 && ws_smem<T, PASS, VPT, FB, QL>(nw, n) > lim) n = n == 2 ? 1 : n - 2;
  int lr = WS_LR;
  while (lr > 2 && ws_smem<T, PASS, VPT, FB, QL>(nw, n, lr) > lim) lr >>= 1;
  size_t sm = ws_smem<T, PASS, VPT, FB, QL>(nw, n, lr);
  int th = 32 * nw;
  if (n == 6) k_wsweep<T, PASS, 6, VPT, FB, QL><<<nwork, th, sm, s>>>(d, work, lr);
  else if (n == 4) k_wsweep<T, PASS, 4, VPT, FB, QL><<<nwork, th, sm, s>>>(d, work, lr);
  else if (n == 2) k_wsweep<T, PASS, 2, VPT, FB, QL><<<nwork, th, sm, s>>>(d, work, lr);
  else k_wsweep<T, PASS, 1, VPT, FB, QL><<<nwork, th, sm, s>>>(d, work, lr);
}

template <typename T, int PASS, int VPT, int FB, int QL> static void ws_attr() {
  int lim = 227 * 1024;
  cudaFuncSetAttribute(k_wsweep<T, PASS, 1, VPT, FB, QL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_wsweep<T, PASS, 2, VPT, FB, QL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_wsweep<T, PASS, 4, VPT, FB, QL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_wsweep<T, PASS, 6, VPT, FB, QL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <int QL> static void ws_attr_all() {
  ws_attr<float, 0, 2, 0, QL>(); ws_attr<float, 0, 4, 0, QL>();
  ws_attr<float, 1, 2, 0, QL>(); ws_attr<float, 1, 4, 0, QL>();
  ws_attr<float, 1, 2, 1, QL>(); ws_attr<float, 1, 4, 1, QL>();
  ws_attr<double, 0, 2, 0, QL>(); ws_attr<double, 1, 2, 0, QL>();
}

void wsweep_setup() {
  ws_attr_all<4>();
  ws_attr_all<2>();
}

// lanes per row: 4 (8 rows a warp) while the tallest block needs at most 32
// bands, else 2 (16 rows a warp)
int wsweep_ql(int max_nj) {
  int ql = max_nj <= 256 ? 4 : 2;
  if (const char *e = getenv("UGKS_SWEEP_QL"))      // tuning: 2 lanes a row (16 rows a warp)
    if (atoi(e) == 2) ql = 2;
  return ql;
}

// shared memory of the backward sweep (the larger one) with ring depth ns
// and the longest link ring for ns > 1, the shortest for ns = 1
template <int QL> static size_t ws_need(int fp32, int fbf, int vpt, int nw, int ns) {
  int lr = ns > 1 ? WS_LR : 2;
  if (!fp32) return ws_smem<double, 1, 2, 0, QL>(nw, ns, lr);
  if (fbf) return vpt == 4 ? ws_smem<float, 1, 4, 1, QL>(nw, ns, lr) : ws_smem<float, 1, 2, 1, QL>(nw, ns, lr);
  return vpt == 4 ? ws_smem<float, 1, 4, 0, QL>(nw, ns, lr) : ws_smem<float, 1, 2, 0, QL>(nw, ns, lr);
}

int wsweep_fits(int fp32, int fbf, int vpt, int nw, int ns, int ql) {
  size_t need = ql == 4 ? ws_need<4>(fp32, fbf, vpt, nw, ns) : ws_need<2>(fp32, fbf, vpt, nw, ns);
  return nw <= 32 && need <= 227 * 1024;
}

template <int QL>
static void ws_dispatch(const Dev &d, cudaStream_t s, int pass, const int *work, int nwork, int nw, int ns, int vpt,
                        int fp32) {
  if (!fp32) {
    if (pass == 0) ws_launch<double, 0, 2, 0, QL>(d, s, work, nwork, nw, ns);
    else ws_launch<double, 1, 2, 0, QL>(d, s, work, nwork, nw, ns);
    return;
  }
  if (pass == 0) {
    if (vpt == 4) ws_launch<float, 0, 4, 0, QL>(d, s, work, nwork, nw, ns);
    else ws_launch<float, 0, 2, 0, QL>(d, s, work, nwork, nw, ns);
  } else if (d.fbf) {
    if (vpt == 4) ws_launch<float, 1, 4, 1, QL>(d, s, work, nwork, nw, ns);
    else ws_launch<float, 1, 2, 1, QL>(d, s, work, nwork, nw, ns);
  } else {
    if (vpt == 4) ws_launch<float, 1, 4, 0, QL>(d, s, work, nwork, nw, ns);
    else ws_launch<float, 1, 2, 0, QL>(d, s, work, nwork, nw, ns);
  }
}

void launch_wsweep(const Dev &d, cudaStream_t s, int pass, const int *work, int nwork, int nw, int ns, int vpt,
                   int fp32, int ql) {
  if (ql == 4) ws_dispatch<4>(d, s, pass, work, nwork, nw, ns, vpt, fp32);
  else ws_dispatch<2>(d, s, pass, work, nwork, nw, ns, vpt, fp32);
}

}  // namespace ugks
