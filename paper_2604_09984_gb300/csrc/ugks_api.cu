// ugks_api.cu -- host orchestration behind the C ABI of include/ugks.h:
// workspace layout, structured-block topology, and the order of the kernels
// of one physical step (arXiv 2604.09984 Sec. 3 Steps 1-3 and Sec. 2.2
// Steps 1-8).  No device allocation happens here: every device array is a
// slice of the caller's workspace.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ugks.h"
#include "ugks_launch.h"

using namespace ugks;

// (cell, velocity) items per diagonal step of the longest macro sweep below
// which the flux pass plus the residual's first pass end within the sweep,
// from the rates measured on GB300: ~1.0e-11 s and ~4.8e-12 s per item for
// the two, ~0.8 us per diagonal step of the sweep
constexpr double kResidualWindow = 5.3e4;

struct ugks_ctx {
  ugks_params p;
  cudaStream_t st = nullptr;
  cudaStream_t side = nullptr;        // macro LU-SGS runs here, overlapped with the flux kernel
  cudaStream_t cap = nullptr;         // step graphs are captured here (the caller's stream may be the legacy one)
  cudaStream_t tail = nullptr;        // split tail (lowest priority: it fills the reduction's free slots)
  cudaEvent_t ev_flux = nullptr, ev_macro = nullptr;
  cudaEvent_t ev_bwd = nullptr, ev_tail = nullptr;   // fork / join of the inner iteration's tail
  // Step 7 of an inner iteration, the receptors' W and q and the W gradients
  // run on the tail stream beside the next iteration's velocity reduction
  // (which reads none of them); not where an outflow ghost state follows W
  // or on a velocity shard (whose Step 7 waits for the host exchange)
  bool split_tail = false;
  // FP32 path: the residual's predictor-free part beside the macro sweep,
  // where the flux pass and that part end within the sweep (not on the FP64
  // path, where the flux pass alone outlasts it, nor for velocity grids large
  // against the sweep's length); not within a batch of several instances,
  // whose other steps fill the SMs the sweep leaves
  bool split_residual = false;
  bool in_batch = false;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  Dev d;
  int fp32 = 0;                       // FP32 arithmetic (also on the BF16-storage path)
  int fbf = 0;                        // f stored as bf16 pairs
  int nblocks = 0;
  std::vector<ugks_block_desc> blocks;
  std::vector<int> cell_off, node_off;
  int max_nj = 0;
  int sweep_nw = 1, sweep_ql = 4, nwork = 0, nsm = 0;  // micro sweeps: warps per CTA, lanes per row, CTAs
  int nwork_cap = 0;                  // work-list capacity (largest tuning candidate)
  int sweep_vpt = 2;                  // micro sweeps: velocities per lane
  int ns_fwd = 4, ns_bwd = 4;         // prefetch ring depths (steps) of the two sweeps
  int face_tile = 0;                  // tile shape of the face kernels (face_tile_shape)
  ugks_exchange_fn xfn = nullptr;     // velocity sharding: the caller's exchange
  void *xuser = nullptr;
  bool debug_sync = false, debug_failed = false;   // UGKS_DEBUG_SYNC
  // CUDA graphs of ugks_step: captured on the first step with a
  // configuration (key: the device struct the kernels take by value -- whose
  // node buffers alternate from step to step --, the launch configuration and
  // whether the step starts with the extra interpolation of uncovered cells)
  // and replayed while it recurs; a few are kept, the least recently used is
  // replaced
  struct StepGraph {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;             // kernel launches one replay stands for
    int64_t used = 0;
  };
  bool graphs = true;
  std::vector<StepGraph> gcache;
  int64_t gclock = 0, gcaptures = 0, greplays = 0;
  bool stepped = false;               // a ugks_step has run (sweep records valid)
  bool metrics = false;               // steps record their metrics (ugks_set_metrics)
  bool metered = false;               // the last step recorded them
  int *work = nullptr;
  int *prev_status = nullptr, *n_orphan = nullptr, *blk_order = nullptr;
  int cap_interp = 0;
  double t = 0.0, t_new = 0.0;
  bool moved = false, mesh_ready = false;
  std::string err;
  int64_t launches = 0;
  std::vector<double> h_affine;
  bool fresh_pending = false;         // cells uncovered by the last assembly await their first values
  std::vector<int> h_wall_faces;      // staging of the wall-face list upload
  std::vector<double> ref_bbox, h_bin_geo;   // per block reference bbox; bin boxes
  std::vector<int> h_bin_dim;
  // per-kernel-group CUDA-event timing (ugks_profile_*)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev;        // pool of events, used in begin/end pairs
  std::vector<int> ev_group;          // group of each recorded pair
  size_t ev_used = 0;
  double prof_ms[UGKS_NPROF] = {0};
  int64_t prof_n[UGKS_NPROF] = {0};
};

namespace {

int fail(ugks_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_check(ugks_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return UGKS_OK;
  return fail(c, UGKS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
  do {                                                             \
    int _r = cuda_check(ctx, (call), #call);                       \
    if (_r) return _r;                                             \
  } while (0)

struct Sizes {
  int nc = 0, nf = 0, nn = 0, nv = 0, nvp = 0, nseg = 0, nring = 0, max_nj = 0, ntiles = 0;
  int nvx = 0, nvy = 0;
  int iy0 = 0, nv_all = 0, nvp_all = 0;   // velocity shard: first row; the whole grid
  size_t nmrec32 = 0;   // FP32 macro records: (ni + nj - 1) nj per block (diagonal-major)
};

int validate(const ugks_params *p, int nb, const ugks_block_desc *b, Sizes &s, std::string &why) {
  if (!p || nb <= 0 || !b) { why = "null params or no blocks"; return UGKS_ERR_ARG; }
  if (p->precision != UGKS_FP64 && p->precision != UGKS_FP32 && p->precision != UGKS_BF16F) {
    why = "precision";
    return UGKS_ERR_ARG;
  }
  if (p->nvx < 2 || p->nvy < 2 || p->nvx * p->nvy > (1 << 20)) { why = "velocity grid size"; return UGKS_ERR_ARG; }
  if (!(p->vx_max > p->vx_min) || !(p->vy_max > p->vy_min)) { why = "velocity bounds"; return UGKS_ERR_ARG; }
  if (p->K < 0 || !(p->Pr > 0) || !(p->mu_ref > 0) || !(p->cfl_s > 0) || !(p->cfl_pseudo > 0)) {
    why = "gas or solver constant"; return UGKS_ERR_ARG;
  }
  int iy0 = 0, iy1 = p->nvy;
  if (p->shard_iy0 != 0 || p->shard_iy1 != 0) {
    if (p->shard_iy0 < 0 || p->shard_iy1 > p->nvy || p->shard_iy0 >= p->shard_iy1) {
      why = "velocity shard rows";
      return UGKS_ERR_ARG;
    }
    iy0 = p->shard_iy0;
    iy1 = p->shard_iy1;
  }
  s.iy0 = iy0;
  s.nv = p->nvx * (iy1 - iy0);
  s.nvp = (s.nv + 3) / 4 * 4;
  s.nv_all = p->nvx * p->nvy;
  s.nvp_all = (s.nv_all + 3) / 4 * 4;
  s.nvx = p->nvx;
  s.nvy = p->nvy;
  for (int i = 0; i < nb; ++i) {
    const ugks_block_desc &B = b[i];
    if (B.ni < 2 || B.nj < 2 || B.nj > 512) { why = "block size (2 <= ni, 2 <= nj <= 512)"; return UGKS_ERR_ARG; }
    if (B.periodic_i && (B.bc[0] != UGKS_BC_NONE || B.bc[1] != UGKS_BC_NONE)) { why = "periodic block with i-side BC"; return UGKS_ERR_ARG; }
    for (int sd = 0; sd < 4; ++sd) {
      if (B.bc[sd] < 0 || B.bc[sd] > 4) { why = "bc kind"; return UGKS_ERR_ARG; }
      if (!B.periodic_i && B.bc[sd] == UGKS_BC_NONE) { why = "non-periodic block side without BC"; return UGKS_ERR_ARG; }
      if (B.bc[sd] == UGKS_BC_WALL && !(B.wall_T[sd] > 0)) { why = "wall temperature"; return UGKS_ERR_ARG; }
      int nseg = (sd < 2) ? B.nj : B.ni;
      if (B.bc[sd] == UGKS_BC_WALL) s.nseg += nseg;
    }
    if (B.n_fringe < 0 || B.n_gap < 0) { why = "fringe"; return UGKS_ERR_ARG; }
    if (B.periodic_i && B.bc[2] == UGKS_BC_WALL) s.nring += B.ni;
    s.nc += B.ni * B.nj;
    s.nn += (B.ni + 1) * (B.nj + 1);
    s.nf += B.nj * (B.periodic_i ? B.ni : B.ni + 1) + B.ni * (B.nj + 1);
    if (B.nj > s.max_nj) s.max_nj = B.nj;
    s.ntiles += tile_count(B.ni, B.nj);
    s.nmrec32 += (size_t)(B.ni + B.nj - 1) * B.nj;
  }
  return UGKS_OK;
}

size_t bin_capacity(const Sizes &s) { return 16 * (size_t)s.nc + 4096; }

struct Carver {
  char *base;
  size_t off = 0;
  explicit Carver(char *b) : base(b) {}
  template <typename T> T *take(size_t n) {
    off = (off + 255) / 256 * 256;
    T *ptr = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += n * sizeof(T) + 16;
    return ptr;
  }
};
// Micro sweeps (skewed wavefront, ugks_sweep.cu): a warp takes a band of
// 32 / QL rows of a block and QL * VPT consecutive velocities (QL lanes a row,
// VPT velocities a lane); a CTA holds, for one block, a warp per band for each
// of its velocity groups; every CTA has nw warps, nw = the largest band count
// of the blocks, so a smaller block takes several groups per CTA.
int max_nj_of(int nb, const ugks_block_desc *b) {
  int m = 1;
  for (int i = 0; i < nb; ++i) m = std::max(m, b[i].nj);
  return m;
}
int bands_of(int nj, int ql) { int rows = 32 / ql; return (nj + rows - 1) / rows; }
int sweep_nw_for(int nb, const ugks_block_desc *b) {
  int ql = wsweep_ql(max_nj_of(nb, b)), m = 1;
  for (int i = 0; i < nb; ++i) m = std::max(m, bands_of(b[i].nj, ql));
  return m;
}

// Velocities per lane: 2 (UGKS_SWEEP_VPT=4 selects four on the FP32 paths).
int sweep_vpt_for(const ugks_params *p) {
  if (p->precision != UGKS_FP64)
    if (const char *e = getenv("UGKS_SWEEP_VPT"))
      if (atoi(e) == 4) return 4;
  return 2;
}

// Work list (block, first velocity, velocity groups in the CTA) per CTA.
std::vector<int> ws_work(int nb, const ugks_block_desc *b, int nvp, int vpt, int nw) {
  std::vector<int> work;
  int ql = wsweep_ql(max_nj_of(nb, b)), vw = ql * vpt;
  int groups = (nvp + vw - 1) / vw;
  for (int i = 0; i < nb; ++i) {
    int gpc = std::max(1, nw / bands_of(b[i].nj, ql));
    for (int g0 = 0; g0 < groups; g0 += gpc) {
      work.push_back(i);
      work.push_back(g0 * vw);
      work.push_back(std::min(gpc, groups - g0));
    }
  }
  return work;
}

// CTAs of the sweeps (nvp: the context's padded velocity count)
int nwork_for(int nvp, int nb, const ugks_block_desc *b, int vpt) {
  return (int)ws_work(nb, b, nvp, vpt, sweep_nw_for(nb, b)).size() / 3;
}

// Candidates of the sweep autotuner: velocities per lane (FP32 paths; FP64
// keeps 2) and prefetch ring depths (steps).
constexpr int kTuneVpt[] = {2, 4};
constexpr int kTuneRing[] = {2, 4, 6};

// Work-list capacity: the most CTAs any candidate needs (sized for the
// whole velocity grid, which covers any shard of it).
int nwork_cap_for(const ugks_params *p, int nb, const ugks_block_desc *b) {
  int nvp = (p->nvx * p->nvy + 3) / 4 * 4;
  int n = nwork_for(nvp, nb, b, sweep_vpt_for(p));
  for (int v : kTuneVpt) n = std::max(n, nwork_for(nvp, nb, b, v));
  return n;
}

// Lay out every device array of the context in the workspace (base may be
// null to measure).  Returns the bytes used.
size_t carve(char *base, const Sizes &s, int nb, int fp32, int fbf, int nwork, int cap_interp, Dev &d) {
  Carver c(base);
  size_t pair = fp32 ? 2 * sizeof(float) : 2 * sizeof(double);
  size_t fpair = fbf ? 4 : pair;       // storage of f (bf16 pairs on the BF16-storage path)
  size_t tsz = fp32 ? sizeof(float) : sizeof(double);
  d.vx = c.take<double>(s.nvp); d.vy = c.take<double>(s.nvp); d.w = c.take<double>(s.nvp);
  d.vxf = c.take<float>(s.nvp); d.vyf = c.take<float>(s.nvp); d.wf = c.take<float>(s.nvp);
  d.wx1f = c.take<float>((size_t)s.nvx); d.wy1f = c.take<float>((size_t)s.nvy);
  d.vy1f = c.take<float>((size_t)s.nvy);
  d.vx1 = c.take<double>((size_t)s.nvx); d.vy1 = c.take<double>((size_t)s.nvy);
  d.wx1 = c.take<double>((size_t)s.nvx); d.wy1 = c.take<double>((size_t)s.nvy);
  d.vxa = c.take<double>(s.nvp_all); d.vya = c.take<double>(s.nvp_all); d.wa = c.take<double>(s.nvp_all);
  d.vxaf = c.take<float>(s.nvp_all); d.vyaf = c.take<float>(s.nvp_all); d.waf = c.take<float>(s.nvp_all);
  d.msum = c.take<double>(6 * (size_t)s.nc);
  d.cell_nodes = c.take<int>(4 * (size_t)s.nc);
  d.cell_faces = c.take<int>(4 * (size_t)s.nc);
  d.cell_sgn = c.take<int8_t>(4 * (size_t)s.nc);
  d.nb_kind = c.take<int>(4 * (size_t)s.nc);
  d.nb_id = c.take<int>(4 * (size_t)s.nc);
  d.nb_shift = c.take<int8_t>(4 * (size_t)s.nc);
  d.cell_row = c.take<int>(2 * (size_t)s.nc);
  d.cell_block = c.take<int>(s.nc);
  d.node_block = c.take<int>(s.nn);
  d.face_L = c.take<int>(s.nf); d.face_R = c.take<int>(s.nf);
  d.face_a = c.take<int>(s.nf); d.face_b = c.take<int>(s.nf);
  d.face_kind = c.take<int>(s.nf); d.face_block = c.take<int>(s.nf);
  d.face_shiftL = c.take<int8_t>(s.nf);
  d.face_Tw = c.take<double>(s.nf);
  d.X_ref = c.take<double>(2 * (size_t)s.nn);
  d.X_old = c.take<double>(2 * (size_t)s.nn);
  d.X_new = c.take<double>(2 * (size_t)s.nn);
  d.Xf = c.take<float2>((size_t)s.nn);
  d.cbb = c.take<float4>((size_t)s.nc);
  d.vol_old = c.take<double>(s.nc); d.vol_new = c.take<double>(s.nc); d.dts = c.take<double>(s.nc);
  d.xc = c.take<double>(2 * (size_t)s.nc); d.xc_new = c.take<double>(2 * (size_t)s.nc);
  d.period = c.take<double>(2 * (size_t)s.nc);
  d.Sn = c.take<double>(2 * (size_t)s.nf); d.nrm = c.take<double>(2 * (size_t)s.nf);
  d.xf = c.take<double>(2 * (size_t)s.nf); d.Uf = c.take<double>(2 * (size_t)s.nf);
  d.S = c.take<double>(s.nf); d.SUn = c.take<double>(s.nf);
  d.slope_flags = c.take<int>(s.nc);
  d.cmask = c.take<int>(s.nc);
  d.jinv = c.take<double>(4 * (size_t)s.nc);
  d.jinvf = c.take<float4>((size_t)s.nc);
  d.fgeo = c.take<char>(tsz * NFG * (size_t)s.nf);
  d.srec = c.take<char>(tsz * NSR * (size_t)s.nc);
  d.affine = c.take<double>(6 * (size_t)nb);
  d.f = c.take<char>(fpair * (size_t)s.nc * s.nvp);
  d.fbf = fbf;
  d.W = c.take<double>(4 * (size_t)s.nc); d.q = c.take<double>(2 * (size_t)s.nc);
  d.status = c.take<int>(s.nc);
  d.Tn = c.take<char>(pair * (size_t)s.nc * s.nvp);
  d.dfs = c.take<char>(pair * (size_t)s.nc * s.nvp);
  d.Dbuf = c.take<char>(pair * (size_t)s.nc * s.nvp);
  d.fval = c.take<char>(2 * pair * (size_t)s.nf * s.nvp);
  d.stepc = c.take<double>(4);
  d.mpart = c.take<double>((size_t)MET_NQ * MET_BLOCKS);
  d.mout = c.take<double>(MET_NQ);
  d.TW = c.take<double>(4 * (size_t)s.nc); d.Fc = c.take<double>(4 * (size_t)s.nc);
  d.dW = c.take<double>(4 * (size_t)s.nc); d.Wp = c.take<double>(4 * (size_t)s.nc);
  d.mrec = c.take<char>(fp32 ? sizeof(float) * NMR32 * s.nmrec32 : sizeof(double) * NMR * (size_t)s.nc);
  d.mrec_off = c.take<int>((size_t)nb + 1);
  d.cpar = c.take<double>(NCP * (size_t)s.nc); d.cparn = c.take<double>(NCP * (size_t)s.nc);
  d.shp = c.take<char>(tsz * NSH * (size_t)s.nc); d.shn = c.take<char>(tsz * NSH * (size_t)s.nc);
  d.gradW = c.take<double>(8 * (size_t)s.nc);
  d.ghostW = c.take<double>(4 * (size_t)s.nf);
  d.fsum = c.take<double>(NFS * (size_t)s.nf);
  d.fpar = c.take<double>(NFP * (size_t)s.nf);
  d.fparT = c.take<char>(tsz * NFP * (size_t)s.nf);
  d.fflux = c.take<double>(4 * (size_t)s.nf);
  d.gam = c.take<double>(s.nf);
  d.wall_loads = c.take<double>(4 * (size_t)nb);
  d.torque_io = c.take<double>(3 * (size_t)nb);
  d.wall_faces = c.take<int>(s.nf);
  d.node_active = c.take<int>(s.nn);
  d.cls = c.take<int>(s.nc);
  d.donors = c.take<int>(5 * (size_t)s.nc);
  d.dwgt = c.take<double>(5 * (size_t)s.nc);
  d.rec_list = c.take<int>(s.nc);
  d.fresh_list = c.take<int>(s.nc);
  d.conn_cnt = c.take<int>(8);
  d.conn_chunk = c.take<int4>(((size_t)s.nc + 1023) / 1024);
  d.itmp = c.take<char>(pair * (size_t)cap_interp * s.nvp);
  d.itmpW = c.take<double>(6 * (size_t)cap_interp);
  d.cap_interp = cap_interp;
  d.wall_seg = c.take<int>(2 * (size_t)s.nseg + 2);
  d.segf = c.take<float4>((size_t)s.nseg + 1);
  d.nseg = s.nseg;
  d.wall_seg_off = c.take<int>(nb + 1);
  d.body_ring = c.take<int>((size_t)s.nring + 1);
  d.body_ring_off = c.take<int>(nb + 1);
  d.body_bb = c.take<float4>(nb);
  d.cell_off = c.take<int>(nb + 1);
  d.node_off = c.take<int>(nb + 1);
  d.blk_info = c.take<int>(8 * (size_t)nb);
  d.bin_geo = c.take<double>(4 * (size_t)nb);
  d.bin_dim = c.take<int>(3 * (size_t)nb);
  d.bin_cnt = c.take<int>((size_t)s.nc + nb + 1);
  d.bin_start = c.take<int>((size_t)s.nc + nb + 2);
  d.bin_items = c.take<int>(bin_capacity(s));
  d.tiles = c.take<int>(3 * (size_t)s.ntiles);
  d.err = c.take<int>(4);
  (void)nwork;
  c.take<int>(3 * (size_t)nwork + 3);   // micro-sweep work list
  c.take<int>(s.nc);                   // previous status / fresh flags
  c.take<int>(4);                      // orphan counter
  c.take<int>(nb);                     // block priority order
  return c.off;
}

int cap_interp_for(const Sizes &s, int nb) { return nb > 1 ? (s.nc / 4 > 1024 ? s.nc / 4 : (s.nc < 1024 ? s.nc : 1024)) : 0; }

// Host topology identical in ordering to the face/cell numbering documented
// in ugks.h.
struct Topo {
  std::vector<int> cell_nodes, cell_faces, nb_kind, nb_id, cell_row, cell_block, node_block;
  std::vector<int8_t> cell_sgn, nb_shift, face_shiftL;
  std::vector<int> face_L, face_R, face_a, face_b, face_kind, face_block;
  std::vector<double> face_Tw;
  std::vector<int> wall_seg, wall_seg_off, body_ring, body_ring_off, blk_info;
};

void build_topology(int nb, const ugks_block_desc *B, const std::vector<int> &coff,
                    const std::vector<int> &noff, int nc, int nn, Topo &T) {
  T.cell_nodes.assign(4 * (size_t)nc, 0);
  T.cell_faces.assign(4 * (size_t)nc, -1);
  T.cell_sgn.assign(4 * (size_t)nc, 0);
  T.nb_kind.assign(4 * (size_t)nc, NB_NONE);
  T.nb_id.assign(4 * (size_t)nc, -1);
  T.nb_shift.assign(4 * (size_t)nc, 0);
  T.cell_row.assign(2 * (size_t)nc, 0);
  T.cell_block.assign(nc, 0);
  T.node_block.assign(nn, 0);
  T.wall_seg_off.push_back(0);
  T.body_ring_off.push_back(0);
  auto add_face = [&](int L, int R, int a, int b, int kind, int blk, int shL, double Tw) {
    T.face_L.push_back(L); T.face_R.push_back(R); T.face_a.push_back(a); T.face_b.push_back(b);
    T.face_kind.push_back(kind); T.face_block.push_back(blk); T.face_shiftL.push_back((int8_t)shL);
    T.face_Tw.push_back(Tw);
    return (int)T.face_L.size() - 1;
  };
  for (int bi = 0; bi < nb; ++bi) {
    const ugks_block_desc &b = B[bi];
    int ni = b.ni, nj = b.nj, co = coff[bi], no = noff[bi];
    auto cid = [&](int i, int j) { return co + j * ni + i; };
    auto nid = [&](int i, int j) { return no + j * (ni + 1) + i; };
    for (int n = noff[bi]; n < noff[bi + 1]; ++n) T.node_block[n] = bi;
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        int c = cid(i, j);
        T.cell_block[c] = bi;
        int *nd = &T.cell_nodes[4 * (size_t)c];
        nd[0] = nid(i, j); nd[1] = nid(i + 1, j); nd[2] = nid(i + 1, j + 1); nd[3] = nid(i, j + 1);
        T.cell_row[2 * (size_t)c] = nid(0, j);
        T.cell_row[2 * (size_t)c + 1] = nid(ni, j);
      }
    auto setf = [&](int c, int slot, int f) { T.cell_faces[4 * (size_t)c + slot] = f; };
    for (int j = 0; j < nj; ++j) {
      int iend = b.periodic_i ? ni : ni + 1;
      for (int i = 0; i < iend; ++i) {
        if (b.periodic_i) {
          int L = cid((i - 1 + ni) % ni, j), R = cid(i, j);
          int f = add_face(L, R, nid(i, j), nid(i, j + 1), UGKS_BC_NONE, bi, i == 0 ? -1 : 0, 0.0);
          setf(L, 1, f); setf(R, 0, f);
        } else if (i == 0) {
          int c = cid(0, j);
          setf(c, 0, add_face(c, -1, nid(0, j + 1), nid(0, j), b.bc[0], bi, 0, b.wall_T[0]));
        } else if (i == ni) {
          int c = cid(ni - 1, j);
          setf(c, 1, add_face(c, -1, nid(ni, j), nid(ni, j + 1), b.bc[1], bi, 0, b.wall_T[1]));
        } else {
          int L = cid(i - 1, j), R = cid(i, j);
          int f = add_face(L, R, nid(i, j), nid(i, j + 1), UGKS_BC_NONE, bi, 0, 0.0);
          setf(L, 1, f); setf(R, 0, f);
        }
      }
    }
    for (int i = 0; i < ni; ++i)
      for (int j = 0; j <= nj; ++j) {
        if (j == 0) {
          int c = cid(i, 0);
          setf(c, 2, add_face(c, -1, nid(i, 0), nid(i + 1, 0), b.bc[2], bi, 0, b.wall_T[2]));
        } else if (j == nj) {
          int c = cid(i, nj - 1);
          setf(c, 3, add_face(c, -1, nid(i + 1, nj), nid(i, nj), b.bc[3], bi, 0, b.wall_T[3]));
        } else {
          int L = cid(i, j - 1), R = cid(i, j);
          int f = add_face(L, R, nid(i + 1, j), nid(i, j), UGKS_BC_NONE, bi, 0, 0.0);
          setf(L, 3, f); setf(R, 2, f);
        }
      }
    const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        int c = cid(i, j);
        for (int s = 0; s < 4; ++s) {
          int ii = i + di[s], jj = j + dj[s];
          size_t q = 4 * (size_t)c + s;
          if (ii >= 0 && ii < ni && jj >= 0 && jj < nj) {
            T.nb_kind[q] = NB_CELL; T.nb_id[q] = cid(ii, jj);
          } else if (di[s] != 0 && b.periodic_i) {
            T.nb_kind[q] = NB_CELL; T.nb_id[q] = cid((ii + ni) % ni, jj); T.nb_shift[q] = (int8_t)di[s];
          } else {
            int kind = b.bc[s];
            if (kind == UGKS_BC_FARFIELD || kind == UGKS_BC_OUTFLOW) {
              T.nb_kind[q] = NB_GHOST; T.nb_id[q] = T.cell_faces[q];
            } else {
              T.nb_kind[q] = NB_NONE;
            }
          }
        }
      }
    // wall segments (node pairs along wall sides) and body ring
    for (int sd = 0; sd < 4; ++sd) {
      if (b.bc[sd] != UGKS_BC_WALL) continue;
      if (sd < 2) {
        int i = sd == 0 ? 0 : ni;
        for (int j = 0; j < nj; ++j) { T.wall_seg.push_back(nid(i, j)); T.wall_seg.push_back(nid(i, j + 1)); }
      } else {
        int j = sd == 2 ? 0 : nj;
        for (int i = 0; i < ni; ++i) { T.wall_seg.push_back(nid(i, j)); T.wall_seg.push_back(nid(i + 1, j)); }
      }
    }
    T.wall_seg_off.push_back((int)T.wall_seg.size() / 2);
    if (b.periodic_i && b.bc[2] == UGKS_BC_WALL)
      for (int i = 0; i < ni; ++i) T.body_ring.push_back(nid(i, 0));
    T.body_ring_off.push_back((int)T.body_ring.size());
    int mask = 0;
    for (int sd = 0; sd < 4; ++sd) if (b.bc[sd] == UGKS_BC_OVERSET) mask |= 1 << sd;
    int info[8] = {ni, nj, b.periodic_i ? 1 : 0, b.priority, b.n_fringe, b.n_gap, mask,
                   (b.periodic_i && b.bc[2] == UGKS_BC_WALL) ? 1 : 0};
    for (int m = 0; m < 8; ++m) T.blk_info.push_back(info[m]);
  }
  for (int c = 0; c < nc; ++c)
    for (int s = 0; s < 4; ++s) {
      int f = T.cell_faces[4 * (size_t)c + s];
      T.cell_sgn[4 * (size_t)c + s] = (T.face_L[f] == c) ? 1 : -1;
    }
}

template <typename V> int up(ugks_ctx *ctx, void *dst, const std::vector<V> &src) {
  if (src.empty()) return UGKS_OK;
  CK(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice, ctx->st));
  return UGKS_OK;
}

int check_err_flag(ugks_ctx *ctx) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->d.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (h) {
    CK(cudaMemsetAsync(ctx->d.err, 0, sizeof(int), ctx->st));
    // causes before consequences: motion and assembly, then the step
    if (h & EF_GEOMETRY) return fail(ctx, UGKS_ERR_GEOMETRY, "non-positive cell volume after mesh move");
    if (h & EF_BINS) return fail(ctx, UGKS_ERR_WORKSPACE, "overset search bins overflowed");
    if (h & EF_CAPACITY) return fail(ctx, UGKS_ERR_WORKSPACE, "more receptors than the interpolation staging holds");
    if (h & EF_ORPHAN) return fail(ctx, UGKS_ERR_ORPHAN, "overset receptors without donor");
    if (h & EF_TIMEOUT) return fail(ctx, UGKS_ERR_TIMEOUT, "a kernel's bounded wait for its data ran out");
    if (h & EF_NONPHYSICAL) return fail(ctx, UGKS_ERR_NONPHYSICAL, "non-finite or non-positive density/temperature");
  }
  return UGKS_OK;
}

int launch_status(ugks_ctx *ctx) { return cuda_check(ctx, cudaPeekAtLastError(), "kernel launch"); }

// Switch the micro sweeps to another number of velocities per lane
// (uploads the work list).
int set_sweep_tiles(ugks_ctx *ctx, int vpt) {
  std::vector<int> work = ws_work(ctx->nblocks, ctx->blocks.data(), ctx->d.nvp, vpt, ctx->sweep_nw);
  if ((int)work.size() / 3 > ctx->nwork_cap) return fail(ctx, UGKS_ERR_WORKSPACE, "sweep work list");
  CK(cudaMemcpyAsync(ctx->work, work.data(), sizeof(int) * work.size(), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->nwork = (int)work.size() / 3;
  ctx->sweep_vpt = vpt;
  return UGKS_OK;
}

// Event pair around one launch of a kernel group (only while profiling).
// With UGKS_DEBUG_SYNC=1 in the environment at context creation, every
// launch group is followed by a stream synchronisation and an error check, and
// the first failing group is named on stderr (diagnosis of device faults).
struct Prof {
  ugks_ctx *c;
  cudaStream_t s;
  int g;
  size_t slot = (size_t)-1;
  Prof(ugks_ctx *ctx, int group, cudaStream_t stream = nullptr) : c(ctx), s(stream ? stream : ctx->st), g(group) {
    if (!c->prof_on) return;
    if (c->ev_used + 2 > c->ev.size()) {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->ev.push_back(e);
      }
      c->ev_group.resize(c->ev.size() / 2);
    }
    slot = c->ev_used;
    c->ev_used += 2;
    c->ev_group[slot / 2] = group;
    cudaEventRecord(c->ev[slot], s);
  }
  ~Prof() {
    if (slot != (size_t)-1) cudaEventRecord(c->ev[slot + 1], s);
    if (c->debug_sync) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess && !c->debug_failed) {
        c->debug_failed = true;
        fprintf(stderr, "ugks debug sync: kernel group %d failed: %s\n", g, cudaGetErrorString(e));
      }
    }
  }
};

// Drain recorded event pairs into the per-group totals.
int prof_drain(ugks_ctx *ctx) {
  if (ctx->ev_used == 0) return UGKS_OK;
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaStreamSynchronize(ctx->side));
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
    int g = ctx->ev_group[i / 2];
    ctx->prof_ms[g] += ms;
    ctx->prof_n[g] += 1;
  }
  ctx->ev_used = 0;
  return UGKS_OK;
}

// Receptor (fresh = 0) or fresh-cell (fresh = 1) interpolation; the list
// length lives on the device.
int do_interp(ugks_ctx *ctx, int fresh, int parts = 3, cudaStream_t s = nullptr) {
  if (ctx->nblocks < 2) return UGKS_OK;
  Dev &d = ctx->d;
  if (!s) s = ctx->st;
  {
    Prof p(ctx, UGKS_PROF_INTERP, s);
    launch_interp(d, s, fresh ? d.fresh_list : d.rec_list, d.conn_cnt + (fresh ? 1 : 0), ctx->nsm, ctx->fp32,
                  parts);
  }
  ctx->launches += 2;
  return UGKS_OK;
}

// Sharded context: the caller's exchange turns the partial sums of buffer
// `which` into the sums over all shards (no-op when not sharded).
int shard_exchange(ugks_ctx *ctx, int which) {
  if (!ctx->d.shard) return UGKS_OK;
  if (!ctx->xfn) return fail(ctx, UGKS_ERR_ORDER, "sharded context without an exchange function");
  if (ctx->xfn(which, (void *)ctx->st, ctx->xuser) != 0) return fail(ctx, UGKS_ERR_ARG, "shard exchange failed");
  return UGKS_OK;
}

// The step size where the step's kernels read it (stream-ordered upload).
int upload_step_size(ugks_ctx *ctx) {
  const Dev &d = ctx->d;
  double v[4] = {d.dt, d.idt, (double)d.idt_f, 0.0};
  return launch_upload(const_cast<double *>(d.stepc), v, sizeof(v), ctx->st);
}

// Ghost states, W gradients, face reduction, face coefficients, per-cell
// macro flux sum (Steps 1 / 3 up to the velocity-resolved flux).
// joined: the W gradients ran on the tail stream (split tail); the face
// state waits for them after the velocity reduction
int flux_prep(ugks_ctx *ctx, int level_n, bool joined = false) {
  Dev &d = ctx->d;
  cudaStream_t s = ctx->st;
  if (!joined) { Prof p(ctx, UGKS_PROF_CELL); launch_ghost_gradW(d, s); }
  { Prof p(ctx, UGKS_PROF_FACE_REDUCE); launch_face_reduce_tile(d, s, ctx->fp32, ctx->face_tile); }
  int r = shard_exchange(ctx, 0);
  if (r) return r;
  if (joined) CK(cudaStreamWaitEvent(s, ctx->ev_tail, 0));
  { Prof p(ctx, UGKS_PROF_FACE_COEF); launch_face_coef(d, s, ctx->fp32); }
  { Prof p(ctx, UGKS_PROF_CELL); launch_cell_macro(d, s, level_n); }
  // ghost states and gradients (or the wait), reduction, face state and
  // coefficients (the wall kernel where there are walls), cell terms
  ctx->launches += (joined ? 0 : 2) + 1 + 2 + (d.nwall > 0 ? 1 : 0) + 1;
  return UGKS_OK;
}

// Overset assembly (Sec. 3.1) and the device-side receptor / fresh lists.
// With sync, waits for the counters, fills stats and reports orphans and
// staging overflow; without, every check is left to the error flag.
int do_connect(ugks_ctx *ctx, ugks_connect_stats *stats, bool initial, bool sync) {
  Dev &d = ctx->d;
  if (ctx->nblocks < 2) {
    if (stats) { stats->n_field = d.nc; stats->n_receptor = stats->n_hole = stats->n_fresh = stats->n_orphan = 0; }
    return UGKS_OK;
  }
  // prev_status: last status (all FIELD initially so no cell is "fresh")
  if (initial) CK(cudaMemsetAsync(ctx->prev_status, 0, sizeof(int) * d.nc, ctx->st));
  else CK(cudaMemcpyAsync(ctx->prev_status, d.status, sizeof(int) * d.nc, cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->n_orphan, 0, sizeof(int), ctx->st));
  {
    // bins over the affine image of each block's reference bounding box
    std::vector<double> geo(4 * (size_t)ctx->nblocks);
    std::vector<int> dim(3 * (size_t)ctx->nblocks);
    int base = 0;
    for (int b = 0; b < ctx->nblocks; ++b) {
      const double *A = &ctx->h_affine[6 * (size_t)b];
      const double *bb = &ctx->ref_bbox[4 * (size_t)b];
      double xl = 1e300, xh = -1e300, yl = 1e300, yh = -1e300;
      for (int corner = 0; corner < 4; ++corner) {
        double x = (corner & 1) ? bb[2] : bb[0], y = (corner & 2) ? bb[3] : bb[1];
        double X = A[0] * x + A[1] * y + A[4], Y = A[2] * x + A[3] * y + A[5];
        xl = std::min(xl, X); xh = std::max(xh, X); yl = std::min(yl, Y); yh = std::max(yh, Y);
      }
      double w = xh - xl, h = yh - yl, pad = 1e-9 * (w + h + 1.0);
      xl -= pad; yl -= pad; w += 2 * pad; h += 2 * pad;
      int ncb = ctx->cell_off[b + 1] - ctx->cell_off[b];
      double target = std::max(1.0, ncb / 2.0);
      int nx = std::max(1, std::min(2048, (int)std::lround(std::sqrt(target * w / h))));
      int ny = std::max(1, std::min(2048, (int)std::lround(target / nx)));
      while ((size_t)nx * ny > (size_t)ncb && nx > 1) --nx;
      while ((size_t)nx * ny > (size_t)ncb && ny > 1) --ny;
      geo[4 * b] = xl; geo[4 * b + 1] = yl; geo[4 * b + 2] = nx / w; geo[4 * b + 3] = ny / h;
      dim[3 * b] = nx; dim[3 * b + 1] = ny; dim[3 * b + 2] = base;
      base += nx * ny;
    }
    d.nbins = base;
    ctx->h_bin_geo = geo;
    ctx->h_bin_dim = dim;
    ctx->launches += launch_upload(d.bin_geo, geo.data(), sizeof(double) * geo.size(), ctx->st);
    ctx->launches += launch_upload(d.bin_dim, dim.data(), sizeof(int) * dim.size(), ctx->st);
  }
  {
    Prof p(ctx, UGKS_PROF_CONNECT);
    launch_connect(d, ctx->st, ctx->prev_status, ctx->blk_order, ctx->n_orphan);
    launch_lists(d, ctx->st, ctx->prev_status, ctx->n_orphan);
  }
  launch_slope_geo(d, ctx->st);     // holes changed
  ctx->launches += 12;
  ctx->fresh_pending = !initial;
  int r = launch_status(ctx);
  if (r || !sync) return r;
  int cnt[8];
  CK(cudaMemcpyAsync(cnt, d.conn_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (stats) {
    stats->n_field = cnt[2]; stats->n_receptor = cnt[0]; stats->n_hole = cnt[3];
    stats->n_fresh = cnt[1]; stats->n_orphan = cnt[4];
  }
  r = check_err_flag(ctx);
  if (r == UGKS_ERR_ORPHAN) return fail(ctx, r, std::to_string(cnt[4]) + " receptors without donor");
  return r;
}

// Steps 1-8 of one physical step (after the motion and the assembly),
// issued on the context's streams without any host synchronisation.
int step_body(ugks_ctx *ctx, int n_inner) {
  Dev &d = ctx->d;
  cudaStream_t s = ctx->st;
  int fp = ctx->fp32;
  // per-kernel event timing wants each group alone on its stream: profiled
  // steps run the tail in line
  const bool split = ctx->split_tail && !ctx->prof_on;
  if (ctx->fresh_pending) do_interp(ctx, 1);
  do_interp(ctx, 0);
  // Steps 1-2: level-n flux, extensive level-n macro term, level-n cell record
  int rx = flux_prep(ctx, 1);
  if (rx) return rx;
  { Prof p(ctx, UGKS_PROF_CELL); launch_cell_params(d, s, d.W, d.cparn, fp); }
  ctx->launches += 1;
  for (int it = 0; it < n_inner; ++it) {
    if (it > 0) {
      if (split) {
        // the previous iteration's Step 7 is still running on the tail
        // stream: interpolate the receptors' f, reduce, then join
        do_interp(ctx, 0, 1);
        if ((rx = flux_prep(ctx, 0, true))) return rx;   // Step 3
      } else {
        do_interp(ctx, 0);
        if ((rx = flux_prep(ctx, 0))) return rx;   // Step 3
      }
    }
    // Step 4 (macro LU-SGS) on the side stream, concurrently with the flux
    // divergence of Step 3 on the main stream; Step 5 joins both
    bool met = ctx->metrics && it == n_inner - 1;    // metrics of the last inner iteration
    { Prof p(ctx, UGKS_PROF_MACRO_SWEEP); launch_macro_prep(d, s, fp); }
    CK(cudaEventRecord(ctx->ev_flux, s));
    CK(cudaStreamWaitEvent(ctx->side, ctx->ev_flux, 0));
    if (met) launch_metrics(d, s, 0, fp);
    { Prof p(ctx, UGKS_PROF_MACRO_SWEEP, ctx->side); launch_macro_sweep(d, ctx->side, ctx->max_nj, fp); }
    CK(cudaEventRecord(ctx->ev_macro, ctx->side));
    { Prof p(ctx, UGKS_PROF_RHS); launch_flux_tile(d, s, fp, ctx->face_tile); }              // Step 3
    if (ctx->split_residual && !ctx->in_batch) {
      // Step 5 without the predictor's collision term while the sweep runs
      { Prof p(ctx, UGKS_PROF_RESIDUAL); launch_residual(d, s, it == 0, fp, 1); }
      CK(cudaStreamWaitEvent(s, ctx->ev_macro, 0));
      { Prof p(ctx, UGKS_PROF_RESIDUAL); launch_residual(d, s, it == 0, fp, 2); }
      ctx->launches += 1;
    } else {
      CK(cudaStreamWaitEvent(s, ctx->ev_macro, 0));
      { Prof p(ctx, UGKS_PROF_RESIDUAL); launch_residual(d, s, it == 0, fp); }               // Step 5
    }
    if (met) launch_metrics(d, s, 1, fp);
    { Prof p(ctx, UGKS_PROF_MICRO_FWD); launch_wsweep(d, s, 0, ctx->work, ctx->nwork, ctx->sweep_nw, ctx->ns_fwd, ctx->sweep_vpt, fp, ctx->sweep_ql); }  // Step 6
    { Prof p(ctx, UGKS_PROF_MICRO_BWD); launch_wsweep(d, s, 1, ctx->work, ctx->nwork, ctx->sweep_nw, ctx->ns_bwd, ctx->sweep_vpt, fp, ctx->sweep_ql); }
    if (split && it + 1 < n_inner) {
      // Step 7, the receptors' W and q and the W gradients of the next
      // iteration on the tail stream, beside its velocity reduction
      CK(cudaEventRecord(ctx->ev_bwd, s));
      CK(cudaStreamWaitEvent(ctx->tail, ctx->ev_bwd, 0));
      { Prof p(ctx, UGKS_PROF_MOMENTS, ctx->tail); launch_moments(d, ctx->tail, fp); }      // Step 7
      do_interp(ctx, 0, 2, ctx->tail);
      { Prof p(ctx, UGKS_PROF_CELL, ctx->tail); launch_gradW(d, ctx->tail); }
      CK(cudaEventRecord(ctx->ev_tail, ctx->tail));
      ctx->launches += 9;
      continue;
    }
    { Prof p(ctx, UGKS_PROF_MOMENTS); launch_moments(d, s, fp); }                          // Step 7
    if (d.shard) {
      if ((rx = shard_exchange(ctx, 1))) return rx;
      { Prof p(ctx, UGKS_PROF_MOMENTS); launch_moments_finish(d, s); }
      ctx->launches += 1;
    }
    if (met) {
      launch_metrics(d, s, 2, fp);
      ctx->launches += 4;
    }
    ctx->launches += 8;
  }
  return UGKS_OK;
}

// What the captured kernels depend on beyond device memory: the device
// struct they take by value and the launch configuration.
std::vector<unsigned char> graph_key(const ugks_ctx *c, int n_inner) {
  int cfg[] = {n_inner, c->fresh_pending ? 1 : 0, c->face_tile, c->sweep_vpt, c->ns_fwd, c->ns_bwd, c->sweep_nw,
               c->sweep_ql, c->nwork, c->nsm, c->max_nj, c->fp32, c->metrics ? 1 : 0, c->split_tail ? 1 : 0,
               c->split_residual && !c->in_batch ? 1 : 0};
  // (the step size is read from device memory; the bin count belongs to the
  // assembly, which is not part of the step)
  Dev d = c->d;
  d.dt = d.idt = 0.0;
  d.idt_f = 0.f;
  d.nbins = 0;
  std::vector<unsigned char> k(sizeof(Dev) + sizeof(cfg));
  memcpy(k.data(), &d, sizeof(Dev));
  memcpy(k.data() + sizeof(Dev), cfg, sizeof(cfg));
  return k;
}

constexpr size_t kStepGraphs = 4;     // executable step graphs kept per context

// The step through a CUDA graph: replay the cached graph of this key, or
// capture the step and instantiate it (or update the least recently used
// cached graph with it), then one graph launch on the context's stream.
int step_graph(ugks_ctx *ctx, int n_inner) {
  std::vector<unsigned char> key = graph_key(ctx, n_inner);
  ugks_ctx::StepGraph *hit = nullptr;
  for (auto &g : ctx->gcache)
    if (g.key == key) hit = &g;
  if (!hit) {
    // captured on the context's private stream (the caller's may be the
    // legacy default stream, which cannot be captured); launched on the
    // caller's stream below
    cudaGraph_t g = nullptr;
    cudaStream_t user = ctx->st;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    ctx->st = ctx->cap;
    int64_t l0 = ctx->launches;
    int r = step_body(ctx, n_inner);
    ctx->st = user;
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
    int64_t nl = ctx->launches - l0;
    ctx->launches = l0;
    if (r != UGKS_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return r != UGKS_OK ? r : cuda_check(ctx, e, "step capture");
    }
    if (ctx->gcache.size() < kStepGraphs) {
      ctx->gcache.emplace_back();
      hit = &ctx->gcache.back();
    } else {
      hit = &ctx->gcache[0];
      for (auto &c : ctx->gcache)
        if (c.used < hit->used) hit = &c;
      cudaGraphExecUpdateResultInfo info;
      if (hit->exec && cudaGraphExecUpdate(hit->exec, g, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(hit->exec);
        hit->exec = nullptr;
      }
    }
    if (!hit->exec) {
      cudaError_t ie = cudaGraphInstantiate(&hit->exec, g, 0);
      if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        hit->exec = nullptr;
        hit->key.clear();
        return cuda_check(ctx, ie, "graph instantiate");
      }
    }
    cudaGraphDestroy(g);
    hit->key.swap(key);
    hit->launches = nl;
    ++ctx->gcaptures;
  } else {
    ++ctx->greplays;
  }
  hit->used = ++ctx->gclock;
  CK(cudaGraphLaunch(hit->exec, ctx->st));
  ctx->launches += hit->launches;
  return UGKS_OK;
}

}  // namespace

extern "C" {

int ugks_workspace_query(const ugks_params *p, int nblocks, const ugks_block_desc *blocks, size_t *bytes) {
  Sizes s;
  std::string why;
  int r = validate(p, nblocks, blocks, s, why);
  if (r) return r;
  if (!bytes) return UGKS_ERR_ARG;
  Dev d;
  memset(&d, 0, sizeof(d));
  *bytes = carve(nullptr, s, nblocks, p->precision != UGKS_FP64, p->precision == UGKS_BF16F,
                 nwork_cap_for(p, nblocks, blocks),
                 cap_interp_for(s, nblocks), d);
  return UGKS_OK;
}

int ugks_create(const ugks_params *p, void *workspace, size_t bytes, void *stream, ugks_ctx **out) {
  if (!p || !out) return UGKS_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace & 255)) return UGKS_ERR_WORKSPACE;
  ugks_ctx *c = new ugks_ctx();
  c->p = *p;
  c->ws = (char *)workspace;
  c->ws_bytes = bytes;
  c->st = (cudaStream_t)stream;
  c->fp32 = p->precision != UGKS_FP64;
  if (const char *e = getenv("UGKS_DEBUG_SYNC")) c->debug_sync = atoi(e) != 0;
  if (const char *e = getenv("UGKS_NO_GRAPH")) c->graphs = atoi(e) == 0;
  c->fbf = p->precision == UGKS_BF16F;
  memset(&c->d, 0, sizeof(c->d));
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  // the macro sweep is a latency-bound wavefront on a few SMs: give its
  // stream the highest priority so its CTAs are placed as soon as a slot frees
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->tail, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_flux, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_macro, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_bwd, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_tail, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return UGKS_ERR_CUDA;
  }
  *out = c;
  return UGKS_OK;
}

int ugks_destroy(ugks_ctx *ctx) {
  if (ctx) {
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    if (ctx->tail) cudaStreamSynchronize(ctx->tail);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    for (auto &g : ctx->gcache)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    if (ctx->ev_flux) cudaEventDestroy(ctx->ev_flux);
    if (ctx->ev_macro) cudaEventDestroy(ctx->ev_macro);
    if (ctx->ev_bwd) cudaEventDestroy(ctx->ev_bwd);
    if (ctx->ev_tail) cudaEventDestroy(ctx->ev_tail);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->tail) cudaStreamDestroy(ctx->tail);
  }
  delete ctx;
  return UGKS_OK;
}

const char *ugks_last_error(const ugks_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t ugks_launch_count(const ugks_ctx *ctx) { return ctx ? ctx->launches : 0; }

int ugks_shard_set_exchange(ugks_ctx *ctx, ugks_exchange_fn fn, void *user) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (!ctx->d.shard) return fail(ctx, UGKS_ERR_ARG, "context holds the whole velocity grid");
  if (!fn) return fail(ctx, UGKS_ERR_ARG, "null exchange function");
  ctx->xfn = fn;
  ctx->xuser = user;
  return UGKS_OK;
}

int ugks_shard_buffers(const ugks_ctx *ctx, size_t *face_off, size_t *face_count, size_t *cell_off,
                       size_t *cell_count) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  const Dev &d = ctx->d;
  if (face_off) *face_off = (size_t)((const char *)d.fsum - ctx->ws);
  if (face_count) *face_count = (size_t)NFS * d.nf;
  if (cell_off) *cell_off = (size_t)((const char *)d.msum - ctx->ws);
  if (cell_count) *cell_count = 6 * (size_t)d.nc;
  return UGKS_OK;
}

int ugks_set_wait_limit(ugks_ctx *ctx, int polls) {
  if (!ctx) return UGKS_ERR_ARG;
  if (polls < 0) return fail(ctx, UGKS_ERR_ARG, "negative poll limit");
  ctx->d.wait_polls = polls == 0 ? kWaitPolls : polls;
  return UGKS_OK;
}

int ugks_sizes(const ugks_ctx *ctx, int *ncells, int *nfaces, int *nv, int *nv_stride) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (ncells) *ncells = ctx->d.nc;
  if (nfaces) *nfaces = ctx->d.nf;
  if (nv) *nv = ctx->d.nv;
  if (nv_stride) *nv_stride = ctx->d.nvp;
  return UGKS_OK;
}

int ugks_init_mesh(ugks_ctx *ctx, int nblocks, const ugks_block_desc *blocks, const double *prim) {
  if (!ctx) return UGKS_ERR_ARG;
  Sizes s;
  std::string why;
  int r = validate(&ctx->p, nblocks, blocks, s, why);
  if (r) return fail(ctx, r, why);
  if (!prim) return fail(ctx, UGKS_ERR_ARG, "null initial state");
  for (int b = 0; b < nblocks; ++b) if (!blocks[b].x_ref) return fail(ctx, UGKS_ERR_ARG, "null x_ref");
  ctx->nblocks = nblocks;
  ctx->blocks.assign(blocks, blocks + nblocks);
  ctx->max_nj = s.max_nj;
  ctx->sweep_vpt = sweep_vpt_for(&ctx->p);
  ctx->sweep_nw = sweep_nw_for(nblocks, blocks);
  ctx->sweep_ql = wsweep_ql(max_nj_of(nblocks, blocks));
  ctx->face_tile = face_tile_default();
  if (const char *e = getenv("UGKS_FACE_TILE")) {      // tuning by hand: index of face_tile_shape
    int v = atoi(e);
    if (v >= 0 && v < face_tile_count()) ctx->face_tile = v;
  }
  if (const char *e = getenv("UGKS_SWEEP_NS")) {
    int n = atoi(e);
    if (n == 2 || n == 4 || n == 6) ctx->ns_fwd = ctx->ns_bwd = n;
  }
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      ctx->nsm = nsm;
    cudaGetLastError();
  }
  ctx->nwork = nwork_for(s.nvp, nblocks, blocks, ctx->sweep_vpt);
  if (!wsweep_fits(ctx->fp32, ctx->fbf, ctx->sweep_vpt, ctx->sweep_nw, 1, ctx->sweep_ql))
    return fail(ctx, UGKS_ERR_ARG, "micro-sweep CTA of the tallest block exceeds shared memory");
  ctx->nwork_cap = nwork_cap_for(&ctx->p, nblocks, blocks);
  ctx->cap_interp = cap_interp_for(s, nblocks);
  Dev &d = ctx->d;
  memset(&d, 0, sizeof(d));
  size_t need = carve(nullptr, s, nblocks, ctx->fp32, ctx->fbf, ctx->nwork_cap, ctx->cap_interp, d);
  if (need > ctx->ws_bytes) return fail(ctx, UGKS_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need));
  carve(ctx->ws, s, nblocks, ctx->fp32, ctx->fbf, ctx->nwork_cap, ctx->cap_interp, d);
  {
    // the trailing private arrays follow d.err in carve order
    Carver c(ctx->ws);
    Dev tmp;
    memset(&tmp, 0, sizeof(tmp));
    c.off = (size_t)((char *)d.err - ctx->ws) + 4 * sizeof(int) + 16;
    ctx->work = c.take<int>(3 * (size_t)ctx->nwork_cap + 3);
    ctx->prev_status = c.take<int>(s.nc);
    ctx->n_orphan = c.take<int>(4);
    ctx->blk_order = c.take<int>(nblocks);
  }
  d.nc = s.nc; d.nf = s.nf; d.nn = s.nn; d.nv = s.nv; d.nvp = s.nvp; d.nblocks = nblocks;
  d.nv_all = s.nv_all; d.iy0 = s.iy0; d.shard = s.nv != s.nv_all;
  d.nvx = ctx->p.nvx; d.nvy = ctx->p.nvy;
  d.Kint = ctx->p.K; d.Keff = 1 + ctx->p.K;
  d.Pr = ctx->p.Pr; d.omega = ctx->p.omega; d.mu_ref = ctx->p.mu_ref;
  d.cfl_s = ctx->p.cfl_s; d.cfl_pseudo = ctx->p.cfl_pseudo;
  d.dt = 1.0; d.idt = 1.0; d.idt_f = 1.0f;
  ctx->launches += upload_step_size(ctx);
  d.wait_polls = kWaitPolls;
  d.vbox[0] = ctx->p.vx_min; d.vbox[1] = ctx->p.vx_max; d.vbox[2] = ctx->p.vy_min; d.vbox[3] = ctx->p.vy_max;
  {
    double lam = 1.0 / (2.0 * ctx->p.farfield[3]);
    conservative(ctx->p.farfield[0], ctx->p.farfield[1], ctx->p.farfield[2], lam, d.Keff, d.Winf);
  }
  // velocity space
  std::vector<double> vx(s.nvp, 0.0), vy(s.nvp, 0.0), w(s.nvp, 0.0);
  std::vector<float> vxf(s.nvp, 0.f), vyf(s.nvp, 0.f), wf(s.nvp, 0.f);
  const ugks_params &P = ctx->p;
  double hx = (P.vx_max - P.vx_min) / (P.nvx - 1), hy = (P.vy_max - P.vy_min) / (P.nvy - 1);
  // the whole grid, and this context's rows of it (all rows unless sharded)
  std::vector<double> vxa(s.nvp_all, 0.0), vya(s.nvp_all, 0.0), wa(s.nvp_all, 0.0);
  std::vector<float> vxaf(s.nvp_all, 0.f), vyaf(s.nvp_all, 0.f), waf(s.nvp_all, 0.f), vy1(P.nvy);
  for (int iy = 0; iy < P.nvy; ++iy) {
    vy1[iy] = (float)(P.vy_min + (P.vy_max - P.vy_min) * iy / (P.nvy - 1));
    for (int ix = 0; ix < P.nvx; ++ix) {
      int k = iy * P.nvx + ix;
      vxa[k] = P.vx_min + (P.vx_max - P.vx_min) * ix / (P.nvx - 1);
      vya[k] = P.vy_min + (P.vy_max - P.vy_min) * iy / (P.nvy - 1);
      double wx = hx * ((ix == 0 || ix == P.nvx - 1) ? 0.5 : 1.0);
      double wy = hy * ((iy == 0 || iy == P.nvy - 1) ? 0.5 : 1.0);
      wa[k] = wy * wx;
      vxaf[k] = (float)vxa[k]; vyaf[k] = (float)vya[k]; waf[k] = (float)wa[k];
    }
  }
  for (int k = 0; k < s.nv; ++k) {
    int ka = s.iy0 * P.nvx + k;
    vx[k] = vxa[ka]; vy[k] = vya[ka]; w[k] = wa[ka];
    vxf[k] = vxaf[ka]; vyf[k] = vyaf[ka]; wf[k] = waf[ka];
  }
  // topology
  ctx->cell_off.assign(1, 0);
  ctx->node_off.assign(1, 0);
  for (int b = 0; b < nblocks; ++b) {
    ctx->cell_off.push_back(ctx->cell_off.back() + blocks[b].ni * blocks[b].nj);
    ctx->node_off.push_back(ctx->node_off.back() + (blocks[b].ni + 1) * (blocks[b].nj + 1));
  }
  Topo T;
  build_topology(nblocks, blocks, ctx->cell_off, ctx->node_off, s.nc, s.nn, T);
  std::vector<double> X(2 * (size_t)s.nn);
  ctx->ref_bbox.assign(4 * (size_t)nblocks, 0.0);
  for (int b = 0; b < nblocks; ++b) {
    size_t n = 2 * (size_t)(blocks[b].ni + 1) * (blocks[b].nj + 1);
    memcpy(&X[2 * (size_t)ctx->node_off[b]], blocks[b].x_ref, n * sizeof(double));
    double xl = 1e300, xh = -1e300, yl = 1e300, yh = -1e300;
    for (size_t q = 0; q < n; q += 2) {
      xl = std::min(xl, blocks[b].x_ref[q]); xh = std::max(xh, blocks[b].x_ref[q]);
      yl = std::min(yl, blocks[b].x_ref[q + 1]); yh = std::max(yh, blocks[b].x_ref[q + 1]);
    }
    double *bb = &ctx->ref_bbox[4 * (size_t)b];
    bb[0] = xl; bb[1] = yl; bb[2] = xh; bb[3] = yh;
  }
  std::vector<int> order(nblocks);
  for (int b = 0; b < nblocks; ++b) order[b] = b;
  for (int a = 0; a < nblocks; ++a)      // priority descending, block index ascending
    for (int b = a + 1; b < nblocks; ++b)
      if (blocks[order[b]].priority > blocks[order[a]].priority ||
          (blocks[order[b]].priority == blocks[order[a]].priority && order[b] < order[a]))
        std::swap(order[a], order[b]);
  std::vector<int> work = ws_work(nblocks, blocks, s.nvp, ctx->sweep_vpt, ctx->sweep_nw);
  if ((int)work.size() / 3 != ctx->nwork || ctx->nwork > ctx->nwork_cap)
    return fail(ctx, UGKS_ERR_WORKSPACE, "sweep work list");
  std::vector<int> tiles;
  for (int b = 0; b < nblocks; ++b) {
    std::vector<int> org(2 * (size_t)tile_count(blocks[b].ni, blocks[b].nj));
    tile_origins(blocks[b].ni, blocks[b].nj, org.data());
    for (size_t q = 0; q < org.size(); q += 2) { tiles.push_back(b); tiles.push_back(org[q]); tiles.push_back(org[q + 1]); }
  }
  d.ntiles = s.ntiles;
  tile_setup();
  sweep_setup();
  wsweep_setup();
  if ((r = up(ctx, (void *)d.vx, vx))) return r;
  if ((r = up(ctx, (void *)d.vy, vy))) return r;
  if ((r = up(ctx, (void *)d.w, w))) return r;
  if ((r = up(ctx, (void *)d.vxf, vxf))) return r;
  if ((r = up(ctx, (void *)d.vyf, vyf))) return r;
  if ((r = up(ctx, (void *)d.wf, wf))) return r;
  if ((r = up(ctx, (void *)d.vxa, vxa))) return r;
  if ((r = up(ctx, (void *)d.vya, vya))) return r;
  if ((r = up(ctx, (void *)d.wa, wa))) return r;
  if ((r = up(ctx, (void *)d.vxaf, vxaf))) return r;
  if ((r = up(ctx, (void *)d.vyaf, vyaf))) return r;
  if ((r = up(ctx, (void *)d.waf, waf))) return r;
  if ((r = up(ctx, (void *)d.vy1f, vy1))) return r;
  {
    // 1D trapezoid weights of the tensor grid (w_k = wy(iy) wx(ix))
    std::vector<float> wx1(ctx->p.nvx), wy1(ctx->p.nvy);
    for (int ix = 0; ix < ctx->p.nvx; ++ix) wx1[ix] = (float)(hx * ((ix == 0 || ix == ctx->p.nvx - 1) ? 0.5 : 1.0));
    for (int iy = 0; iy < ctx->p.nvy; ++iy) wy1[iy] = (float)(hy * ((iy == 0 || iy == ctx->p.nvy - 1) ? 0.5 : 1.0));
    if ((r = up(ctx, (void *)d.wx1f, wx1))) return r;
    if ((r = up(ctx, (void *)d.wy1f, wy1))) return r;
    // and in FP64 with the nodes (the FP64 path's separable velocity sums)
    std::vector<double> vx1d(ctx->p.nvx), vy1d(ctx->p.nvy), wx1d(ctx->p.nvx), wy1d(ctx->p.nvy);
    for (int ix = 0; ix < ctx->p.nvx; ++ix) {
      vx1d[ix] = vxa[ix];
      wx1d[ix] = hx * ((ix == 0 || ix == ctx->p.nvx - 1) ? 0.5 : 1.0);
    }
    for (int iy = 0; iy < ctx->p.nvy; ++iy) {
      vy1d[iy] = vya[(size_t)iy * ctx->p.nvx];
      wy1d[iy] = hy * ((iy == 0 || iy == ctx->p.nvy - 1) ? 0.5 : 1.0);
    }
    if ((r = up(ctx, (void *)d.vx1, vx1d))) return r;
    if ((r = up(ctx, (void *)d.vy1, vy1d))) return r;
    if ((r = up(ctx, (void *)d.wx1, wx1d))) return r;
    if ((r = up(ctx, (void *)d.wy1, wy1d))) return r;
  }
  if ((r = up(ctx, (void *)d.cell_nodes, T.cell_nodes))) return r;
  if ((r = up(ctx, (void *)d.cell_faces, T.cell_faces))) return r;
  if ((r = up(ctx, (void *)d.cell_sgn, T.cell_sgn))) return r;
  if ((r = up(ctx, (void *)d.nb_kind, T.nb_kind))) return r;
  if ((r = up(ctx, (void *)d.nb_id, T.nb_id))) return r;
  if ((r = up(ctx, (void *)d.nb_shift, T.nb_shift))) return r;
  if ((r = up(ctx, (void *)d.cell_row, T.cell_row))) return r;
  if ((r = up(ctx, (void *)d.cell_block, T.cell_block))) return r;
  if ((r = up(ctx, (void *)d.node_block, T.node_block))) return r;
  if ((r = up(ctx, (void *)d.face_L, T.face_L))) return r;
  if ((r = up(ctx, (void *)d.face_R, T.face_R))) return r;
  if ((r = up(ctx, (void *)d.face_a, T.face_a))) return r;
  if ((r = up(ctx, (void *)d.face_b, T.face_b))) return r;
  if ((r = up(ctx, (void *)d.face_kind, T.face_kind))) return r;
  {
    bool outflow = false;
    for (int f = 0; f < s.nf; ++f) outflow = outflow || T.face_kind[f] == BC_OUTFLOW;
    const char *e = getenv("UGKS_SERIAL_TAIL");      // 1: Step 7 and the gradients in line
    ctx->split_tail = !outflow && !d.shard && !(e && atoi(e) != 0);
    const char *e1 = getenv("UGKS_RESIDUAL_ONE_PASS");   // 1: the residual in one pass
    long steps = 0;                                       // diagonal steps of the longest macro sweep
    for (int b = 0; b < nblocks; ++b) steps = std::max(steps, 2L * (blocks[b].ni + blocks[b].nj - 1));
    double items = (double)s.nc * s.nv;
    ctx->split_residual = ctx->fp32 && !(e1 && atoi(e1) != 0) && items < kResidualWindow * (double)steps;
  }
  {
    std::vector<int> wf;
    for (int f = 0; f < s.nf; ++f)
      if (T.face_kind[f] == BC_WALL) wf.push_back(f);
    d.nwall = (int)wf.size();
    ctx->h_wall_faces = wf;
    if ((r = up(ctx, (void *)d.wall_faces, ctx->h_wall_faces))) return r;
  }
  if ((r = up(ctx, (void *)d.face_block, T.face_block))) return r;
  if ((r = up(ctx, (void *)d.face_shiftL, T.face_shiftL))) return r;
  if ((r = up(ctx, (void *)d.face_Tw, T.face_Tw))) return r;
  if ((r = up(ctx, (void *)d.wall_seg, T.wall_seg))) return r;
  if ((r = up(ctx, (void *)d.wall_seg_off, T.wall_seg_off))) return r;
  if ((r = up(ctx, (void *)d.body_ring, T.body_ring))) return r;
  if ((r = up(ctx, (void *)d.body_ring_off, T.body_ring_off))) return r;
  if ((r = up(ctx, (void *)d.cell_off, ctx->cell_off))) return r;
  if ((r = up(ctx, (void *)d.node_off, ctx->node_off))) return r;
  if ((r = up(ctx, (void *)d.blk_info, T.blk_info))) return r;
  {
    std::vector<int> mo(nblocks + 1, 0);     // diagonal-major FP32 macro records per block
    for (int b = 0; b < nblocks; ++b) mo[b + 1] = mo[b] + (blocks[b].ni + blocks[b].nj - 1) * blocks[b].nj;
    if ((r = up(ctx, (void *)d.mrec_off, mo))) return r;
  }
  if ((r = up(ctx, (void *)ctx->blk_order, order))) return r;
  if ((r = up(ctx, (void *)ctx->work, work))) return r;
  if ((r = up(ctx, (void *)d.tiles, tiles))) return r;
  if ((r = up(ctx, (void *)d.X_ref, X))) return r;
  // identity placement at t = 0
  ctx->h_affine.assign(6 * (size_t)nblocks, 0.0);
  for (int b = 0; b < nblocks; ++b) { ctx->h_affine[6 * b] = 1.0; ctx->h_affine[6 * b + 3] = 1.0; }
  if ((r = up(ctx, (void *)d.affine, ctx->h_affine))) return r;
  d.bin_cap = (int)bin_capacity(s);
  CK(cudaMemsetAsync(d.err, 0, sizeof(int), ctx->st));
  CK(cudaMemsetAsync(d.status, 0, sizeof(int) * s.nc, ctx->st));
  CK(cudaMemsetAsync(d.donors, 0xff, sizeof(int) * 5 * (size_t)s.nc, ctx->st));
  CK(cudaMemsetAsync(d.Tn, 0, (ctx->fp32 ? 8 : 16) * (size_t)s.nc * s.nvp, ctx->st));
  CK(cudaMemsetAsync(d.dfs, 0, (ctx->fp32 ? 8 : 16) * (size_t)s.nc * s.nvp, ctx->st));
  launch_move_nodes(d, ctx->st);
  CK(cudaMemcpyAsync(d.X_old, d.X_new, sizeof(double) * 2 * s.nn, cudaMemcpyDeviceToDevice, ctx->st));
  launch_geometry(d, ctx->st, ctx->fp32);
  ctx->launches += 5;
  // initial state from the primitive field (staged through cpar)
  if (s.nc * 4 > s.nc * NCP) return fail(ctx, UGKS_ERR_WORKSPACE, "staging");
  CK(cudaMemcpyAsync(d.cpar, prim, sizeof(double) * 4 * s.nc, cudaMemcpyHostToDevice, ctx->st));
  launch_init_state(d, ctx->st, d.cpar, ctx->fp32);
  ctx->launches += 1;
  CK(cudaStreamSynchronize(ctx->st));
  r = launch_status(ctx);
  if (r) return r;
  ctx->mesh_ready = true;
  ctx->t = 0.0;
  ctx->moved = false;
  r = do_connect(ctx, nullptr, true, true);
  if (r) return r;
  launch_slope_geo(d, ctx->st);
  ctx->launches += 1;
  r = check_err_flag(ctx);
  if (r) return r;
  return launch_status(ctx);
}

int ugks_move_mesh(ugks_ctx *ctx, double t_new, const double *affine) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (!affine) return fail(ctx, UGKS_ERR_ARG, "null affine");
  if (!(t_new > ctx->t)) return fail(ctx, UGKS_ERR_ARG, "t_new must exceed the current time");
  Dev &d = ctx->d;
  ctx->h_affine.assign(affine, affine + 6 * (size_t)ctx->nblocks);
  // the nodes at t become the old level; a second move before the step
  // replaces the pending one and keeps the nodes at t
  if (!ctx->moved) std::swap(d.X_old, d.X_new);
  ctx->launches += launch_upload(d.affine, ctx->h_affine.data(), sizeof(double) * 6 * ctx->nblocks, ctx->st);
  d.dt = t_new - ctx->t;
  d.idt = 1.0 / d.dt;
  d.idt_f = (float)d.idt;
  ctx->launches += upload_step_size(ctx);
  ctx->t_new = t_new;
  {
    Prof p(ctx, UGKS_PROF_GEOMETRY);
    launch_move_nodes(d, ctx->st);
    launch_geometry(d, ctx->st, ctx->fp32);
    launch_slope_geo(d, ctx->st);
  }
  ctx->launches += 6;
  ctx->moved = true;
  return launch_status(ctx);
}

int ugks_overset_connect(ugks_ctx *ctx, ugks_connect_stats *stats) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (!ctx->moved) return fail(ctx, UGKS_ERR_ORDER, "ugks_overset_connect needs a preceding ugks_move_mesh");
  int r = check_err_flag(ctx);
  if (r) return r;
  return do_connect(ctx, stats, false, true);
}

int ugks_step(ugks_ctx *ctx, double dt, int n_inner) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (!ctx->moved) return fail(ctx, UGKS_ERR_ORDER, "ugks_step needs a preceding ugks_move_mesh");
  if (n_inner < 1) return fail(ctx, UGKS_ERR_ARG, "n_inner must be >= 1");
  Dev &d = ctx->d;
  if (fabs(dt - d.dt) > 1e-12 * fabs(d.dt)) return fail(ctx, UGKS_ERR_ARG, "dt differs from the move's step");
  // graphs need a step free of host work: not while profiling or checking
  // each launch, and not on a velocity shard (its exchange runs on the host)
  bool graph = ctx->graphs && !ctx->prof_on && !ctx->debug_sync && !d.shard;
  int rx = graph ? step_graph(ctx, n_inner) : step_body(ctx, n_inner);
  if (rx) return rx;
  ctx->fresh_pending = false;
  ctx->stepped = true;
  ctx->metered = ctx->metrics;
  ctx->t = ctx->t_new;
  ctx->moved = false;
  return launch_status(ctx);
}

int ugks_set_metrics(ugks_ctx *ctx, int on) {
  if (!ctx) return UGKS_ERR_ARG;
  ctx->metrics = on != 0;
  return UGKS_OK;
}

int ugks_get_metrics(ugks_ctx *ctx, ugks_step_metrics *out) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (!out) return fail(ctx, UGKS_ERR_ARG, "null output");
  if (!ctx->metered) return fail(ctx, UGKS_ERR_ORDER, "the last ugks_step recorded no metrics");
  double m[MET_NQ];
  CK(cudaMemcpyAsync(m, ctx->d.mout, sizeof(m), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  out->res_macro_sq = m[MET_R2];
  out->res_micro_sq = m[MET_RMICRO2];
  out->fix_sq = m[MET_FIX2];
  for (int i = 0; i < 4; ++i) out->total[i] = m[MET_TOT + i];
  return launch_status(ctx);
}

int ugks_set_graphs(ugks_ctx *ctx, int on) {
  if (!ctx) return UGKS_ERR_ARG;
  ctx->graphs = on != 0;
  return UGKS_OK;
}

int ugks_graph_stats(const ugks_ctx *ctx, int64_t *captures, int64_t *replays) {
  if (!ctx) return UGKS_ERR_ARG;
  if (captures) *captures = ctx->gcaptures;
  if (replays) *replays = ctx->greplays;
  return UGKS_OK;
}

int ugks_advance_batch(ugks_ctx *const *ctx, int n, const double *t_new, const double *const *affine,
                       int n_inner, int *failed) {
  if (failed) *failed = -1;
  if (n < 0 || (n > 0 && (!ctx || !t_new || !affine))) return UGKS_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctx[i] || !ctx[i]->mesh_ready) {
      if (failed) *failed = i;
      return UGKS_ERR_ORDER;
    }
    if (ctx[i]->d.shard) {
      if (failed) *failed = i;
      return fail(ctx[i], UGKS_ERR_ARG, "velocity shards are stepped one context per call (ugks_step)");
    }
  }
  // stage-major issue order: every instance's motion, then every assembly,
  // then every step, so that all streams have work queued early
  for (int stage = 0; stage < 3; ++stage)
    for (int i = 0; i < n; ++i) {
      ugks_ctx *c = ctx[i];
      int r;
      if (stage == 0) r = ugks_move_mesh(c, t_new[i], affine[i]);
      else if (stage == 1) r = c->mesh_ready ? do_connect(c, nullptr, false, false) : UGKS_ERR_ORDER;
      else {
        c->in_batch = n > 1;
        r = ugks_step(c, c->d.dt, n_inner);
        c->in_batch = false;
      }
      if (r) {
        if (failed) *failed = i;
        return r;
      }
    }
  return UGKS_OK;
}

int ugks_autotune(ugks_ctx *ctx, int reps, int *items_out, int *vpt_out, int *ring_fwd_out, int *ring_bwd_out,
                  int *face_vk_out, int *face_nh_out) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (!ctx->stepped) return fail(ctx, UGKS_ERR_ORDER, "ugks_autotune needs a preceding ugks_step");
  if (reps < 1) reps = 3;
  Dev &d = ctx->d;
  cudaStream_t s = ctx->st;
  int fp = ctx->fp32;
  size_t fbytes = (ctx->fbf ? 4 : fp ? 8 : 16) * (size_t)d.nc * d.nvp;
  // f is restored afterwards (kept in the level-n term's buffer, which the
  // next step rewrites); the sweep buffer, the flux divergence and the face
  // sums are rewritten by every inner iteration, so the trials may use them
  CK(cudaMemcpyAsync(d.Tn, d.f, fbytes, cudaMemcpyDeviceToDevice, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int r = UGKS_OK;
  // time `launch` (reps passes after one warm-up)
  auto timed = [&](auto launch, float &ms) -> int {
    for (int rep = 0; rep <= reps; ++rep) {
      if (rep == 1) cudaEventRecord(e0, s);
      launch();
    }
    cudaEventRecord(e1, s);
    int q = cuda_check(ctx, cudaEventSynchronize(e1), "autotune");
    ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ctx->launches += reps + 1;
    return q;
  };
  // face kernels: reduction + flux divergence for every tile shape (FP32)
  int bt = ctx->face_tile;
  if (fp) {
    float best = 1e30f;
    for (int v = 0; v < face_tile_count() && !r; ++v) {
      float m1, m2;
      if ((r = timed([&] { launch_face_reduce_tile(d, s, fp, v); }, m1))) break;
      if ((r = timed([&] { launch_flux_tile(d, s, fp, v); }, m2))) break;
      if (m1 + m2 < best) { best = m1 + m2; bt = v; }
    }
  }
  // micro sweeps: velocities per lane, and per sweep the ring depth
  float best = 1e30f;
  int bv = ctx->sweep_vpt, bf = ctx->ns_fwd, bb = ctx->ns_bwd;
  for (int vpt : kTuneVpt) {
    if (r) break;
    if (!fp && vpt != 2) continue;
    if ((r = set_sweep_tiles(ctx, vpt))) break;
    float tf = 1e30f, tb = 1e30f;
    int nf = 0, nb = 0;
    for (int ns : kTuneRing) {
      if (!wsweep_fits(fp, ctx->fbf, vpt, ctx->sweep_nw, ns, ctx->sweep_ql)) continue;
      float ms;
      if ((r = timed([&] { launch_wsweep(d, s, 0, ctx->work, ctx->nwork, ctx->sweep_nw, ns, vpt, fp, ctx->sweep_ql); }, ms))) break;
      if (ms < tf) { tf = ms; nf = ns; }
      if ((r = timed([&] { launch_wsweep(d, s, 1, ctx->work, ctx->nwork, ctx->sweep_nw, ns, vpt, fp, ctx->sweep_ql); }, ms))) break;
      if (ms < tb) { tb = ms; nb = ns; }
    }
    if (r) break;
    if (nf && nb && tf + tb < best) { best = tf + tb; bv = vpt; bf = nf; bb = nb; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r) return r;
  CK(cudaMemcpyAsync(d.f, d.Tn, fbytes, cudaMemcpyDeviceToDevice, s));
  if ((r = set_sweep_tiles(ctx, bv))) return r;
  ctx->ns_fwd = bf;
  ctx->ns_bwd = bb;
  ctx->face_tile = bt;
  int vk, nh;
  face_tile_shape(fp ? bt : -1, &vk, &nh);
  if (!fp) { vk = 8; nh = 2; }
  if (items_out) *items_out = 32 * bv;
  if (vpt_out) *vpt_out = bv;
  if (ring_fwd_out) *ring_fwd_out = bf;
  if (ring_bwd_out) *ring_bwd_out = bb;
  if (face_vk_out) *face_vk_out = vk;
  if (face_nh_out) *face_nh_out = nh;
  return launch_status(ctx);
}

int ugks_moments(ugks_ctx *ctx, double *W, double *q, int32_t *status, double *wall_loads) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  Dev &d = ctx->d;
  launch_wall_loads(d, ctx->st);
  ctx->launches += 1;
  if (W) CK(cudaMemcpyAsync(W, d.W, sizeof(double) * 4 * d.nc, cudaMemcpyDefault, ctx->st));
  if (q) CK(cudaMemcpyAsync(q, d.q, sizeof(double) * 2 * d.nc, cudaMemcpyDefault, ctx->st));
  if (status) CK(cudaMemcpyAsync(status, d.status, sizeof(int) * d.nc, cudaMemcpyDefault, ctx->st));
  if (wall_loads) CK(cudaMemcpyAsync(wall_loads, d.wall_loads, sizeof(double) * 4 * d.nblocks, cudaMemcpyDefault, ctx->st));
  int r = check_err_flag(ctx);
  if (r) return r;
  return launch_status(ctx);
}

int ugks_wall_torque(ugks_ctx *ctx, const double *center, double *torque) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (!center || !torque) return fail(ctx, UGKS_ERR_ARG, "null center or torque");
  Dev &d = ctx->d;
  ctx->launches += launch_upload(d.torque_io, center, sizeof(double) * 2 * d.nblocks, ctx->st);
  double *out = d.torque_io + 2 * (size_t)d.nblocks;
  launch_wall_torque(d, ctx->st, d.torque_io, out);
  ctx->launches += 1;
  CK(cudaMemcpyAsync(torque, out, sizeof(double) * d.nblocks, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return launch_status(ctx);
}

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ugks_get_state(ugks_ctx *ctx, double *f, double *W, double *q) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  Dev &d = ctx->d;
  if (f) {
    if (!is_device_ptr(f)) return fail(ctx, UGKS_ERR_ARG, "f must be a device pointer");
    launch_f_convert(d, ctx->st, f, nullptr, ctx->fp32);
    ctx->launches += 1;
  }
  if (W) CK(cudaMemcpyAsync(W, d.W, sizeof(double) * 4 * d.nc, cudaMemcpyDefault, ctx->st));
  if (q) CK(cudaMemcpyAsync(q, d.q, sizeof(double) * 2 * d.nc, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return launch_status(ctx);
}

int ugks_set_state(ugks_ctx *ctx, const double *f, const double *W, const double *q) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  Dev &d = ctx->d;
  if (f) {
    if (!is_device_ptr(f)) return fail(ctx, UGKS_ERR_ARG, "f must be a device pointer");
    launch_f_convert(d, ctx->st, nullptr, f, ctx->fp32);
    ctx->launches += 1;
  }
  if (W) CK(cudaMemcpyAsync(d.W, W, sizeof(double) * 4 * d.nc, cudaMemcpyDefault, ctx->st));
  if (q) CK(cudaMemcpyAsync(d.q, q, sizeof(double) * 2 * d.nc, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return launch_status(ctx);
}

int ugks_get_checkpoint(ugks_ctx *ctx, double *t, double *nodes, int32_t *status) {
  if (!ctx || !ctx->mesh_ready || ctx->moved) return UGKS_ERR_ORDER;
  Dev &d = ctx->d;
  if (t) *t = ctx->t;
  if (nodes) CK(cudaMemcpyAsync(nodes, d.X_new, sizeof(double) * 2 * d.nn, cudaMemcpyDefault, ctx->st));
  if (status) CK(cudaMemcpyAsync(status, d.status, sizeof(int) * d.nc, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return launch_status(ctx);
}

int ugks_set_checkpoint(ugks_ctx *ctx, double t, const double *nodes, const int32_t *status) {
  if (!ctx || !ctx->mesh_ready || ctx->moved) return UGKS_ERR_ORDER;
  if (!nodes || !status) return fail(ctx, UGKS_ERR_ARG, "null nodes or status");
  Dev &d = ctx->d;
  // the nodes at t become the old level of the next move
  CK(cudaMemcpyAsync(d.X_new, nodes, sizeof(double) * 2 * d.nn, cudaMemcpyDefault, ctx->st));
  CK(cudaMemcpyAsync(d.status, status, sizeof(int) * d.nc, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->t = t;
  ctx->fresh_pending = false;
  return launch_status(ctx);
}

int ugks_eval_flux(ugks_ctx *ctx, double *D, double *F) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  if (!ctx->moved) return fail(ctx, UGKS_ERR_ORDER, "ugks_eval_flux needs a preceding ugks_move_mesh");
  Dev &d = ctx->d;
  if (D && !is_device_ptr(D)) return fail(ctx, UGKS_ERR_ARG, "D must be a device pointer");
  do_interp(ctx, 0);
  int r = flux_prep(ctx, 0);
  if (r) return r;
  if (D) { launch_flux_div_all(d, ctx->st, D, ctx->fp32); ctx->launches += 1; }
  if (F) CK(cudaMemcpyAsync(F, d.Fc, sizeof(double) * 4 * d.nc, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return launch_status(ctx);
}

int ugks_get_connectivity(ugks_ctx *ctx, int32_t *status, int32_t *donors, double *weights) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  Dev &d = ctx->d;
  if (status) CK(cudaMemcpyAsync(status, d.status, sizeof(int) * d.nc, cudaMemcpyDefault, ctx->st));
  if (donors) CK(cudaMemcpyAsync(donors, d.donors, sizeof(int) * 5 * d.nc, cudaMemcpyDefault, ctx->st));
  if (weights) CK(cudaMemcpyAsync(weights, d.dwgt, sizeof(double) * 5 * d.nc, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return UGKS_OK;
}

int ugks_get_geometry(ugks_ctx *ctx, double *vol_old, double *vol_new, double *xc, double *dts,
                      double *Sn, double *SUn) {
  if (!ctx || !ctx->mesh_ready) return UGKS_ERR_ORDER;
  Dev &d = ctx->d;
  if (vol_old) CK(cudaMemcpyAsync(vol_old, d.vol_old, sizeof(double) * d.nc, cudaMemcpyDefault, ctx->st));
  if (vol_new) CK(cudaMemcpyAsync(vol_new, d.vol_new, sizeof(double) * d.nc, cudaMemcpyDefault, ctx->st));
  if (xc) CK(cudaMemcpyAsync(xc, d.xc, sizeof(double) * 2 * d.nc, cudaMemcpyDefault, ctx->st));
  if (dts) CK(cudaMemcpyAsync(dts, d.dts, sizeof(double) * d.nc, cudaMemcpyDefault, ctx->st));
  if (Sn) CK(cudaMemcpyAsync(Sn, d.Sn, sizeof(double) * 2 * d.nf, cudaMemcpyDefault, ctx->st));
  if (SUn) CK(cudaMemcpyAsync(SUn, d.SUn, sizeof(double) * d.nf, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return check_err_flag(ctx);
}

int ugks_profile_enable(ugks_ctx *ctx, int on) {
  if (!ctx) return UGKS_ERR_ARG;
  if (!on) {
    int r = prof_drain(ctx);
    if (r) return r;
  }
  ctx->prof_on = on != 0;
  return UGKS_OK;
}

int ugks_profile_read(ugks_ctx *ctx, double *ms, int64_t *launches, int reset) {
  if (!ctx) return UGKS_ERR_ARG;
  int r = prof_drain(ctx);
  if (r) return r;
  for (int g = 0; g < UGKS_NPROF; ++g) {
    if (ms) ms[g] = ctx->prof_ms[g];
    if (launches) launches[g] = ctx->prof_n[g];
    if (reset) { ctx->prof_ms[g] = 0; ctx->prof_n[g] = 0; }
  }
  return UGKS_OK;
}

}  // extern "C"
