// ugks_launch.h -- host-side launch wrappers of the libugks kernels.
#pragma once
#include <cuda_runtime.h>
#include "ugks_internal.cuh"

namespace ugks {
int launch_upload(void *dst, const void *src, size_t n, cudaStream_t s);   // kernels launched
void launch_move_nodes(const Dev &d, cudaStream_t s);
void launch_geometry(const Dev &d, cudaStream_t s, int fp32);   // 4 kernels
void launch_slope_geo(const Dev &d, cudaStream_t s);
void launch_ghost_gradW(const Dev &d, cudaStream_t s);                      // 2 kernels
void launch_gradW(const Dev &d, cudaStream_t s);                            // the gradients alone
void launch_face_coef(const Dev &d, cudaStream_t s, int fp32);
void launch_cell_macro(const Dev &d, cudaStream_t s, int level_n);
void launch_cell_params(const Dev &d, cudaStream_t s, const double *W, double *out, int fp32);
void launch_macro_prep(const Dev &d, cudaStream_t s, int fp32);
void launch_macro_sweep(const Dev &d, cudaStream_t s, int rows, int fp32);   // sweep + post (after launch_macro_prep)
// micro LU-SGS sweeps (ugks_sweep.cu): pass 0 forward, 1 backward; nw warps
// per CTA, ns prefetch steps (1, 2, 4 or 6), vpt velocities per lane, ql
// lanes per row (4 or 2: wsweep_ql of the tallest block)
void launch_wsweep(const Dev &d, cudaStream_t s, int pass, const int *work, int nwork, int nw, int ns, int vpt,
                   int fp32, int ql);
void wsweep_setup();
int wsweep_ql(int max_nj);
int wsweep_fits(int fp32, int fbf, int vpt, int nw, int ns, int ql);
void sweep_setup();
void launch_moments(const Dev &d, cudaStream_t s, int fp32);
void launch_moments_finish(const Dev &d, cudaStream_t s);   // sharded step, after the exchange
// step metrics: stage 0 after the macro prep (|R|^2), 1 after the residual
// (|r|^2), 2 after the moments (|W - W'|^2, totals; 2 kernels)
void launch_metrics(const Dev &d, cudaStream_t s, int stage, int fp32);
void launch_init_state(const Dev &d, cudaStream_t s, const double *prim, int fp32);
void launch_flux_div_all(const Dev &d, cudaStream_t s, double *D, int fp32);
void launch_wall_loads(const Dev &d, cudaStream_t s);
void launch_wall_torque(const Dev &d, cudaStream_t s, const double *ctr, double *out);
void launch_f_convert(const Dev &d, cudaStream_t s, double *out, const double *in, int fp32);
void launch_connect(const Dev &d, cudaStream_t s, int *prev_status, const int *blk_order,
                    int *n_orphan);                           // 9 kernels
void launch_lists(const Dev &d, cudaStream_t s, const int *fresh_flag, const int *n_orphan);  // 2 kernels
// parts: 1 the distributions, 2 W and q, 3 both
void launch_interp(const Dev &d, cudaStream_t s, const int *list, const int *cnt, int nsm, int fp32,
                   int parts = 3);   // 2 kernels
// tiled kernels (ugks_tile.cu)
void tile_setup();
int tile_count(int ni, int nj);
void tile_origins(int ni, int nj, int *out);
// face kernels: `tile` indexes the tile shapes (velocities per chunk, threads
// per face slot) of face_tile_shape; the FP64 path has one shape
void launch_flux_tile(const Dev &d, cudaStream_t s, int fp32, int tile);
// part 0: the residual in one pass; 1: its part without the predictor W'
// (beside the macro sweep); 2: the collision term at W' added (after it)
void launch_residual(const Dev &d, cudaStream_t s, int first_iter, int fp32, int part = 0);
void launch_face_reduce_tile(const Dev &d, cudaStream_t s, int fp32, int tile);
int face_tile_count();
int face_tile_default();
void face_tile_shape(int tile, int *vk, int *nh);
}  // namespace ugks
