// Launchers of the solver kernels (host-callable; defined in mp_kernels.cu).
#pragma once

#include "mp_common.cuh"

namespace mp {

struct LaunchCfg {
  int rows = 1;    // rows per pass-A work item
  long long items_a = 1;
  int grid_a = 1;  // pass-A grid (persistent, one error partial per block)
  int grid_y = 1;
  int grid_z = 1;
  int grid_v = 1;  // per-voxel kernels (init, commit, fields)
};

// rows_wanted > 0: that many rows per pass-A item (halved until the tile fits).
template <class R>
LaunchCfg make_launch_cfg(const CellDev<R>& c, int nsm, int rows_wanted = 0);
// Whether the kernels' shared-memory tiles fit for this grid in precision R.
template <class R>
bool sizes_fit(int n1, int n2, int n3);

// The kernels of one fixed-point iteration, one launch each (y pass dir -1 forward, +1 inverse).
template <class R>
cudaError_t launch_fft_y(const LaunchCfg& L, const CellDev<R>& c, int dir, cudaStream_t st);
template <class R>
cudaError_t launch_green_z(const LaunchCfg& L, const CellDev<R>& c, cudaStream_t st);
template <class R>
cudaError_t launch_pass_a_iter(const LaunchCfg& L, const CellDev<R>& c, double* partials, cudaStream_t st);
template <class R>
cudaError_t launch_reduce_err(const LaunchCfg& L, const CellDev<R>& c, const double* partials,
                              int err_kind, double* err_out, cudaStream_t st);
// The error reduction of a loop decided on the device: additionally counts
// the iteration in err_out[6] (zeroed before the loop) and sets `handle` (a
// conditional WHILE node's) to continue while err > tol, err finite and
// <= div_limit, no failure recorded, fewer than max_iter iterations ran and
// (stag > 0) the stagnation watch (stall_step, window stag, widening when
// adapt) has not tripped (err_out[6..10]: loop iterations, last low, its
// iteration, stopped by the watch, longest gap between lows).
template <class R>
cudaError_t launch_reduce_err_loop(const LaunchCfg& L, const CellDev<R>& c, const double* partials, int err_kind,
                                   double* err_out, double tol, int max_iter, double div_limit, int stag,
                                   int adapt, cudaGraphConditionalHandle handle, cudaStream_t st);
// One fixed-point iteration; writes err and the four per-field errors to err_out[0..4].
template <class R>
cudaError_t launch_iteration(const LaunchCfg& L, const CellDev<R>& c, double* partials,
                             double* err_out, int err_kind, cudaStream_t st);
// Start of a load increment: (first ? zero state + e = E : predictor already in place),
// Algorithm 1 at the predictor, polarizations, forward x transform.
template <class R>
cudaError_t launch_start(const LaunchCfg& L, const CellDev<R>& c, int first, cudaStream_t st);
// Commit of a converged increment (c.predict / c.ratio select the predictor);
// avg_out[0..39] receives the homogenized averages.
template <class R>
cudaError_t launch_commit(const LaunchCfg& L, const CellDev<R>& c, double* partials, double* avg_out,
                          cudaStream_t st);

// Multi-cell launches: each Work lists the entries (cells) and their item
// prefix for one kernel family; the cells' descriptors live in device memory.
template <class R>
struct MultiCfg {
  Work<R> wy, wz, wa;   // iterating cells: y columns, z columns, pass-A items
  Work<R> ws;           // cells starting an increment: pass-A items
  Work<R> wv, wv0;      // 256-voxel chunks: commit, first-increment initialisation
  long long items_y = 0, items_z = 0, items_a = 0, items_s = 0, items_v = 0, items_v0 = 0;
  size_t smem_y = 0, smem_z = 0, smem_a = 0;  // largest tile over the entries (smem_a: pass A, both modes)
  int grid_y = 1, grid_z = 1, grid_a = 1, grid_s = 1, grid_v = 1, grid_v0 = 1;
};
template <class R>
void multi_grids(MultiCfg<R>& m, int nsm);
template <class R>
cudaError_t launch_multi_iteration(const MultiCfg<R>& m, cudaStream_t st);
template <class R>
cudaError_t launch_multi_start(const MultiCfg<R>& m, cudaStream_t st);
template <class R>
cudaError_t launch_multi_commit(const MultiCfg<R>& m, cudaStream_t st);
template <class R>
size_t smem_pass_a(int n1, int rows);
template <class R>
size_t smem_line_pass(int n);
template <class R>
cudaError_t launch_fields(const LaunchCfg& L, const CellDev<R>& c, int from_elast, double* fe,
                          double* fg, double* ft, double* fm, double* fp, double* fq, cudaStream_t st);
// ctl (FP32 cells with spectral_fused_ok only; else NULL): the fused spectral
// pass's control words, which select it for the y / z work.
template <class R>
cudaError_t launch_green_apply(const LaunchCfg& L, const CellDev<R>& c, const R* tau, const R* mu,
                               R* e_out, R* g_out, cudaStream_t st, int* ctl = nullptr, int nsm = 0);
template <class R>
cudaError_t launch_radial_return(int nsm, long long count, const uint16_t* phase,
                                 const PhaseDev<R>* phases, const R* e, const R* g, const R* e_n,
                                 const R* g_n, const R* t_n, const R* m_n, const double* p_n,
                                 const double* q_n, R* t, R* m, double* p, double* q,
                                 cudaStream_t st);

// Fused spectral pass (y forward, z forward, Green operator, z inverse, y
// inverse in one persistent launch; mp_spectral.cu) for FP32 cells whose y
// and z lengths are 256.  ctl: spectral_ctl_ints(c.kx) ints of device memory
// (zeroed by the launcher on `st`).
bool spectral_fused_ok(const CellDev<float>& c);
size_t spectral_ctl_ints(int kx);
cudaError_t launch_spectral(const CellDev<float>& c, int* ctl, int nsm, cudaStream_t st);

// dst[i] = (D) src[i], i < n (state of a cell changing precision).
template <class S, class D>
cudaError_t launch_convert(const S* src, D* dst, long long n, int nsm, cudaStream_t st);

}  // namespace mp
