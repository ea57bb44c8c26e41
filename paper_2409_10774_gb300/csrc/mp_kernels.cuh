// Launchers of the solver kernels (host-callable; defined in mp_kernels.cu).
#pragma once

#include "mp_common.cuh"

namespace mp {

struct LaunchCfg {
  int rows = 1;    // rows per pass-A work item
  int grid_a = 1;  // pass-A grid (persistent, one error partial per block)
  int grid_y = 1;
  int grid_z = 1;
  int grid_v = 1;  // per-voxel kernels (init, commit, fields)
};

template <class R>
LaunchCfg make_launch_cfg(const CellDev<R>& c, int nsm);
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
// One fixed-point iteration; writes err and the four per-field errors to err_out[0..4].
template <class R>
cudaError_t launch_iteration(const LaunchCfg& L, const CellDev<R>& c, double* partials,
                             double* err_out, int err_kind, cudaStream_t st);
// Start of a load increment: (first ? zero state + e = E : predictor already in place),
// Algorithm 1 at the predictor, polarizations, forward x transform.
template <class R>
cudaError_t launch_start(const LaunchCfg& L, const CellDev<R>& c, int first, cudaStream_t st);
// Commit of a converged increment; avg_out[0..39] receives the homogenized averages.
template <class R>
cudaError_t launch_commit(const LaunchCfg& L, const CellDev<R>& c, int predict, double ratio,
                          double* partials, double* avg_out, cudaStream_t st);
template <class R>
cudaError_t launch_fields(const LaunchCfg& L, const CellDev<R>& c, int from_elast, double* fe,
                          double* fg, double* ft, double* fm, double* fp, double* fq, cudaStream_t st);
template <class R>
cudaError_t launch_green_apply(const LaunchCfg& L, const CellDev<R>& c, const R* tau, const R* mu,
                               R* e_out, R* g_out, cudaStream_t st);
template <class R>
cudaError_t launch_radial_return(int nsm, long long count, const uint16_t* phase,
                                 const PhaseDev<R>* phases, const R* e, const R* g, const R* e_n,
                                 const R* g_n, const R* t_n, const R* m_n, const double* p_n,
                                 const double* q_n, R* t, R* m, double* p, double* q,
                                 cudaStream_t st);

}  // namespace mp
