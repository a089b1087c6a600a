// The per-iteration hot path (FP64): two fused kernels per PDHG evaluation.
//
//   row kernel, iteration t:   K^ x~_t (tiled SpMV over the rows of K^), then per row the lazy
//     Halpern / reflected blend of the dual iterate y_t from the previous PDHG point (eq. hpdhg /
//     eq. hrpdhg, or the restart point T(z) of Algorithms 1/2), the dual step of eq. pdhg,
//     y~_t = proj_Y(y_t + sigma (q - 2 K x~_t + K x_t)), and the dual parts of the fixed-point
//     residual ||z_t - T(z_t)||_P^2.  Its last CTA completes the residual, applies the restart
//     rule of eq. adaptive-restart (Section 3) and the primal-weight update, and records the
//     decision for the next blend.
//   column kernel, iteration t: K^T y~_t (tiled SpMV over the rows of K^T), the termination test
//     at (x~_t, y~_t) on check iterations, the certificate test at restart points
//     (Theorem infeas), then the primal blend to x_{t+1} and the primal step of eq. pdhg,
//     x~_{t+1} = proj_X(x_{t+1} - tau (c - K^T y_{t+1})).
//
// K x and K^T y of the blended iterates are never recomputed: the blends are linear, so the
// products are blended with the same weights from the products of the PDHG points, which the
// SpMVs deliver (K x_{t+1} = w (rho K x~_t + (1 - rho) K x_t) + (1 - w) K x^{n,0}).  Each iteration
// therefore needs exactly the two SpMVs of eq. pdhg.
#include "internal.h"
#include "iter_common.cuh"

namespace rh {

namespace {

// sums: 0 dy2, 1 cross, 2 ya2, 3 rp2, 4 qy, 5 qv ; maxima: 0 yneg, 1 kd_eq, 2 kd_in
using RowAcc = Acc<6, 3>;
// sums: 0 dx2, 1 xa2, 2 rd2, 3 cx, 4 bnd, 5 cd, 6 uterm, 7 lterm ;
// maxima: 0 dlb, 1 dub, 2 ainf_u, 3 ainf_l
using ColAcc = Acc<8, 4>;

template <int RHO2>
__global__ void __launch_bounds__(kBlockThreads)
k_row_iter(SideLayout lay, SideVals<double> vals, WalkScratch ws, const double *__restrict__ xt,
           RowVecs v, Ctl *ctl, double *part, IterConsts ic) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning || ctl->stage != 0) return;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const int restart = ctl->restart_pending;
  const double w = ctl->w, sigma = ctl->sigma;
  const bool check = ((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters);
  const bool rp = (k == 0 && n_ep >= 1);
  const int m_eq = ic.m_eq;
  RowAcc a, al;   // al: contributions of long rows (see walk_tiles)
  a.zero();
  al.zero();
  double *my = smem + (threadIdx.x >> 5) * lay.seg;

  StepFlags fl{restart, w, sigma, check, rp, m_eq};
  auto body = [&](int i, double dot, RowAcc &acc) { row_epilogue<RHO2>(i, dot, v, fl, acc); };
  auto epi = [&](int i, double dot, bool lg) {
    if (lg) body(i, dot, al);
    else body(i, dot, a);
  };
  const unsigned smask = 0x7u | (check ? 0x18u : 0u) | (rp ? 0x20u : 0u);
  const unsigned mmask = rp ? 0x7u : 0u;
  auto gdone = [&](int grp) { store_group(al, smask, mmask, ws.group_part, grp); };
  auto gather = [&](int j) { return xt[j]; };
  walk_tiles<double, double>(lay, vals, gather, my, ws, epi, gdone);

  if (cta_reduce_and_ticket(a, smask, mmask, 0u, part, &ctl->cnt_row)) {
    double r[9];
    grid_finish<6, 3>(part, r, smask, mmask, ws.group_part, lay.n_long_tiles);
    if (threadIdx.x == 0) row_finalize(ctl, ic, r, t, k, n_ep, sigma);
  }
}

template <int RHO2>
__global__ void __launch_bounds__(kBlockThreads)
k_col_iter(SideLayout lay, SideVals<double> vals, WalkScratch ws, const double *__restrict__ ytv,
           ColVecs v, Ctl *ctl, double *part, IterConsts ic, int phase) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning || ctl->stage != 1) return;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const int restart = ctl->restart_pending;
  const double w = ctl->w, tau = ctl->tau;
  const bool check = phase == 0 && (((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters));
  const bool rp = phase == 0 && (k == 0 && n_ep >= 1);
  ColAcc a, al;
  a.zero();
  al.zero();
  double *my = smem + (threadIdx.x >> 5) * lay.seg;

  StepFlags fl{restart, w, tau, check, rp, ic.m_eq};
  auto body = [&](int j, double dot, ColAcc &acc) { col_epilogue<RHO2>(j, dot, v, fl, acc); };
  auto epi = [&](int j, double dot, bool lg) {
    if (lg) body(j, dot, al);
    else body(j, dot, a);
  };
  const unsigned smask = 0x3u | (check ? 0x1Cu : 0u) | (rp ? 0xE0u : 0u);
  const unsigned mmask = rp ? 0xFu : 0u;
  auto gdone = [&](int grp) { store_group(al, smask, mmask, ws.group_part, grp); };
  auto gather = [&](int j) { return ytv[j]; };
  walk_tiles<double, double>(lay, vals, gather, my, ws, epi, gdone);

  if (cta_reduce_and_ticket(a, smask, mmask, 0u, part, &ctl->cnt_col)) {
    double r[12];
    grid_finish<8, 4>(part, r, smask, mmask, ws.group_part, lay.n_long_tiles);
    if (threadIdx.x == 0) col_finalize(ctl, ic, r, t, check, rp, phase);
  }
}

__global__ void k_unscale(int n, int m, const double *e, const double *xs, const double *d,
                          const double *ys, double *xo, double *yo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xo[i] = e[i] * xs[i];
  if (i < m) yo[i] = d[i] * ys[i];
}

}  // namespace

void launch_row_iter(cudaStream_t st, const SideStore &side, const double *xt, const RowVecs &v,
                     Ctl *ctl, double *part, const IterConsts &ic, int grid, int smem) {
  if (ic.rho2)
    k_row_iter<1><<<grid, kBlockThreads, smem, st>>>(side.lay, side.v64, side.wa, xt, v, ctl,
                                                      part, ic);
  else
    k_row_iter<0><<<grid, kBlockThreads, smem, st>>>(side.lay, side.v64, side.wa, xt, v, ctl,
                                                      part, ic);
}

void launch_col_iter(cudaStream_t st, const SideStore &side, const double *yt, const ColVecs &v,
                     Ctl *ctl, double *part, const IterConsts &ic, int grid, int smem,
                     int phase) {
  if (ic.rho2)
    k_col_iter<1><<<grid, kBlockThreads, smem, st>>>(side.lay, side.v64, side.wa, yt, v, ctl,
                                                      part, ic, phase);
  else
    k_col_iter<0><<<grid, kBlockThreads, smem, st>>>(side.lay, side.v64, side.wa, yt, v, ctl,
                                                      part, ic, phase);
}

void launch_unscale(cudaStream_t st, int n, int m, const double *e, const double *xs,
                    const double *d, const double *ys, double *xo, double *yo) {
  int N = n > m ? n : m;
  k_unscale<<<(N + 255) / 256 > 0 ? (N + 255) / 256 : 1, 256, 0, st>>>(n, m, e, xs, d, ys, xo, yo);
}

void allow_large_smem(int bytes) {
  cudaFuncSetAttribute(k_row_iter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_row_iter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_col_iter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_col_iter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int row_iter_blocks_per_sm(int smem) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_row_iter<0>, kBlockThreads, smem);
  int b2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_row_iter<1>, kBlockThreads, smem);
  return b < b2 ? b : b2;
}

int col_iter_blocks_per_sm(int smem) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_col_iter<0>, kBlockThreads, smem);
  int b2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_col_iter<1>, kBlockThreads, smem);
  return b < b2 ? b : b2;
}

}  // namespace rh
