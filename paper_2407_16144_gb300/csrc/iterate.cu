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
//     at (x~_t, y~_t) on check iterations, the certificate test of T(z_t) - z_t at restart points
//     (Theorem infeas) and check iterations, then the primal blend to x_{t+1} and the primal step
//     of eq. pdhg, x~_{t+1} = proj_X(x_{t+1} - tau (c - K^T y_{t+1})).  At a restart decision it
//     also forms the column parts of the second candidate, the anchor movement
//     z^{n+1,0} - z^{n,0}; the next row kernel adds the row parts and completes its test.
//
// K x and K^T y of the blended iterates are never recomputed: the blends are linear, so the
// products are blended with the same weights from the products of the PDHG points, which the
// SpMVs deliver (K x_{t+1} = w (rho K x~_t + (1 - rho) K x_t) + (1 - w) K x^{n,0}).  Each iteration
// therefore needs exactly the two SpMVs of eq. pdhg.
#include "internal.h"
#include "iter_common.cuh"

namespace rh {

namespace {

// The FP64 iteration kernels are bound by the FP64 pipe; 128 registers a thread (16 resident
// warps per SM) keep it busy, and the register cap keeps the grid at that size.
constexpr int kFp64MaxRegs = 128;

template <int RHO2, bool GRP>
__global__ void __maxnreg__(kFp64MaxRegs)
k_row_iter(SideLayout lay, SideVals<double> vals, WalkScratch ws, const double *__restrict__ xt,
           RowVecs v, Ctl *ctl, double *part, IterConsts ic, DeferredCol dc) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning) return;
  // stage 1 here: the preceding ordinary column stage deferred its reduction (col_defers)
  const bool dcol = ctl->stage == 1 && ctl->col_deferred && !ic.adaptive;
  if (ctl->stage != 0 && !dcol) return;
  const long long t = dcol ? ctl->t + 1 : ctl->t;
  const long long k = dcol ? ctl->k_next : ctl->k;
  const long long n_ep = dcol ? ctl->n_next : ctl->n;
  const int restart = ctl->restart_pending;
  const double w = ctl->w, sigma = ctl->sigma;
  const bool check = ((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters);
  const bool rp = (k == 0 && n_ep >= 1);
  const bool cert = rp || check;
  const bool move = restart && ctl->mv_ready;
  RowAcc a;
  RowAccL al;     // long-row sums (see walk_tiles)
  a.zero();
  al.zero();
  double *my = smem + (threadIdx.x >> 5) * lay.seg;

  StepFlags fl{restart, w, sigma, check, cert, rp, (bool)move, false, ic.m_eq};
  fl.redo = ic.adaptive && ctl->redo;
  fl.keep = ic.adaptive && !RHO2;
  auto epi = [&](int i, double dot, bool lg) {
    if (lg) row_epilogue<RHO2>(i, dot, v, fl, al, a);
    else row_epilogue<RHO2>(i, dot, v, fl, a, a);
  };
  const unsigned smask = row_smask(check, cert, move);
  const unsigned mmask = row_mmask(cert, move);
  auto gdone = [&](int grp) { store_group(al, smask, ws.group_part, grp); };
  auto gather = [&](int j) { return xt[j]; };
  walk_tiles<double, double, GRP>(lay, vals, gather, my, ws, epi, gdone);

  if (cta_reduce_and_ticket(a, smask, mmask, 0u, part, &ctl->cnt_row)) {
    DcolPre pre;
    if (dcol) dcol_prefetch(dc, pre);   // in flight during the row reduction
    double r[13];
    grid_finish<7, 6, false>(part, r, smask, mmask, ws.group_part, lay.n_long_tiles);
    double rc[2] = {0.0, 0.0};
    if (dcol)   // the deferred ordinary column stage's two sums
      dcol_finish<0, true>(dc, pre, rc);
    if (threadIdx.x == 0) row_finalize(ctl, ic, r, t, k, n_ep, sigma, move, dcol, rc);
  }
}

template <int RHO2, bool GRP>
__global__ void __maxnreg__(kFp64MaxRegs)
k_col_iter(SideLayout lay, SideVals<double> vals, WalkScratch ws, const double *__restrict__ ytv,
           ColVecs v, Ctl *ctl, double *part, IterConsts ic, int phase) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning || ctl->stage != 1) return;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const int restart = ctl->restart_pending;
  const double w = ctl->w, tau = ctl->tau;
  const bool check = phase == 0 && (((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters));
  const bool rp = phase == 0 && (k == 0 && n_ep >= 1);
  const bool cert = rp || check;
  const bool move = phase == 0 && restart;
  const long long tn = phase == 0 ? t + 1 : t;     // the iteration this kernel's x_{t+1} opens
  const bool stash = ic.adaptive || ((tn + 1) % ic.check_every == 0) || (tn + 1 >= ic.max_iters);
  if (ic.adaptive && ctl->redo) {
    // adaptive step: x~_t = proj_X(x_t - tau (c - K^T y_t)) again, from the stored x_t and
    // K^T y_t, with the smaller step; no product is needed
    Acc<2, 0> a;
    a.zero();
    const double tau = ctl->tau;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < lay.nrows; j += gridDim.x * blockDim.x) {
      const double xj = v.x[j];
      const double xtn = fmin(fmax(xj - tau * (v.c[j] - v.kty[j]), v.l[j]), v.u[j]);
      v.xt[j] = xtn;
      const double dx = xj - xtn, xa = xtn - v.x0[j];
      a.s[0] += dx * dx;
      a.s[1] += xa * xa;
    }
    if (cta_reduce_and_ticket(a, 0x3u, 0u, 0u, part, &ctl->cnt_col)) {
      double r[19] = {0.0};
      grid_finish<2, 0, false>(part, r, 0x3u, 0u);
      if (threadIdx.x == 0) col_finalize(ctl, ic, r, t, false, false, false, false, phase);
    }
    return;
  }
  ColAcc a;
  ColAccL al;
  a.zero();
  al.zero();
  double *my = smem + (threadIdx.x >> 5) * lay.seg;

  StepFlags fl{restart, w, tau, check, cert, rp, move, stash, ic.m_eq};
  Tel tl;
  auto epi = [&](int j, double dot, bool lg) {
    if (lg) col_epilogue<RHO2>(j, dot, v, fl, al, a, tl);
    else col_epilogue<RHO2>(j, dot, v, fl, a, a, tl);
  };
  const unsigned smask = col_smask(check, cert, move);
  const unsigned mmask = col_mmask(cert, move);
  auto gdone = [&](int grp) { store_group(al, smask, ws.group_part, grp); };
  auto gather = [&](int j) { return ytv[j]; };
  walk_tiles<double, double, GRP>(lay, vals, gather, my, ws, epi, gdone);
  if (check) tel_flush(ctl, tl);

  if (col_defers(ic, phase, check, cert, move)) {
    cta_reduce_store(a, smask, mmask, part);   // reduced by the next row kernel
    if (threadIdx.x == 0) ctl->col_deferred = 1;
    return;
  }
  if (cta_reduce_and_ticket(a, smask, mmask, 0u, part, &ctl->cnt_col)) {
    double r[19];
    grid_finish<11, 8, false>(part, r, smask, mmask, ws.group_part, lay.n_long_tiles);
    if (threadIdx.x == 0) col_finalize(ctl, ic, r, t, check, cert, rp, move, phase);
  }
}

__global__ void k_unscale(int n, int m, const double *e, const double *xs, const double *d,
                          const double *ys, double *xo, double *yo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xo[i] = e[i] * xs[i];
  if (i < m) yo[i] = d[i] * ys[i];
}

}  // namespace

// GRP: the grouped walk for sides whose short tiles are walked several at a time.
void launch_row_iter(cudaStream_t st, const SideStore &side, const double *xt, const RowVecs &v,
                     Ctl *ctl, double *part, const IterConsts &ic, int grid, int smem,
                     const DeferredCol &dc) {
  const int threads = side.lay.cta_warps * kWarp;
  auto go = [&](auto kern) {
    kern<<<grid, threads, smem, st>>>(side.lay, side.v64, side.wa, xt, v, ctl, part, ic, dc);
  };
  const bool grp = side.lay.tile_mult > 1;
  if (ic.rho2) grp ? go(k_row_iter<1, true>) : go(k_row_iter<1, false>);
  else grp ? go(k_row_iter<0, true>) : go(k_row_iter<0, false>);
}

void launch_col_iter(cudaStream_t st, const SideStore &side, const double *yt, const ColVecs &v,
                     Ctl *ctl, double *part, const IterConsts &ic, int grid, int smem,
                     int phase) {
  const int threads = side.lay.cta_warps * kWarp;
  auto go = [&](auto kern) {
    kern<<<grid, threads, smem, st>>>(side.lay, side.v64, side.wa, yt, v, ctl, part, ic, phase);
  };
  const bool grp = side.lay.tile_mult > 1;
  if (ic.rho2) grp ? go(k_col_iter<1, true>) : go(k_col_iter<1, false>);
  else grp ? go(k_col_iter<0, true>) : go(k_col_iter<0, false>);
}

void launch_unscale(cudaStream_t st, int n, int m, const double *e, const double *xs,
                    const double *d, const double *ys, double *xo, double *yo) {
  int N = n > m ? n : m;
  k_unscale<<<(N + 255) / 256 > 0 ? (N + 255) / 256 : 1, 256, 0, st>>>(n, m, e, xs, d, ys, xo, yo);
}

void allow_large_smem(int bytes) {
  const void *k[] = {(const void *)k_row_iter<0, false>, (const void *)k_row_iter<1, false>,
                     (const void *)k_col_iter<0, false>, (const void *)k_col_iter<1, false>,
                     (const void *)k_row_iter<0, true>,  (const void *)k_row_iter<1, true>,
                     (const void *)k_col_iter<0, true>,  (const void *)k_col_iter<1, true>};
  for (const void *f : k) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Resident CTAs per SM of the FP64 iteration kernels of one side (all instantiations).
static int fp64_blocks_per_sm(const void *const *k, int nk, int smem, int threads) {
  int mn = 1 << 30;
  for (int i = 0; i < nk; ++i) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k[i], threads, smem);
    mn = b < mn ? b : mn;
  }
  return mn;
}

int row_iter_blocks_per_sm(int smem, int threads) {
  const void *k[] = {(const void *)k_row_iter<0, false>, (const void *)k_row_iter<1, false>,
                     (const void *)k_row_iter<0, true>, (const void *)k_row_iter<1, true>};
  return fp64_blocks_per_sm(k, 4, smem, threads);
}

int col_iter_blocks_per_sm(int smem, int threads) {
  const void *k[] = {(const void *)k_col_iter<0, false>, (const void *)k_col_iter<1, false>,
                     (const void *)k_col_iter<0, true>, (const void *)k_col_iter<1, true>};
  return fp64_blocks_per_sm(k, 4, smem, threads);
}

}  // namespace rh
