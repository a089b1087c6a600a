// Mixed-precision hot path: FP32 matrix values and FP32 iterates stored as offsets from FP64
// anchors, FP64 for the anchors z^{n,0}, their products K x^{n,0} and K^T y^{n,0}, the restart and
// termination reductions, and every restart's re-anchoring.
//
// Representation.  Within epoch n the iterate and its PDHG point are
//     x_t = x0 + dx_t,  x~_t = x0 + dxt_t,  y_t = y0 + dy_t,  y~_t = y0 + dyt_t
// with (x0, y0) = z^{n,0} in FP64 and the offsets in FP32.  Because the Halpern blends of
// eq. hpdhg / eq. hrpdhg are affine with weights summing to one, the offsets blend exactly like
// the iterates with the anchor's offset equal to zero:
//     rHPDHG   dx_{t+1} = w dxt_t                 r2HPDHG  dx_{t+1} = w (2 dxt_t - dx_t)
// and the products of the offsets blend the same way, so K x_t = K x0 + K dx_t needs only the FP32
// product K dxt_t of each iteration.  The steps of eq. pdhg become, per element,
//     dxt = clamp(dx + s0 + tau K^T dy,  xlo, xhi),   s0 = -tau (c - K^T y0),
//                                                     xlo = l - x0 (rounded up), xhi = u - x0 (down)
//     dyt = dy + r0 + sigma (K dx - 2 K dxt)  [>= ylo on G rows],
//                                                     r0 = sigma (q - K x0), ylo = -y0 (rounded up)
// where s0, r0, xlo, xhi, ylo are FP32 images of FP64 anchor quantities, recomputed at each
// restart.  Precision is therefore relative to the size of the offsets, which shrink as the
// method converges; the bound offsets are zero exactly when the anchor sits on its bound, and
// rounding them towards the feasible side keeps every PDHG point inside [l, u] and y_G >= 0.
//
// Restart (Algorithms 1/2: z^{n+1,0} = T(z^{n,k})).  The column kernel that follows a restart
// decision forms x0' = x0 + dxt and computes K^T y0' with the FP64 matrix directly from the
// gathered sum y0 + dyt (no FP32 rounding of the anchor), and the first PDHG point of the new
// epoch in FP64; the next row kernel forms y0', computes K x0' and the new dual step with the
// FP64 matrix, and the column kernel after it K^T (y~ - y0') in FP64.  The restart point's
// displacement T(z^{n,0}) - z^{n,0}, the certificate candidate of Theorem infeas, is therefore
// exact to FP64; all offsets restart from there.
#include <type_traits>

#include "internal.h"
#include "iter_common.cuh"
#include "iter_mx_common.cuh"

namespace rh {

namespace {

// Matrix values of the ordinary kernels: FP32 (LP = 0) or BF16 (LP = 1, precision 2: exact
// values of a matrix of at most 8 significant bits under power-of-two scaling).
template <int LP>
using LowT = std::conditional_t<LP == 1, __nv_bfloat16, float>;

// packed slots of the CTA accumulators: the restart-norm sums of the ordinary kernels
template <int MODE>
constexpr int row_df_slots() { return MODE == 0 ? 3 : 0; }
template <int MODE>
constexpr int col_df_slots() { return MODE == 0 ? 2 : 0; }

// Register budgets: the ordinary kernels (MODE 0) of the plain and grouped walks 64 (32 resident
// warps per SM), the wide walk 80 (96 with double-float sums), the restart kernels (MODE 1) 128.
// The CTA width is chosen at launch (up to kMaxBlockThreads).
__host__ __device__ constexpr int mx_max_regs(int mode, int walk, int dfs) {
  return mode == 1 ? 128 : (walk == kWalkWide ? (dfs ? 96 : 80) : 64);
}

// MODE 0 runs the ordinary (FP32) iterations and returns at once when a restart is pending;
// MODE 1 runs only the restart iterations (FP64 walks) and returns at once otherwise.  Both are
// launched every iteration; splitting them keeps the register footprint of the FP32 kernel small.
// CP: the matrix stream's cache policy of the ordinary kernels' walk (see Vec4 in common.cuh).
template <int RHO2, int MODE, int WALK, int DFS, int LP, int CP = 0>
__global__ void __maxnreg__(mx_max_regs(MODE, WALK, DFS))
k_row_iter_mx(SideLayout lay, SideVals<double> v64, SideVals<LowT<LP>> v32, WalkScratch wa,
              WalkScratch wb, RowVecsMx v, const float *__restrict__ dxt,
              const double *__restrict__ dxt64, const double *__restrict__ x0, Ctl *ctl,
              double *part, IterConsts ic, DeferredCol dc) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning) return;
  // stage 1 here: the preceding ordinary column stage deferred its reduction (col_defers); this
  // iteration is the one after it (an ordinary column stage leaves no restart pending)
  const int stage = ctl->stage;
  const bool dcol = MODE == 0 && stage == 1 && ctl->col_deferred;
  if (stage != 0 && !dcol) return;
  const int restart = ctl->restart_pending;
  if (restart != MODE) return;
  const long long t = dcol ? ctl->t + 1 : ctl->t;
  const long long k = dcol ? ctl->k_next : ctl->k;
  const long long n_ep = dcol ? ctl->n_next : ctl->n;
  const double w = ctl->w, sigma = ctl->sigma;
  const float wf = (float)w, sigf = (float)sigma;
  const bool check = ((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters);
  const bool rp = (k == 0 && n_ep >= 1);
  const bool move = restart && ctl->mv_ready;
  const int m_eq = ic.m_eq;
  // staging: FP64 walks use (32 L + 4) doubles per warp, FP32 walks (32 L + 4) floats (the
  // FP32-only kernels are launched with half the shared memory)
  double *my64 = smem + (threadIdx.x >> 5) * lay.seg;
  float *my32 = reinterpret_cast<float *>(smem) + (threadIdx.x >> 5) * lay.seg;
  constexpr int ND = row_df_slots<MODE>();
  Acc<7, 6, ND, DFS == 1> a;
  Acc<7, 0, ND, DFS == 1> al;   // long-row sums (see walk_tiles); long-row maxima go to a
  a.zero();
  al.zero();
  const unsigned smask = row_smask(check, rp, move);
  const unsigned mmask = row_mmask(rp, move);

  if constexpr (MODE == 1) {
    // Restart point z^{n+1,0} = T(z^{n,k}).  First K x0' with the FP64 matrix (x0' was formed by
    // the preceding column kernel); then, in FP64 throughout, K dxt (dxt = x~ - x0' of this
    // iteration, exact in dxt64) and the dual step, so the restart point's T(z) - z, which
    // Theorem infeas uses as the certificate candidate, carries no FP32 rounding.
    // With move set, the old anchor first gives the row parts of the anchor movement
    // z^{n+1,0} - z^{n,0} (y0' = y0 + dyt, K x0' from this walk), in FP64.
    auto epiA = [&](int i, double dot, bool lg) {
      if (move) {
        if (lg) row_mx_move(i, dot, v, m_eq, al, a);
        else row_mx_move(i, dot, v, m_eq, a, a);
      }
      v.kx0[i] = dot;
    };
    auto gA = [&](int j) { return x0[j]; };
    auto gdoneA = [&](int grp) { store_group(al, smask & 0x40u, wb.group_part, grp); };
    walk_tiles<double, double>(lay, v64, gA, my64, wa, epiA, gdoneA);
    auto epi = [&](int i, double kd, bool lg) {
      if (lg) row_mx_restart<RHO2>(i, kd, v, sigma, m_eq, check, rp, al, a);
      else row_mx_restart<RHO2>(i, kd, v, sigma, m_eq, check, rp, a, a);
    };
    auto gdone = [&](int grp) { store_group(al, smask & ~0x40u, wb.group_part, grp); };
    auto gB = [&](int j) { return dxt64[j]; };
    walk_tiles<double, double>(lay, v64, gB, my64, wb, epi, gdone);
  } else {
    FprSums<3, DFS> fa, fl;   // restart-norm sums of short rows and of long rows
    auto epi = [&](int i, float kd, bool lg) {
      if (lg) row_mx_ordinary<RHO2>(i, kd, v, wf, sigf, m_eq, check, al, fl);
      else row_mx_ordinary<RHO2>(i, kd, v, wf, sigf, m_eq, check, a, fa);
    };
    auto gdone = [&](int grp) {
      fl.flush(al);
      store_group(al, smask, wb.group_part, grp);
    };
    auto gB = [&](int j) { return dxt[j]; };
    auto pre = [&](int i) {
      prefetch_l1(v.dyt + i);
      prefetch_l1(v.kdxt + i);
      if (RHO2) {
        prefetch_l1(v.dy + i);
        prefetch_l1(v.kdx + i);
      }
      prefetch_l1(v.r0 + i);
      if (i >= m_eq) prefetch_l1(v.ylo + i);
    };
    walk_tiles<LowT<LP>, float, WALK == kWalkGrouped, walk_unroll(WALK), CP>(lay, v32, gB, my32, wb,
                                                                       epi, gdone, pre);
    fa.flush(a);
  }
  if (cta_reduce_and_ticket(a, smask, mmask, 0u, part, &ctl->cnt_row)) {
    DcolPre pre;
    if (dcol) dcol_prefetch(dc, pre);   // in flight during the row reduction
    double r[13];
    grid_finish<7, 6, true, ND, DFS == 1>(part, r, smask, mmask, wb.group_part,
                                          lay.n_long_tiles);
    double rc[2] = {0.0, 0.0};
    if (dcol)   // the deferred ordinary column stage's two sums (its packed slots)
      dcol_finish<col_df_slots<0>(), DFS == 1>(dc, pre, rc);
    if (threadIdx.x == 0) row_finalize(ctl, ic, r, t, k, n_ep, sigma, move, dcol, rc);
  }
}

// MODE 0: ordinary iterations (no pending restart, not a restart point); MODE 1: the rest.
template <int RHO2, int MODE, int WALK, int DFS, int LP, int CP = 0>
__global__ void __maxnreg__(mx_max_regs(MODE, WALK, DFS))
k_col_iter_mx(SideLayout lay, SideVals<double> v64, SideVals<LowT<LP>> v32, WalkScratch wa,
              WalkScratch wb, ColVecsMx v, const float *__restrict__ dyt,
              const double *__restrict__ dyt64, const double *__restrict__ y0, Ctl *ctl,
              double *part, IterConsts ic, int phase) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning || ctl->stage != 1) return;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const int restart = ctl->restart_pending;
  const bool rp = phase == 0 && (k == 0 && n_ep >= 1);
  if ((restart || rp) != (MODE == 1)) return;
  const bool move = phase == 0 && restart;
  const double w = ctl->w, tau = ctl->tau;
  const float wf = (float)w, tauf = (float)tau;
  const bool check = phase == 0 && (((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters));
  const bool no_upper = ic.no_upper;
  // staging: FP64 walks use (32 L + 4) doubles per warp, FP32 walks (32 L + 4) floats (the
  // FP32-only kernels are launched with half the shared memory)
  double *my64 = smem + (threadIdx.x >> 5) * lay.seg;
  float *my32 = reinterpret_cast<float *>(smem) + (threadIdx.x >> 5) * lay.seg;
  constexpr int ND = col_df_slots<MODE>();
  Acc<11, 8, ND, DFS == 1> a;
  Acc<11, 0, ND, DFS == 1> al;  // long-row sums (see walk_tiles); long-row maxima go to a
  a.zero();
  al.zero();
  FprSums<2, DFS> fa, fl;   // restart-norm sums of the ordinary iterations (MODE 0)
  Tel tl;         // active-set telemetry (ordinary check iterations)
  const unsigned smask = col_smask(check, rp, move);
  const unsigned mmask = col_mmask(rp, move);

  auto gdone = [&](int grp) {
    if constexpr (MODE == 0) fl.flush(al);
    store_group(al, smask, (restart ? wa : wb).group_part, grp);
  };

  if constexpr (MODE == 1) {
   if (restart) {
    // z^{n+1,0} = T(z^{n,k}): K^T y0' exactly (FP64 matrix, gathered y0 + dyt), x0' = x0 + dxt,
    // and the next PDHG point x~_{t+1} - x0' in FP64 (kept in dxt64 for the restart point's
    // certificate test)
    auto epi = [&](int j, double kty, bool lg) {
      if (lg) col_mx_restart<RHO2>(j, kty, v, tau, check, rp, move, al, a);
      else col_mx_restart<RHO2>(j, kty, v, tau, check, rp, move, a, a);
    };
    auto gA = [&](int i) { return y0[i] + (double)dyt[i]; };
    walk_tiles<double, double>(lay, v64, gA, my64, wa, epi, gdone);
   } else {
    // first iteration of an epoch: K^T (y~ - y0) in FP64 from the exact dyt64 of the row kernel
    auto epi = [&](int j, double ktd, bool lg) {
      if (lg) col_mx_first<RHO2>(j, ktd, v, wf, tauf, check, rp, no_upper, al, a);
      else col_mx_first<RHO2>(j, ktd, v, wf, tauf, check, rp, no_upper, a, a);
    };
    auto gA = [&](int i) { return dyt64[i]; };
    walk_tiles<double, double>(lay, v64, gA, my64, wb, epi, gdone);
   }
  } else {
    auto epi = [&](int j, float ktdyt, bool lg) {
      if (lg) col_mx_ordinary<RHO2>(j, ktdyt, v, wf, tauf, check, no_upper, al, a, fl, tl);
      else col_mx_ordinary<RHO2>(j, ktdyt, v, wf, tauf, check, no_upper, a, a, fa, tl);
    };
    auto gB = [&](int i) { return dyt[i]; };
    auto pre = [&](int j) {
      prefetch_l1(v.dxt + j);
      if (RHO2) {
        prefetch_l1(v.dx + j);
        prefetch_l1(v.ktdy + j);
      }
      prefetch_l1(v.s0 + j);
      prefetch_l1(v.xlo + j);
      if (!no_upper) prefetch_l1(v.xhi + j);
    };
    walk_tiles<LowT<LP>, float, WALK == kWalkGrouped, walk_unroll(WALK), CP>(lay, v32, gB, my32, wb,
                                                                       epi, gdone, pre);
    if (check) tel_flush(ctl, tl);
    fa.flush(a);
  }
  if (MODE == 0 && col_defers(ic, phase, check, rp, move)) {
    cta_reduce_store(a, smask, mmask, part);   // reduced by the next row kernel
    if (threadIdx.x == 0) ctl->col_deferred = 1;
    return;
  }
  if (cta_reduce_and_ticket(a, smask, mmask, 0u, part, &ctl->cnt_col)) {
    double r[19];
    grid_finish<11, 8, true, ND, DFS == 1>(part, r, smask, mmask,
                                           (restart ? wa : wb).group_part, lay.n_long_tiles);
    if (threadIdx.x == 0) col_finalize(ctl, ic, r, t, check, rp, rp, move, phase, MODE == 0);
  }
}

// unscaled outputs: x = E (x0 + dxt) is already xout's E-image at checks; y = D (y0 + dyt)
__global__ void k_unscale_mx(int n, int m, const double *e, const double *xs, const double *d,
                             const double *y0, const float *dyt, double *xo, double *yo,
                             double *yt64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xo[i] = e[i] * xs[i];
  if (i < m) {
    const double y = y0[i] + (double)dyt[i];
    yt64[i] = y;
    yo[i] = d[i] * y;
  }
}

__global__ void k_zero_f32(int n, float *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 0.f;
}

}  // namespace

// The restart-mode kernel (MODE 1) of each stage is launched first and returns at entry unless
// the stage needs it; the ordinary kernel (MODE 0) follows, in the instantiation of the side's
// walk (SideLayout::walk) and of the solve's restart-norm sums (IterConsts::df_sums).
template <int V>
using IC = std::integral_constant<int, V>;

// f(IC<walk>) for the walks a side's ordinary kernel may take (the wide staging round is a row
// side instantiation only)
template <bool ROW, class F>
void with_walk(int walk, F &&f) {
  if (walk == kWalkGrouped) f(IC<kWalkGrouped>{});
  else if (ROW && walk == kWalkWide) f(IC<ROW ? kWalkWide : kWalkPlain>{});
  else f(IC<kWalkPlain>{});
}

template <class F>
void with_rho_dfs(int rho2, int dfs, F &&f) {
  auto g = [&](auto R) { dfs ? f(R, IC<1>{}) : f(R, IC<0>{}); };
  rho2 ? g(IC<1>{}) : g(IC<0>{});
}

// grid: CTAs of the ordinary kernel; grid1: CTAs of the restart-mode kernel, at most one resident
// wave (its walk and its grid reduction serve any grid), so that its launch, which returns at
// entry in all but a few iterations, takes a single wave of CTAs.
void launch_row_iter_mx(cudaStream_t st, const SideStore &side, const RowVecsMx &v,
                        const float *dxt, const double *dxt64, const double *x0, Ctl *ctl,
                        double *part, const IterConsts &ic, int grid, int grid1, int smem,
                        const DeferredCol &dc) {
  const int threads = side.lay.cta_warps * kWarp;
  auto go = [&](auto kern, int g, int sm, auto vals) {
    kern<<<g, threads, sm, st>>>(side.lay, side.v64, vals, side.wa, side.wb, v, dxt, dxt64, x0,
                                 ctl, part, ic, dc);
  };
  with_rho_dfs(ic.rho2, ic.df_sums, [&](auto R, auto D) {
    go(k_row_iter_mx<R(), 1, kWalkGrouped, 0, 0>, grid1, smem, side.v32);
    with_walk<true>(side.lay.walk, [&](auto W) {
      // evict-first matrix stream only for FP32 values with FP32 restart-norm sums (the
      // default); with BF16 values it measured slower
      const bool cp = ic.l2_first && ic.df_sums == 0;
      if (ic.bf16) go(k_row_iter_mx<R(), 0, W(), 0, 1>, grid, smem / 2, side.v16);
      else if (cp) go(k_row_iter_mx<R(), 0, W(), 0, 0, 1>, grid, smem / 2, side.v32);
      else go(k_row_iter_mx<R(), 0, W(), D(), 0>, grid, smem / 2, side.v32);
    });
  });
}

void launch_col_iter_mx(cudaStream_t st, const SideStore &side, const ColVecsMx &v,
                        const float *dyt, const double *dyt64, const double *y0, Ctl *ctl,
                        double *part, const IterConsts &ic, int grid, int grid1, int smem,
                        int phase) {
  const int threads = side.lay.cta_warps * kWarp;
  auto go = [&](auto kern, int g, int sm, auto vals) {
    kern<<<g, threads, sm, st>>>(side.lay, side.v64, vals, side.wa, side.wb, v, dyt, dyt64, y0,
                                 ctl, part, ic, phase);
  };
  with_rho_dfs(ic.rho2, ic.df_sums, [&](auto R, auto D) {
    go(k_col_iter_mx<R(), 1, kWalkGrouped, 0, 0>, grid1, smem, side.v32);
    with_walk<false>(side.lay.walk, [&](auto W) {
      const bool cp = ic.l2_first && ic.df_sums == 0;
      if (ic.bf16) go(k_col_iter_mx<R(), 0, W(), 0, 1>, grid, smem / 2, side.v16);
      else if (cp) go(k_col_iter_mx<R(), 0, W(), 0, 0, 1>, grid, smem / 2, side.v32);
      else go(k_col_iter_mx<R(), 0, W(), D(), 0>, grid, smem / 2, side.v32);
    });
  });
}

void launch_unscale_mx(cudaStream_t st, int n, int m, const double *e, const double *xs,
                       const double *d, const double *y0, const float *dyt, double *xo,
                       double *yo, double *yt64) {
  int N = n > m ? n : m;
  k_unscale_mx<<<(N + 255) / 256 > 0 ? (N + 255) / 256 : 1, 256, 0, st>>>(n, m, e, xs, d, y0, dyt,
                                                                           xo, yo, yt64);
}

void zero_f32(cudaStream_t st, int n, float *x) {
  if (n > 0) k_zero_f32<<<(n + 255) / 256, 256, 0, st>>>(n, x);
}

void allow_large_smem_mx(int bytes) {
  auto set = [&](const void *f) {
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  for (int rho2 = 0; rho2 < 2; ++rho2)
    for (int dfs = 0; dfs < 2; ++dfs)
      with_rho_dfs(rho2, dfs, [&](auto R, auto D) {
        set((const void *)k_row_iter_mx<R(), 1, kWalkGrouped, 0, 0>);
        set((const void *)k_col_iter_mx<R(), 1, kWalkGrouped, 0, 0>);
        for (int w : {kWalkPlain, kWalkWide, kWalkGrouped}) {
          with_walk<true>(w, [&](auto W) {
            set((const void *)k_row_iter_mx<R(), 0, W(), D(), 0>);
            set((const void *)k_row_iter_mx<R(), 0, W(), 0, 1>);
            set((const void *)k_row_iter_mx<R(), 0, W(), 0, 0, 1>);
          });
          with_walk<false>(w, [&](auto W) {
            set((const void *)k_col_iter_mx<R(), 0, W(), D(), 0>);
            set((const void *)k_col_iter_mx<R(), 0, W(), 0, 1>);
            set((const void *)k_col_iter_mx<R(), 0, W(), 0, 0, 1>);
          });
        }
      });
}

int iter_mx_restart_blocks_per_sm(int smem, bool row, int threads) {
  int mn = 1 << 30;
  auto occ = [&](const void *f) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, threads, smem);
    mn = b < mn ? b : mn;
  };
  if (row) {
    occ((const void *)k_row_iter_mx<0, 1, kWalkGrouped, 0, 0>);
    occ((const void *)k_row_iter_mx<1, 1, kWalkGrouped, 0, 0>);
  } else {
    occ((const void *)k_col_iter_mx<0, 1, kWalkGrouped, 0, 0>);
    occ((const void *)k_col_iter_mx<1, 1, kWalkGrouped, 0, 0>);
  }
  return mn;
}

int iter_mx_blocks_per_sm(int smem, bool row, int walk, int threads, int dfs, int lp) {
  // the ordinary kernels of one side in one walk instantiation, one kind of restart-norm sums
  // and one value type (both reflection settings)
  int mn = 1 << 30;
  auto occ = [&](const void *f) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, threads, smem / 2);
    mn = b < mn ? b : mn;
  };
  for (int rho2 = 0; rho2 < 2; ++rho2)
    with_rho_dfs(rho2, dfs, [&](auto R, auto D) {
      // both cache-policy instantiations of FP32 values (the choice is made after the geometry)
      if (row)
        with_walk<true>(walk, [&](auto W) {
          occ(lp ? (const void *)k_row_iter_mx<R(), 0, W(), 0, 1>
                 : (const void *)k_row_iter_mx<R(), 0, W(), D(), 0>);
          if (!lp) occ((const void *)k_row_iter_mx<R(), 0, W(), 0, 0, 1>);
        });
      else
        with_walk<false>(walk, [&](auto W) {
          occ(lp ? (const void *)k_col_iter_mx<R(), 0, W(), 0, 1>
                 : (const void *)k_col_iter_mx<R(), 0, W(), D(), 0>);
          if (!lp) occ((const void *)k_col_iter_mx<R(), 0, W(), 0, 0, 1>);
        });
    });
  return mn;
}

}  // namespace rh
