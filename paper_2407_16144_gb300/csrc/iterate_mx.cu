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
#include "internal.h"
#include "iter_common.cuh"

namespace rh {

namespace {

// The restart test's norms (||dy||^2, dy^T K dx, ||y~ - y0||^2 and ||dx||^2, ||x~ - x0||^2) of
// the ordinary kernels are double-float sums (common.cuh) of exact products of the FP32 offsets:
// FP64-grade sums that run on the FP32 pipe.  The restart kernels (MODE 1) sum in FP64.
template <int MODE>
constexpr int row_df_slots() { return MODE == 0 ? 3 : 0; }
template <int MODE>
constexpr int col_df_slots() { return MODE == 0 ? 2 : 0; }
__device__ __forceinline__ void df_acc(DF &d, float a, float b) { d = df_add(d, df_prod(a, b)); }

// Register budgets: the ordinary kernels (MODE 0) of the plain and grouped walks 64 (32 resident
// warps per SM), the wide walk 80, the restart kernels (MODE 1) 128.  The CTA width is chosen
// at launch (up to kMaxBlockThreads).
__host__ __device__ constexpr int mx_max_regs(int mode, int walk) {
  return mode == 1 ? 128 : (walk == kWalkWide ? 80 : 64);
}

// MODE 0 runs the ordinary (FP32) iterations and returns at once when a restart is pending;
// MODE 1 runs only the restart iterations (FP64 walks) and returns at once otherwise.  Both are
// launched every iteration; splitting them keeps the register footprint of the FP32 kernel small.
template <int RHO2, int MODE, int WALK>
__global__ void __maxnreg__(mx_max_regs(MODE, WALK))
k_row_iter_mx(SideLayout lay, SideVals<double> v64, SideVals<float> v32, WalkScratch wa,
              WalkScratch wb, RowVecsMx v, const float *__restrict__ dxt,
              const double *__restrict__ dxt64, const double *__restrict__ x0, Ctl *ctl,
              double *part, IterConsts ic) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning || ctl->stage != 0) return;
  const int restart = ctl->restart_pending;
  if (restart != MODE) return;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
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
  Acc<7, 6, ND> a;
  Acc<7, 0, ND> al;     // long-row sums (see walk_tiles); long-row maxima go to a
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
    auto moveparts = [&](int i, double dot, auto &S) {
      const double y0i = v.y0[i];
      const double dyb = (y0i + (double)v.dyt[i]) - y0i;
      const double kdb = (dot - v.kx0[i]) * v.dinv[i];
      const double di = v.d[i];
      S.s[6] += v.q[i] * dyb;
      if (i >= m_eq) a.mx[3] = fmax(a.mx[3], fmax(-dyb * di, 0.0));
      if (i < m_eq) a.mx[4] = fmax(a.mx[4], fabs(kdb));
      else a.mx[5] = fmax(a.mx[5], fmax(-kdb, 0.0));
      v.certy2[i] = dyb * di;
    };
    auto epiA = [&](int i, double dot, bool lg) {
      if (move) {
        if (lg) moveparts(i, dot, al);
        else moveparts(i, dot, a);
      }
      v.kx0[i] = dot;
    };
    auto gA = [&](int j) { return x0[j]; };
    auto gdoneA = [&](int grp) { store_group(al, smask & 0x40u, wb.group_part, grp); };
    walk_tiles<double, double>(lay, v64, gA, my64, wa, epiA, gdoneA);
    auto body = [&](int i, double kd, auto &A) {
      const double y0i = v.y0[i] + (double)v.dyt[i];     // y0' = y~ of the restart iteration
      v.y0[i] = y0i;
      const double kx0i = __ldcg(v.kx0 + i);              // may come from another warp
      const double qi = v.q[i];
      v.r0[i] = (float)(sigma * (qi - kx0i));
      v.ylo[i] = (i >= m_eq) ? __double2float_ru(-y0i) : -INFINITY;
      if (RHO2) { v.dy[i] = 0.f; v.kdx[i] = 0.f; }
      double nd = sigma * (qi - kx0i - 2.0 * kd);
      if (i >= m_eq) nd = fmax(nd, -y0i);
      v.dyt64[i] = nd;
      v.dyt[i] = (float)nd;
      v.kdxt[i] = (float)kd;
      A.s[0] += nd * nd;            // dy = 0
      A.s[1] += -nd * (-kd);        // (dy - dyt) (K dx - K dxt) with dy = 0, K dx = 0
      A.s[2] += nd * nd;
      if (check) {
        double r = (qi - kx0i - kd) * v.dinv[i];
        if (i >= m_eq) r = fmax(r, 0.0);
        A.s[3] += r * r;
        A.s[4] += qi * (y0i + nd);
      }
      if (rp) {
        A.s[5] += qi * nd;
        const double di = v.d[i];
        if (i >= m_eq) a.mx[0] = fmax(a.mx[0], fmax(-nd * di, 0.0));
        const double kdd = kd * v.dinv[i];
        if (i < m_eq) a.mx[1] = fmax(a.mx[1], fabs(kdd));
        else a.mx[2] = fmax(a.mx[2], fmax(-kdd, 0.0));
        v.certy[i] = nd * di;
      }
    };
    auto epi = [&](int i, double kd, bool lg) {
      if (lg) body(i, kd, al);
      else body(i, kd, a);
    };
    auto gdone = [&](int grp) { store_group(al, smask & ~0x40u, wb.group_part, grp); };
    auto gB = [&](int j) { return dxt64[j]; };
    walk_tiles<double, double>(lay, v64, gB, my64, wb, epi, gdone);
  } else {
    auto body = [&](int i, float kd, auto &A) {
      const float dytp = v.dyt[i], kdxtp = v.kdxt[i];
      float dy, kdx;
      if (RHO2) {
        dy = wf * (2.f * dytp - v.dy[i]);
        kdx = wf * (2.f * kdxtp - v.kdx[i]);
        v.dy[i] = dy;
        v.kdx[i] = kdx;
      } else {
        dy = wf * dytp;
        kdx = wf * kdxtp;
      }
      float nd = dy + v.r0[i] + sigf * (kdx - 2.f * kd);
      if (i >= m_eq) nd = fmaxf(nd, v.ylo[i]);
      v.dyt[i] = nd;
      v.kdxt[i] = kd;
      const float ddy = dy - nd;
      df_acc(A.d[0], ddy, ddy);
      df_acc(A.d[1], ddy, kdx - kd);
      df_acc(A.d[2], nd, nd);
      if (check) {
        const double qi = v.q[i];
        double r = (qi - v.kx0[i] - (double)kd) * v.dinv[i];
        if (i >= m_eq) r = fmax(r, 0.0);
        A.s[3] += r * r;
        A.s[4] += qi * (v.y0[i] + (double)nd);
      }
    };
    auto epi = [&](int i, float kd, bool lg) {
      if (lg) body(i, kd, al);
      else body(i, kd, a);
    };
    auto gdone = [&](int grp) { store_group(al, smask, wb.group_part, grp); };
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
    walk_tiles<float, float, WALK == kWalkGrouped, walk_unroll(WALK)>(lay, v32, gB, my32, wb,
                                                                       epi, gdone, pre);
  }
  if (cta_reduce_and_ticket(a, smask, mmask, 0u, part, &ctl->cnt_row)) {
    double r[13];
    grid_finish<7, 6, true, ND>(part, r, smask, mmask, wb.group_part, lay.n_long_tiles);
    if (threadIdx.x == 0) row_finalize(ctl, ic, r, t, k, n_ep, sigma, move);
  }
}

// MODE 0: ordinary iterations (no pending restart, not a restart point); MODE 1: the rest.
template <int RHO2, int MODE, int WALK>
__global__ void __maxnreg__(mx_max_regs(MODE, WALK))
k_col_iter_mx(SideLayout lay, SideVals<double> v64, SideVals<float> v32, WalkScratch wa,
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
  // staging: FP64 walks use (32 L + 4) doubles per warp, FP32 walks (32 L + 4) floats (the
  // FP32-only kernels are launched with half the shared memory)
  double *my64 = smem + (threadIdx.x >> 5) * lay.seg;
  float *my32 = reinterpret_cast<float *>(smem) + (threadIdx.x >> 5) * lay.seg;
  constexpr int ND = col_df_slots<MODE>();
  Acc<11, 8, ND> a;
  Acc<11, 0, ND> al;    // long-row sums (see walk_tiles); long-row maxima go to a
  a.zero();
  al.zero();
  Tel tl;         // active-set telemetry (ordinary check iterations)
  const unsigned smask = col_smask(check, rp, move);
  const unsigned mmask = col_mmask(rp, move);

  // checks and certificates at (x~_t, y~_t) given x~_t - x0 (xo), K^T y~_t (kty) and
  // K^T (y~_t - y_t) (ktd), all FP64
  auto checks = [&](int j, double x0j, double xo, double kty, double ktd, auto &A) {
    const double cj = v.c[j], lj = v.l[j], uj = v.u[j];
    if (check) {
      const double g = cj - kty;
      const double lam = proj_lambda(g, lj, uj);
      const double rd = (g - lam) * v.einv[j];
      A.s[2] += rd * rd;
      const double xt = x0j + xo;
      A.s[3] += cj * xt;
      if (lam > 0.0) A.s[4] += lj * lam;
      else if (lam < 0.0) A.s[4] += uj * lam;
      v.xout[j] = xt;
    }
    // x-part of T(z) - z at the restart point, and K^T of its y-part
    if (rp) col_cert_parts(j, xo, ktd, v, cj, lj, uj, A, a, 5, 0, v.certx);
  };
  auto gdone = [&](int grp) { store_group(al, smask, (restart ? wa : wb).group_part, grp); };

  if constexpr (MODE == 1) {
   if (restart) {
    // z^{n+1,0} = T(z^{n,k}): K^T y0' exactly (FP64 matrix, gathered y0 + dyt), x0' = x0 + dxt,
    // and the next PDHG point x~_{t+1} - x0' in FP64 (kept in dxt64 for the restart point's
    // certificate test)
    auto body = [&](int j, double kty, auto &A) {
      const double x0j = v.x0[j];
      const float dxtj = v.dxt[j];
      const double ktd = kty - v.kty0[j];
      checks(j, x0j, (double)dxtj, kty, ktd, A);
      const double x0n = x0j + (double)dxtj;
      // column parts of the anchor movement z^{n+1,0} - z^{n,0}, against the old anchor
      if (move)
        col_cert_parts(j, x0n - x0j, ktd, v, v.c[j], v.l[j], v.u[j], A, a, 8, 4, v.certx2);
      v.x0[j] = x0n;
      v.kty0[j] = kty;
      const double cj = v.c[j], lj = v.l[j], uj = v.u[j];
      v.s0[j] = (float)(-tau * (cj - kty));
      v.xlo[j] = __double2float_ru(lj - x0n);
      v.xhi[j] = __double2float_rd(uj - x0n);
      if (RHO2) { v.dx[j] = 0.f; v.ktdy[j] = 0.f; }
      const double nt = fmin(fmax(x0n - tau * (cj - kty), lj), uj) - x0n;
      v.dxt64[j] = nt;
      v.dxt[j] = (float)nt;
      A.s[0] += nt * nt;
      A.s[1] += nt * nt;
    };
    auto epi = [&](int j, double kty, bool lg) {
      if (lg) body(j, kty, al);
      else body(j, kty, a);
    };
    auto gA = [&](int i) { return y0[i] + (double)dyt[i]; };
    walk_tiles<double, double>(lay, v64, gA, my64, wa, epi, gdone);
   } else {
    // first iteration of an epoch: K^T (y~ - y0) in FP64 from the exact dyt64 of the row kernel
    auto body = [&](int j, double ktd, auto &A) {
      const double xo = v.dxt64[j];
      const double x0j = check ? v.x0[j] : 0.0;
      const double kty = check ? v.kty0[j] + ktd : 0.0;
      checks(j, x0j, xo, kty, ktd, A);
      const float dxtj = (float)xo, ktdyt = (float)ktd;
      float dxn, ktn;
      if (RHO2) {
        dxn = wf * (2.f * dxtj - v.dx[j]);
        ktn = wf * (2.f * ktdyt - v.ktdy[j]);
        v.dx[j] = dxn;
        v.ktdy[j] = ktn;
      } else {
        dxn = wf * dxtj;
        ktn = wf * ktdyt;
      }
      const float nt = fminf(fmaxf(dxn + v.s0[j] + tauf * ktn, v.xlo[j]), v.xhi[j]);
      v.dxt[j] = nt;
      const float ddx = dxn - nt;
      A.s[0] += (double)ddx * (double)ddx;
      A.s[1] += (double)nt * (double)nt;
    };
    auto epi = [&](int j, double ktd, bool lg) {
      if (lg) body(j, ktd, al);
      else body(j, ktd, a);
    };
    auto gA = [&](int i) { return dyt64[i]; };
    walk_tiles<double, double>(lay, v64, gA, my64, wb, epi, gdone);
   }
  } else {
    auto body = [&](int j, float ktdyt, auto &A) {
      const float dxtj = v.dxt[j];
      if (check) {
        tel_column(j, dxtj == v.xlo[j] || dxtj == v.xhi[j], v.act, tl);
        const double x0j = v.x0[j];
        checks(j, x0j, (double)dxtj, v.kty0[j] + (double)ktdyt, (double)ktdyt, A);
      }
      float dxn, ktn;
      if (RHO2) {
        dxn = wf * (2.f * dxtj - v.dx[j]);
        ktn = wf * (2.f * ktdyt - v.ktdy[j]);
        v.dx[j] = dxn;
        v.ktdy[j] = ktn;
      } else {
        dxn = wf * dxtj;
        ktn = wf * ktdyt;
      }
      const float nt = fminf(fmaxf(dxn + v.s0[j] + tauf * ktn, v.xlo[j]), v.xhi[j]);
      v.dxt[j] = nt;
      const float ddx = dxn - nt;
      df_acc(A.d[0], ddx, ddx);
      df_acc(A.d[1], nt, nt);
    };
    auto epi = [&](int j, float ktdyt, bool lg) {
      if (lg) body(j, ktdyt, al);
      else body(j, ktdyt, a);
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
      prefetch_l1(v.xhi + j);
    };
    walk_tiles<float, float, WALK == kWalkGrouped, walk_unroll(WALK)>(lay, v32, gB, my32, wb,
                                                                       epi, gdone, pre);
    if (check) tel_flush(ctl, tl);
  }
  if (cta_reduce_and_ticket(a, smask, mmask, 0u, part, &ctl->cnt_col)) {
    double r[19];
    grid_finish<11, 8, true, ND>(part, r, smask, mmask, (restart ? wa : wb).group_part,
                                 lay.n_long_tiles);
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
// walk (SideLayout::walk).
void launch_row_iter_mx(cudaStream_t st, const SideStore &side, const RowVecsMx &v,
                        const float *dxt, const double *dxt64, const double *x0, Ctl *ctl,
                        double *part, const IterConsts &ic, int grid, int smem) {
  const int threads = side.lay.cta_warps * kWarp;
  auto go = [&](auto kern, int sm) {
    kern<<<grid, threads, sm, st>>>(side.lay, side.v64, side.v32, side.wa, side.wb, v, dxt,
                                    dxt64, x0, ctl, part, ic);
  };
  const int w = side.lay.walk;
  if (ic.rho2) {
    go(k_row_iter_mx<1, 1, kWalkGrouped>, smem);
    if (w == kWalkGrouped) go(k_row_iter_mx<1, 0, kWalkGrouped>, smem / 2);
    else if (w == kWalkWide) go(k_row_iter_mx<1, 0, kWalkWide>, smem / 2);
    else go(k_row_iter_mx<1, 0, kWalkPlain>, smem / 2);
  } else {
    go(k_row_iter_mx<0, 1, kWalkGrouped>, smem);
    if (w == kWalkGrouped) go(k_row_iter_mx<0, 0, kWalkGrouped>, smem / 2);
    else if (w == kWalkWide) go(k_row_iter_mx<0, 0, kWalkWide>, smem / 2);
    else go(k_row_iter_mx<0, 0, kWalkPlain>, smem / 2);
  }
}

void launch_col_iter_mx(cudaStream_t st, const SideStore &side, const ColVecsMx &v,
                        const float *dyt, const double *dyt64, const double *y0, Ctl *ctl,
                        double *part, const IterConsts &ic, int grid, int smem, int phase) {
  const int threads = side.lay.cta_warps * kWarp;
  auto go = [&](auto kern, int sm) {
    kern<<<grid, threads, sm, st>>>(side.lay, side.v64, side.v32, side.wa, side.wb, v, dyt,
                                    dyt64, y0, ctl, part, ic, phase);
  };
  const bool grp = side.lay.walk == kWalkGrouped;
  if (ic.rho2) {
    go(k_col_iter_mx<1, 1, kWalkGrouped>, smem);
    grp ? go(k_col_iter_mx<1, 0, kWalkGrouped>, smem / 2) : go(k_col_iter_mx<1, 0, kWalkPlain>, smem / 2);
  } else {
    go(k_col_iter_mx<0, 1, kWalkGrouped>, smem);
    grp ? go(k_col_iter_mx<0, 0, kWalkGrouped>, smem / 2) : go(k_col_iter_mx<0, 0, kWalkPlain>, smem / 2);
  }
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
  const void *k[] = {
      (const void *)k_row_iter_mx<0, 0, kWalkPlain>,   (const void *)k_row_iter_mx<1, 0, kWalkPlain>,
      (const void *)k_row_iter_mx<0, 0, kWalkWide>,    (const void *)k_row_iter_mx<1, 0, kWalkWide>,
      (const void *)k_row_iter_mx<0, 0, kWalkGrouped>, (const void *)k_row_iter_mx<1, 0, kWalkGrouped>,
      (const void *)k_row_iter_mx<0, 1, kWalkGrouped>, (const void *)k_row_iter_mx<1, 1, kWalkGrouped>,
      (const void *)k_col_iter_mx<0, 0, kWalkPlain>,   (const void *)k_col_iter_mx<1, 0, kWalkPlain>,
      (const void *)k_col_iter_mx<0, 0, kWalkGrouped>, (const void *)k_col_iter_mx<1, 0, kWalkGrouped>,
      (const void *)k_col_iter_mx<0, 1, kWalkGrouped>, (const void *)k_col_iter_mx<1, 1, kWalkGrouped>};
  for (const void *f : k) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int iter_mx_blocks_per_sm(int smem, bool row, int walk, int threads) {
  // the ordinary kernels of one side in one walk instantiation (both reflection settings)
  const void *k[2];
  if (row) {
    k[0] = walk == kWalkGrouped ? (const void *)k_row_iter_mx<0, 0, kWalkGrouped>
           : walk == kWalkWide  ? (const void *)k_row_iter_mx<0, 0, kWalkWide>
                                : (const void *)k_row_iter_mx<0, 0, kWalkPlain>;
    k[1] = walk == kWalkGrouped ? (const void *)k_row_iter_mx<1, 0, kWalkGrouped>
           : walk == kWalkWide  ? (const void *)k_row_iter_mx<1, 0, kWalkWide>
                                : (const void *)k_row_iter_mx<1, 0, kWalkPlain>;
  } else {
    k[0] = walk == kWalkGrouped ? (const void *)k_col_iter_mx<0, 0, kWalkGrouped>
                                : (const void *)k_col_iter_mx<0, 0, kWalkPlain>;
    k[1] = walk == kWalkGrouped ? (const void *)k_col_iter_mx<1, 0, kWalkGrouped>
                                : (const void *)k_col_iter_mx<1, 0, kWalkPlain>;
  }
  int mn = 1 << 30;
  for (const void *f : k) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, threads, smem / 2);
    mn = b < mn ? b : mn;
  }
  return mn;
}

}  // namespace rh
