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

namespace rh {

namespace {

__device__ __forceinline__ double proj_lambda(double g, double l, double u) {
  // reduced cost lambda = proj onto {0} (free), [0,inf) (l finite), (-inf,0] (u finite), R
  const bool lf = isfinite(l), uf = isfinite(u);
  if (lf && uf) return g;
  if (lf) return fmax(g, 0.0);
  if (uf) return fmin(g, 0.0);
  return 0.0;
}

// sums: 0 dy2, 1 cross, 2 ya2, 3 rp2, 4 qy, 5 qv ; maxima: 0 yneg, 1 kd_eq, 2 kd_in
using RowAcc = Acc<6, 3>;
// sums: 0 dx2, 1 xa2, 2 rd2, 3 cx, 4 bnd, 5 cd, 6 uterm, 7 lterm ;
// maxima: 0 dlb, 1 dub, 2 ainf_u, 3 ainf_l
using ColAcc = Acc<8, 4>;

template <int RHO2>
__global__ void __launch_bounds__(kBlockThreads)
k_row_iter(SideLayout<double> lay, const double *__restrict__ xt, RowVecs v, Ctl *ctl,
           double *part, IterConsts ic) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning) return;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const int restart = ctl->restart_pending;
  const double w = ctl->w, sigma = ctl->sigma;
  const bool check = ((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters);
  const bool rp = (k == 0 && n_ep >= 1);
  const int m_eq = ic.m_eq;
  RowAcc a;
  a.zero();
  double *my = smem + (threadIdx.x >> 5) * (kTileRows * lay.L);

  auto epi = [&](int i, double dot) {
    const double ytp = v.yt[i], kxtp = v.kxt[i];
    double yi, kxi, y0i;
    if (restart) {
      yi = ytp; kxi = kxtp; y0i = yi;
      v.y0[i] = yi; v.kx0[i] = kxi;
      if (RHO2) { v.y[i] = yi; v.kx[i] = kxi; }
    } else {
      y0i = v.y0[i];
      const double kx0i = v.kx0[i];
      if (RHO2) {
        yi = w * (2.0 * ytp - v.y[i]) + (1.0 - w) * y0i;
        kxi = w * (2.0 * kxtp - v.kx[i]) + (1.0 - w) * kx0i;
        v.y[i] = yi; v.kx[i] = kxi;
      } else {
        yi = w * ytp + (1.0 - w) * y0i;
        kxi = w * kxtp + (1.0 - w) * kx0i;
      }
    }
    const double qi = v.q[i];
    double yn = yi + sigma * (qi - 2.0 * dot + kxi);
    if (i >= m_eq) yn = fmax(yn, 0.0);
    v.yt[i] = yn;
    v.kxt[i] = dot;
    const double dy = yi - yn;
    a.s[0] += dy * dy;
    a.s[1] += dy * (kxi - dot);
    const double ya = yn - y0i;
    a.s[2] += ya * ya;
    if (check) {
      double r = (qi - dot) * v.dinv[i];
      if (i >= m_eq) r = fmax(r, 0.0);
      a.s[3] += r * r;
      a.s[4] += qi * yn;
    }
    if (rp) {
      const double vy = yn - yi;            // y-part of T(z) - z at the restart point
      a.s[5] += qi * vy;
      const double di = v.d[i];
      if (i >= m_eq) a.mx[0] = fmax(a.mx[0], fmax(-vy * di, 0.0));
      const double kd = (dot - kxi) * v.dinv[i];   // K d (unscaled), d = x~ - x
      if (i < m_eq) a.mx[1] = fmax(a.mx[1], fabs(kd));
      else a.mx[2] = fmax(a.mx[2], fmax(-kd, 0.0));
      v.certy[i] = vy * di;
    }
  };
  walk_tiles(lay, xt, my, epi);

  if (cta_reduce_and_ticket(a, part, &ctl->cnt_row)) {
    double r[9];
    grid_finish<6, 3>(part, r);
    if (threadIdx.x == 0) {
      const double tau = ctl->tau, omega = ctl->omega;
      const double fpr2 = ctl->dx_sq / tau + r[0] / sigma + 2.0 * r[1];
      const double fpr0 = (k == 0) ? fpr2 : ctl->fpr0_sq;
      bool rs;
      if (ic.restart_scheme == 1) {
        rs = ic.max_epoch_len > 0 && k >= ic.max_epoch_len;
      } else {
        rs = (n_ep == 0 && k > ic.first_epoch_len) || (n_ep >= 1 && fpr2 <= ic.beta2 * fpr0) ||
             (ic.max_epoch_len > 0 && k >= ic.max_epoch_len);
      }
      if (ic.trace && t < ic.trace_cap) {
        TraceRec tr;
        tr.t = t; tr.epoch = n_ep; tr.k = k; tr.fpr_sq = fpr2; tr.omega = omega;
        tr.restart = rs ? 1 : 0; tr.pad = 0;
        ic.trace[t] = tr;
      }
      ctl->fpr0_sq = fpr0;
      ctl->fpr_sq = fpr2;
      ctl->rp_sq = r[3];
      ctl->qy = r[4];
      ctl->inf_qv = r[5];
      ctl->inf_yneg = r[6];
      ctl->inf_kd_eq = r[7];
      ctl->inf_kd_in = r[8];
      if (!isfinite(fpr2)) ctl->status = kNumericalError;
      if (rs) {
        if (ic.pw_update) {
          const double dxa = sqrt(ctl->xa_sq), dya = sqrt(r[2]);
          const double ratio = dxa > 1e-10 ? dya / dxa : 0.0;
          if (dxa > 1e-10 && dya > 1e-10 && ratio > 0.0 && isfinite(ratio)) {
            const double om = exp(0.5 * log(ratio) + 0.5 * log(omega));
            ctl->omega = om;
            ctl->tau = ic.eta / om;
            ctl->sigma = ic.eta * om;
          }
        }
        ctl->k_next = 0;
        ctl->n_next = n_ep + 1;
      } else {
        ctl->w = (k + 1.0) / (k + 2.0);
        ctl->k_next = k + 1;
        ctl->n_next = n_ep;
      }
      ctl->restart_pending = rs ? 1 : 0;
      ctl->cnt_row = 0;
    }
  }
}

template <int RHO2>
__global__ void __launch_bounds__(kBlockThreads)
k_col_iter(SideLayout<double> lay, const double *__restrict__ ytv, ColVecs v, Ctl *ctl,
           double *part, IterConsts ic, int phase) {
  extern __shared__ double smem[];
  if (ctl->status != kRunning) return;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const int restart = ctl->restart_pending;
  const double w = ctl->w, tau = ctl->tau;
  const bool check = phase == 0 && (((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters));
  const bool rp = phase == 0 && (k == 0 && n_ep >= 1);
  ColAcc a;
  a.zero();
  double *my = smem + (threadIdx.x >> 5) * (kTileRows * lay.L);

  auto epi = [&](int j, double dot) {
    const double xtj = v.xt[j];
    const double cj = v.c[j], lj = v.l[j], uj = v.u[j];
    if (check) {
      const double g = cj - dot;
      const double lam = proj_lambda(g, lj, uj);
      const double rd = (g - lam) * v.einv[j];
      a.s[2] += rd * rd;
      a.s[3] += cj * xtj;
      if (lam > 0.0) a.s[4] += lj * lam;
      else if (lam < 0.0) a.s[4] += uj * lam;
      v.xout[j] = xtj;
    }
    double x0j = v.x0[j], kty0j = v.kty0[j];
    if (rp) {
      // restart point: x_t = x^{n,0} and K^T y_t = K^T y^{n,0}
      const double dsc = xtj - x0j;               // x-part of T(z) - z (scaled)
      a.s[5] += cj * dsc;
      const double du = dsc * v.e[j];
      const bool lf = isfinite(lj), uf = isfinite(uj);
      if (lf) a.mx[0] = fmax(a.mx[0], fmax(-du, 0.0));
      if (uf) a.mx[1] = fmax(a.mx[1], fmax(du, 0.0));
      const double kv = dot - kty0j;              // K^T (y~ - y) (scaled)
      if (uf) a.s[6] += fmax(kv, 0.0) * uj;
      else a.mx[2] = fmax(a.mx[2], fmax(kv * v.einv[j], 0.0));
      if (lf) a.s[7] += fmax(-kv, 0.0) * lj;
      else a.mx[3] = fmax(a.mx[3], fmax(-kv * v.einv[j], 0.0));
      v.certx[j] = du;
    }
    double xn, kn;
    if (restart) {
      xn = xtj; kn = dot;
      v.x0[j] = xn; v.kty0[j] = kn;
      x0j = xn; kty0j = kn;
      if (RHO2) { v.x[j] = xn; v.kty[j] = kn; }
    } else if (RHO2) {
      xn = w * (2.0 * xtj - v.x[j]) + (1.0 - w) * x0j;
      kn = w * (2.0 * dot - v.kty[j]) + (1.0 - w) * kty0j;
      v.x[j] = xn; v.kty[j] = kn;
    } else {
      xn = w * xtj + (1.0 - w) * x0j;
      kn = w * dot + (1.0 - w) * kty0j;
    }
    const double xtn = fmin(fmax(xn - tau * (cj - kn), lj), uj);
    v.xt[j] = xtn;
    const double dx = xn - xtn;
    a.s[0] += dx * dx;
    const double xa = xtn - x0j;
    a.s[1] += xa * xa;
  };
  walk_tiles(lay, ytv, my, epi);

  if (cta_reduce_and_ticket(a, part, &ctl->cnt_col)) {
    double r[12];
    grid_finish<8, 4>(part, r);
    if (threadIdx.x == 0) {
      ctl->dx_sq = r[0];
      ctl->xa_sq = r[1];
      int st = kRunning;
      if (rp) {
        const double obj = ctl->inf_qv - r[6] + r[7];
        const double vy = fmax(fmax(r[10], r[11]), ctl->inf_yneg);
        const double cd = r[5];
        const double vx = fmax(fmax(ctl->inf_kd_eq, ctl->inf_kd_in), fmax(r[8], r[9]));
        if (obj > 0.0 && vy / obj <= ic.eps_infeas) st = kPrimalInfeasible;
        else if (cd < 0.0 && vx / (-cd) <= ic.eps_infeas) st = kDualInfeasible;
      }
      if (st == kRunning && check) {
        const double rel_p = sqrt(ctl->rp_sq) / ic.qn1;
        const double rel_d = sqrt(r[2]) / ic.cn1;
        const double pobj = r[3] + ic.obj_offset;
        const double dobj = ctl->qy + r[4] + ic.obj_offset;
        const double gap = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
        ctl->rel_p = rel_p;
        ctl->rel_d = rel_d;
        ctl->rel_gap = gap;
        ctl->pobj = pobj;
        ctl->dobj = dobj;
        ctl->check_t = t;
        const double kkt = fmax(rel_p, fmax(rel_d, gap));
        if (!isfinite(kkt)) st = kNumericalError;
        else if (kkt <= ic.eps_kkt) st = kOptimal;
        else if (t + 1 >= ic.max_iters) st = kIterLimit;
      }
      if (st == kRunning && !isfinite(r[0])) st = kNumericalError;
      if (st != kRunning) ctl->status = st;
      ctl->t = (phase == 0) ? t + 1 : 0;
      if (st == kRunning) {     // a final iteration keeps its own (k, n)
        ctl->k = ctl->k_next;
        ctl->n = ctl->n_next;
      }
      ctl->cnt_col = 0;
    }
  }
}

__global__ void k_unscale(int n, int m, const double *e, const double *xs, const double *d,
                          const double *ys, double *xo, double *yo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xo[i] = e[i] * xs[i];
  if (i < m) yo[i] = d[i] * ys[i];
}

}  // namespace

void launch_row_iter(cudaStream_t st, const SideLayout<double> &lay, const double *xt,
                     const RowVecs &v, Ctl *ctl, double *part, const IterConsts &ic, int grid,
                     int smem) {
  if (ic.rho2)
    k_row_iter<1><<<grid, kBlockThreads, smem, st>>>(lay, xt, v, ctl, part, ic);
  else
    k_row_iter<0><<<grid, kBlockThreads, smem, st>>>(lay, xt, v, ctl, part, ic);
}

void launch_col_iter(cudaStream_t st, const SideLayout<double> &lay, const double *yt,
                     const ColVecs &v, Ctl *ctl, double *part, const IterConsts &ic, int grid,
                     int smem, int phase) {
  if (ic.rho2)
    k_col_iter<1><<<grid, kBlockThreads, smem, st>>>(lay, yt, v, ctl, part, ic, phase);
  else
    k_col_iter<0><<<grid, kBlockThreads, smem, st>>>(lay, yt, v, ctl, part, ic, phase);
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
