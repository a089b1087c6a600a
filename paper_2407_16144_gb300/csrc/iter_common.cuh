// Device logic shared by the FP64 and mixed-precision iteration kernels: the reduced-cost
// projection, and the last-CTA finalisations (restart rule and primal weight in the row kernel;
// termination and certificate tests in the column kernel).
#pragma once

#include "common.cuh"
#include "internal.h"

namespace rh {

// reduced cost lambda = proj onto {0} (free), [0,inf) (l finite), (-inf,0] (u finite), R
__device__ __forceinline__ double proj_lambda(double g, double l, double u) {
  const bool lf = isfinite(l), uf = isfinite(u);
  if (lf && uf) return g;
  if (lf) return fmax(g, 0.0);
  if (uf) return fmin(g, 0.0);
  return 0.0;
}

// Row-kernel slots: sums 0 dy2, 1 cross, 2 ya2, 3 rp2, 4 qy, 5 qv ; maxima 6 yneg, 7 kd_eq,
// 8 kd_in.  Completes ||z_t - T(z_t)||_P^2 = ||dx||^2/tau + ||dy||^2/sigma + 2 dy^T K dx, applies
// the restart rule of eq. adaptive-restart (first epoch: k > tau^0; later: FPR <= beta FPR_0;
// plus the epoch cap, or the fixed frequency of eq. fixed-restart) and the primal-weight update.
__device__ __forceinline__ void row_finalize(Ctl *ctl, const IterConsts &ic, const double *r,
                                             long long t, long long k, long long n_ep,
                                             double sigma) {
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
  ctl->stage = 1;
}

// Column-kernel slots: sums 0 dx2, 1 xa2, 2 rd2, 3 cx, 4 bnd, 5 cd, 6 uterm, 7 lterm ;
// maxima 8 dlb, 9 dub, 10 ainf_u, 11 ainf_l.  Certificate tests at restart points (the
// displacement T(z^{n,0}) - z^{n,0}, Theorem infeas; normalised so the ray objective is 1),
// then the rel-KKT termination test on check iterations, then the iteration counters.
__device__ __forceinline__ void col_finalize(Ctl *ctl, const IterConsts &ic, const double *r,
                                             long long t, bool check, bool rp, int phase) {
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
    // With FP32 offsets a diverging iterate carries about 1e-5 relative rounding, so a
    // certificate cannot reach eps_infeas; once the candidate comes within 1e-3 of certifying,
    // the solve continues in FP64 from this restart point.
    else if (ic.mixed && ((obj > 0.0 && vy / obj <= 1e-3) || (cd < 0.0 && vx / (-cd) <= 1e-3)))
      st = kEscalate;
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
  ctl->t = (phase == 0) ? t + 1 : t;
  if (st == kRunning) {     // a final iteration keeps its own (k, n)
    ctl->k = ctl->k_next;
    ctl->n = ctl->n_next;
  }
  ctl->cnt_col = 0;
  ctl->stage = 0;
}

// ---------------------------------------------------------------------------------------------
// The FP64 per-row epilogues of one PDHG evaluation, shared by the tiled single-LP kernels and
// the CTA-resident batched kernel.

struct StepFlags {
  int restart;      // the pending transition is a restart: z_t = T(z_{t-1})
  double w;         // Halpern weight (k+1)/(k+2) of the pending blend
  double step;      // sigma (row epilogue) or tau (column epilogue)
  bool check;       // termination-check iteration
  bool rp;          // restart point (k == 0, n >= 1): certificate test
  int m_eq;
};

// Row i of K^ x~_t = dot: forms y_t and K x_t by the pending blend (eq. hpdhg / eq. hrpdhg, or
// the restart point), takes the dual step of eq. pdhg, and accumulates the fixed-point-residual
// parts (0 ||dy||^2, 1 dy^T (K x - K x~), 2 ||y~ - y0||^2), the check parts (3 primal residual^2,
// 4 q^T y~) and the certificate parts (5 q^T (y~ - y), maxima 0..2).
template <int RHO2>
__device__ __forceinline__ void row_epilogue(int i, double dot, const RowVecs &v,
                                             const StepFlags &f, Acc<6, 3> &a) {
  const double ytp = v.yt[i], kxtp = v.kxt[i];
  const double w = f.w, sigma = f.step;
  double yi, kxi, y0i;
  if (f.restart) {
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
  if (i >= f.m_eq) yn = fmax(yn, 0.0);
  v.yt[i] = yn;
  v.kxt[i] = dot;
  const double dy = yi - yn;
  a.s[0] += dy * dy;
  a.s[1] += dy * (kxi - dot);
  const double ya = yn - y0i;
  a.s[2] += ya * ya;
  if (f.check) {
    double r = (qi - dot) * v.dinv[i];
    if (i >= f.m_eq) r = fmax(r, 0.0);
    a.s[3] += r * r;
    a.s[4] += qi * yn;
  }
  if (f.rp) {
    const double vy = yn - yi;            // y-part of T(z) - z at the restart point
    a.s[5] += qi * vy;
    const double di = v.d[i];
    if (i >= f.m_eq) a.mx[0] = fmax(a.mx[0], fmax(-vy * di, 0.0));
    const double kd = (dot - kxi) * v.dinv[i];   // K d (unscaled), d = x~ - x
    if (i < f.m_eq) a.mx[1] = fmax(a.mx[1], fabs(kd));
    else a.mx[2] = fmax(a.mx[2], fmax(-kd, 0.0));
    v.certy[i] = vy * di;
  }
}

// Column j of K^T y~_t = dot: the check parts at (x~_t, y~_t) (2 dual residual^2, 3 c^T x~,
// 4 bound terms of the dual objective), the certificate parts at restart points (5 c^T d,
// 6/7 bound terms of the ray objective, maxima 0..3), then the blend to x_{t+1} and the primal
// step x~_{t+1} = proj_X(x_{t+1} - tau (c - K^T y_{t+1})) with parts 0 ||x - x~||^2,
// 1 ||x~ - x0||^2.
template <int RHO2>
__device__ __forceinline__ void col_epilogue(int j, double dot, const ColVecs &v,
                                             const StepFlags &f, Acc<8, 4> &a) {
  const double xtj = v.xt[j];
  const double cj = v.c[j], lj = v.l[j], uj = v.u[j];
  const double w = f.w, tau = f.step;
  if (f.check) {
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
  if (f.rp) {
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
  if (f.restart) {
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
}

}  // namespace rh
