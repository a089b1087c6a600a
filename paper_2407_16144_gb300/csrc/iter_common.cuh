// Device logic shared by the FP64 and mixed-precision iteration kernels: the reduced-cost
// projection, and the last-CTA finalisations (restart rule and primal weight in the row kernel;
// termination and certificate tests in the column kernel).
#pragma once

#include "common.cuh"

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
  ctl->stage = 0;
}

}  // namespace rh
