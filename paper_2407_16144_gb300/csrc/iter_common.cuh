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

// Reduction slots.  Row kernel: sums 0 ||dy||^2, 1 dy^T (K dx), 2 ||y~ - y0||^2, 3 primal
// residual^2, 4 q^T y~, 5 q^T (y-part of T(z) - z), 6 q^T (y-part of z^{n+1,0} - z^{n,0});
// maxima 7..9 the T(z) - z row tests (y_G sign, |K d| on A rows, (K d)^- on G rows) and
// 10..12 the same for the anchor movement.
using RowAcc = Acc<7, 6>;
using RowAccL = Acc<7, 0>;     // long-row sums (see store_group)
// Column kernel: sums 0 ||dx||^2, 1 ||x~ - x0||^2, 2 dual residual^2, 3 c^T x~, 4 bound terms of
// the dual objective, 5 c^T d, 6/7 bound terms of the ray objective for T(z) - z, 8..10 the same
// for the anchor movement; maxima 11..14 the T(z) - z column tests (d bound signs, (K^T y)^+ on
// infinite u, (K^T y)^- on infinite l) and 15..18 the same for the anchor movement.
using ColAcc = Acc<11, 8>;
using ColAccL = Acc<11, 0>;

__device__ __forceinline__ unsigned row_smask(bool check, bool cert, bool move) {
  return 0x7u | (check ? 0x18u : 0u) | (cert ? 0x20u : 0u) | (move ? 0x40u : 0u);
}
__device__ __forceinline__ unsigned row_mmask(bool cert, bool move) {
  return (cert ? 0x7u : 0u) | (move ? 0x38u : 0u);
}
__device__ __forceinline__ unsigned col_smask(bool check, bool cert, bool move) {
  return 0x3u | (check ? 0x1Cu : 0u) | (cert ? 0xE0u : 0u) | (move ? 0x700u : 0u);
}
__device__ __forceinline__ unsigned col_mmask(bool cert, bool move) {
  return (cert ? 0xFu : 0u) | (move ? 0xF0u : 0u);
}

// Farkas tests of one candidate from its reduced parts (Proposition full-infeas, normalised so
// that the ray objective is 1): the y-part first, then the x-part.
__device__ __forceinline__ int farkas_status(double qv, double uterm, double lterm, double vy_max,
                                             double cd, double vx_max, double eps) {
  const double obj = qv - uterm + lterm;
  if (obj > 0.0 && vy_max / obj <= eps) return kPrimalInfeasible;
  if (cd < 0.0 && vx_max / (-cd) <= eps) return kDualInfeasible;
  return kRunning;
}

// Completes ||z_t - T(z_t)||_P^2 = ||dx||^2/tau + ||dy||^2/sigma + 2 dy^T K dx, applies the
// restart rule (scheme 0: eq. adaptive-restart, first epoch k > tau^0, later FPR <= beta FPR_0,
// plus the epoch cap; scheme 1: the fixed frequency of eq. fixed-restart; scheme 2: the two-phase
// schedule of the remark after Theorem infeas, a first epoch of first_epoch_len iterations and
// then the fixed frequency max_epoch_len) and the primal-weight update.
// With move set (the restart applied by this kernel was decided by a phase-0 column kernel that
// staged its parts) it first completes the anchor-movement candidate's test.
// An ordinary column stage (phase 0, no termination check, no certificate test, no restart
// transition, no adaptive step) needs from its grid reduction only ||x_t - x~_t||^2 and
// ||x~_t - x^{n,0}||^2, and from its finaliser only their storage and the advance of (t, k, n).
// It therefore writes its CTA partials and ends without a ticket (the control block keeps
// stage = 1, and every CTA sets col_deferred); the next row kernel adds those partials in its last
// CTA and row_finalize applies the column update first (dcol).  (stage = 1 alone does not mark a
// deferral: in mixed precision the restart-mode row kernel, launched before the ordinary one,
// also leaves stage = 1 when it runs.)  Its serial tail (ticket, grid reduction, finaliser) leaves the
// critical path of every ordinary iteration.
__device__ __forceinline__ bool col_defers(const IterConsts &ic, int phase, bool check, bool cert,
                                           bool move) {
  return phase == 0 && !check && !cert && !move && !ic.adaptive;
}

// rc: the deferred column stage's sums (dcol; see col_defers), (t, k, n_ep) the iteration after
// it.
__device__ __forceinline__ void row_finalize(Ctl *ctl, const IterConsts &ic, const double *r,
                                             long long t, long long k, long long n_ep,
                                             double sigma, bool move, bool dcol = false,
                                             const double *rc = nullptr) {
  if (dcol) {
    // the finaliser the column stage left: its sums and the advance of (t, k, n)
    ctl->col_deferred = 0;
    ctl->dx_sq = rc[0];
    ctl->xa_sq = rc[1];
    ctl->t = t;
    ctl->k = k;
    ctl->n = n_ep;
    if (!isfinite(rc[0])) {
      ctl->status = kNumericalError;
      ctl->cnt_row = 0;
      return;
    }
  }
  if (move) {
    ctl->mv_ready = 0;
    const int st = farkas_status(r[6], ctl->mv_u, ctl->mv_l,
                                 fmax(fmax(ctl->mv_au, ctl->mv_al), r[10]), ctl->mv_cd,
                                 fmax(fmax(r[11], r[12]), fmax(ctl->mv_dlb, ctl->mv_dub)),
                                 ic.eps_infeas);
    if (st != kRunning) {
      ctl->status = st;
      ctl->cert_src = kCertAnchorMove;
      ctl->cnt_row = 0;
      return;
    }
  }
  const double omega = ctl->omega;
  if (ic.adaptive) {
    // the step eta is admissible while eta <= eta_bar = ||dz||_w^2 / (2 |dy^T K dx|),
    // ||dz||_w^2 = omega ||dx||^2 + ||dy||^2 / omega; the next step is
    // min((1 - j^-0.3) eta_bar, (1 + j^-0.6) eta), j = t + 2; an inadmissible step is redone
    const double eta = ctl->eta;
    const double cross = fabs(r[1]);
    const double num = omega * ctl->dx_sq + r[0] / omega;
    const double eta_bar = cross > 0.0 ? num / (2.0 * cross) : INFINITY;
    const double j = (double)t + 2.0;
    const double nxt = fmin((1.0 - pow(j, -0.3)) * eta_bar, (1.0 + pow(j, -0.6)) * eta);
    if (eta > eta_bar) {
      ctl->retries += 1;
      if (ctl->retries > 64 || !(nxt > 0.0) || !isfinite(nxt)) ctl->status = kNumericalError;
      ctl->eta = nxt;
      set_steps(ctl, nxt, omega);
      ctl->redo = 1;
      ctl->cnt_row = 0;
      ctl->stage = 1;
      return;
    }
    ctl->eta_next = nxt;
  }
  const double fpr2 = ctl->dx_sq * ctl->tau_inv + r[0] * ctl->sigma_inv + 2.0 * r[1];
  const double fpr0 = (k == 0) ? fpr2 : ctl->fpr0_sq;
  bool rs;
  if (ic.restart_scheme == 1) {
    rs = ic.max_epoch_len > 0 && k >= ic.max_epoch_len;
  } else if (ic.restart_scheme == 2) {
    rs = k >= (n_ep == 0 ? (long long)ic.first_epoch_len : ic.max_epoch_len);
  } else {
    rs = (n_ep == 0 && k > ic.first_epoch_len) || (n_ep >= 1 && fpr2 <= ic.beta2 * fpr0) ||
         (ic.max_epoch_len > 0 && k >= ic.max_epoch_len);
  }
  if (ic.trace && t < ic.trace_cap) {
    TraceRec tr;
    tr.t = t; tr.epoch = n_ep; tr.k = k; tr.fpr_sq = fpr2; tr.omega = omega;
    tr.restart = rs ? 1 : 0; tr.retries = ctl->retries;
    tr.active = -1; tr.changed = -1;
    ic.trace[t] = tr;
  }
  ctl->fpr0_sq = fpr0;
  ctl->fpr_sq = fpr2;
  ctl->rp_sq = r[3];
  ctl->qy = r[4];
  ctl->inf_qv = r[5];
  ctl->inf_yneg = r[7];
  ctl->inf_kd_eq = r[8];
  ctl->inf_kd_in = r[9];
  if (!isfinite(fpr2)) ctl->status = kNumericalError;
  // the accepted step's successor takes effect from the next PDHG evaluation
  const double eta_now = ic.adaptive ? ctl->eta_next : ic.eta;
  if (ic.adaptive) {
    ctl->eta = eta_now;
    set_steps(ctl, eta_now, omega);
    ctl->redo = 0;
    ctl->retries = 0;
  }
  if (rs) {
    if (ic.pw_update) {
      const double dxa = sqrt(ctl->xa_sq), dya = sqrt(r[2]);
      const double ratio = dxa > 1e-10 ? dya / dxa : 0.0;
      if (dxa > 1e-10 && dya > 1e-10 && ratio > 0.0 && isfinite(ratio)) {
        const double om = exp(0.5 * log(ratio) + 0.5 * log(omega));
        ctl->omega = om;
        set_steps(ctl, eta_now, om);
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

// Certificate test of the displacement T(z) - z (cert: at restart points, Theorem infeas, and
// at check iterations), then the rel-KKT termination test on check iterations, then the
// iteration counters.  With move set (this kernel applied a restart decision) the column parts
// of the anchor-movement candidate are staged for the next row kernel.
__device__ __forceinline__ void col_finalize(Ctl *ctl, const IterConsts &ic, const double *r,
                                             long long t, bool check, bool cert, bool rp,
                                             bool move, int phase, bool tel = true) {
  if (ctl->redo) {          // x~_t recomputed with the smaller step; the row stage follows
    ctl->dx_sq = r[0];
    ctl->xa_sq = r[1];
    ctl->cnt_col = 0;
    ctl->stage = 0;
    return;
  }
  ctl->dx_sq = r[0];
  ctl->xa_sq = r[1];
  int st = kRunning;
  if (cert) {
    const double vy = fmax(fmax(r[13], r[14]), ctl->inf_yneg);
    const double vx = fmax(fmax(ctl->inf_kd_eq, ctl->inf_kd_in), fmax(r[11], r[12]));
    st = farkas_status(ctl->inf_qv, r[6], r[7], vy, r[5], vx, ic.eps_infeas);
    if (st != kRunning) {
      ctl->cert_src = rp ? kCertRestartPoint : kCertCheck;
    } else if (ic.mixed && rp) {
      // With FP32 offsets a diverging iterate carries about 1e-5 relative rounding, so this
      // candidate cannot reach eps_infeas; once it comes within 1e-3 of certifying at two
      // restart points in a row, the solve continues in FP64 from this restart point.  (One
      // restart point alone can pass the loose test on a feasible LP, early in its solve.)
      const bool near = farkas_status(ctl->inf_qv, r[6], r[7], vy, r[5], vx, 1e-3) != kRunning;
      ctl->near_cert = near ? ctl->near_cert + 1 : 0;
      if (ctl->near_cert >= 2) st = kEscalate;
    }
  }
  if (move) {
    ctl->mv_cd = r[8];
    ctl->mv_u = r[9];
    ctl->mv_l = r[10];
    ctl->mv_dlb = r[15];
    ctl->mv_dub = r[16];
    ctl->mv_au = r[17];
    ctl->mv_al = r[18];
    ctl->mv_ready = 1;
  }
  if (check) {
    // active-set telemetry (the partition of Section 4 as the iterates see it)
    const unsigned long long ua = atomicExch(&ctl->tel_act, 0ull);
    const unsigned long long uc = atomicExch(&ctl->tel_chg, 0ull);
    const long long na = tel ? (long long)ua : -1;
    const long long nc = tel ? (long long)uc : -1;
    ctl->act_last = na;
    ctl->chg_last = nc;
    if (ic.trace && t < ic.trace_cap) {
      ic.trace[t].active = na;
      ic.trace[t].changed = nc;
    }
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
// the CTA-resident batched kernel.  Sums go to S (the lane's own accumulator, or the long-row
// accumulator whose order is fixed per group), maxima always to M.

struct StepFlags {
  int restart;      // the pending transition is a restart: z_t = T(z_{t-1})
  double w;         // Halpern weight (k+1)/(k+2) of the pending blend
  double step;      // sigma (row epilogue) or tau (column epilogue)
  bool check;       // termination-check iteration
  bool cert;        // certificate test of T(z) - z at this iteration (restart point or check)
  bool rp;          // restart point (k == 0, n >= 1): z_t is the anchor
  bool move;        // this restart's anchor movement z^{n+1,0} - z^{n,0} is tested
  bool stash;       // rHPDHG: keep x_{t+1}, K^T y_{t+1} (next iteration a check, or adaptive)
  int m_eq;
  bool redo = false;   // adaptive step: recompute T(z_t) from the stored z_t
  bool keep = false;   // adaptive step, rHPDHG: keep y_t, K x_t for a redo
};

// Row i of K^ x~_t = dot: forms y_t and K x_t by the pending blend (eq. hpdhg / eq. hrpdhg, or
// the restart point), takes the dual step of eq. pdhg, and accumulates the fixed-point-residual,
// check and certificate parts (slots above).  At a restart with move set, the old anchor gives
// the row parts of z^{n+1,0} - z^{n,0} before it is replaced.
template <int RHO2, class AS, class AM>
__device__ __forceinline__ void row_epilogue(int i, double dot, const RowVecs &v,
                                             const StepFlags &f, AS &S, AM &M) {
  const double ytp = v.yt[i], kxtp = v.kxt[i];
  const double w = f.w, sigma = f.step;
  const double qi = v.q[i];
  double yi, kxi, y0i;
  if (f.redo) {
    yi = v.y[i]; kxi = v.kx[i]; y0i = v.y0[i];
  } else if (f.restart) {
    if (f.move) {
      const double dyb = ytp - v.y0[i];                  // y^{n+1,0} - y^{n,0} (scaled)
      const double kdb = (kxtp - v.kx0[i]) * v.dinv[i];  // K (x^{n+1,0} - x^{n,0}) (unscaled)
      const double di = v.d[i];
      S.s[6] += qi * dyb;
      if (i >= f.m_eq) M.mx[3] = fmax(M.mx[3], fmax(-dyb * di, 0.0));
      if (i < f.m_eq) M.mx[4] = fmax(M.mx[4], fabs(kdb));
      else M.mx[5] = fmax(M.mx[5], fmax(-kdb, 0.0));
      v.certy2[i] = dyb * di;
    }
    yi = ytp; kxi = kxtp; y0i = yi;
    v.y0[i] = yi; v.kx0[i] = kxi;
    if (RHO2 || f.keep) { v.y[i] = yi; v.kx[i] = kxi; }
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
      if (f.keep) { v.y[i] = yi; v.kx[i] = kxi; }
    }
  }
  double yn = yi + sigma * (qi - 2.0 * dot + kxi);
  if (i >= f.m_eq) yn = fmax(yn, 0.0);
  v.yt[i] = yn;
  v.kxt[i] = dot;
  const double dy = yi - yn;
  S.s[0] += dy * dy;
  S.s[1] += dy * (kxi - dot);
  const double ya = yn - y0i;
  S.s[2] += ya * ya;
  if (f.check) {
    double r = (qi - dot) * v.dinv[i];
    if (i >= f.m_eq) r = fmax(r, 0.0);
    S.s[3] += r * r;
    S.s[4] += qi * yn;
  }
  if (f.cert) {
    const double vy = yn - yi;            // y-part of T(z) - z
    S.s[5] += qi * vy;
    const double di = v.d[i];
    if (i >= f.m_eq) M.mx[0] = fmax(M.mx[0], fmax(-vy * di, 0.0));
    const double kd = (dot - kxi) * v.dinv[i];   // K d (unscaled), d = x~ - x
    if (i < f.m_eq) M.mx[1] = fmax(M.mx[1], fabs(kd));
    else M.mx[2] = fmax(M.mx[2], fmax(-kd, 0.0));
    v.certy[i] = vy * di;
  }
}

// Column parts of one certificate candidate: d (scaled x-part), kv = K^T of its y-part
// (scaled); sums at s0 (c^T d), s0+1 / s0+2 (bound terms of the ray objective), maxima at
// m0..m0+3.  Writes the unscaled d to cert.
template <class V, class AS, class AM>
__device__ __forceinline__ void col_cert_parts(int j, double d, double kv, const V &v,
                                               double cj, double lj, double uj, AS &S, AM &M,
                                               int s0, int m0, double *cert) {
  S.s[s0] += cj * d;
  const double du = d * v.e[j];
  const bool lf = isfinite(lj), uf = isfinite(uj);
  if (lf) M.mx[m0] = fmax(M.mx[m0], fmax(-du, 0.0));
  if (uf) M.mx[m0 + 1] = fmax(M.mx[m0 + 1], fmax(du, 0.0));
  if (uf) S.s[s0 + 1] += fmax(kv, 0.0) * uj;
  else M.mx[m0 + 2] = fmax(M.mx[m0 + 2], fmax(kv * v.einv[j], 0.0));
  if (lf) S.s[s0 + 2] += fmax(-kv, 0.0) * lj;
  else M.mx[m0 + 3] = fmax(M.mx[m0 + 3], fmax(-kv * v.einv[j], 0.0));
  cert[j] = du;
}

// Column j of K^T y~_t = dot: the check parts at (x~_t, y~_t), the T(z) - z certificate parts
// (z_t is the anchor at a restart point, else the stored x_t, K^T y_t), then the blend to
// x_{t+1} (at a restart with move set, first the anchor-movement parts against the old
// anchor) and the primal step x~_{t+1} = proj_X(x_{t+1} - tau (c - K^T y_{t+1})).
// Per-thread active-set counts of a check iteration (see tel_flush).
struct Tel {
  int act = 0, chg = 0;
};

// Column j's on-bound status at a check: counts it and records it for the next check.
__device__ __forceinline__ void tel_column(int j, bool at, unsigned char *act, Tel &tl) {
  const unsigned char prev = act[j];
  tl.act += at ? 1 : 0;
  tl.chg += (at ? 1 : 0) != prev ? 1 : 0;
  act[j] = at ? 1 : 0;
}

// Adds the CTA's telemetry counts to the control block (integer atomics: exact and
// order-independent); called by every thread before the CTA's reduction and ticket.
__device__ __forceinline__ void tel_flush(Ctl *ctl, const Tel &tl) {
  int a = tl.act, c = tl.chg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0 && (a | c)) {
    atomicAdd(&ctl->tel_act, (unsigned long long)a);
    atomicAdd(&ctl->tel_chg, (unsigned long long)c);
  }
}

template <int RHO2, class AS, class AM>
__device__ __forceinline__ void col_epilogue(int j, double dot, const ColVecs &v,
                                             const StepFlags &f, AS &S, AM &M, Tel &tl) {
  const double xtj = v.xt[j];
  const double cj = v.c[j], lj = v.l[j], uj = v.u[j];
  const double w = f.w, tau = f.step;
  if (f.check) {
    tel_column(j, xtj == lj || xtj == uj, v.act, tl);
    const double g = cj - dot;
    const double lam = proj_lambda(g, lj, uj);
    const double rd = (g - lam) * v.einv[j];
    S.s[2] += rd * rd;
    S.s[3] += cj * xtj;
    if (lam > 0.0) S.s[4] += lj * lam;
    else if (lam < 0.0) S.s[4] += uj * lam;
    v.xout[j] = xtj;
  }
  double x0j = v.x0[j], kty0j = v.kty0[j];
  if (f.cert) {
    const double xc = f.rp ? x0j : v.x[j];
    const double kc = f.rp ? kty0j : v.kty[j];
    col_cert_parts(j, xtj - xc, dot - kc, v, cj, lj, uj, S, M, 5, 0, v.certx);
  }
  double xn, kn;
  if (f.restart) {
    if (f.move) col_cert_parts(j, xtj - x0j, dot - kty0j, v, cj, lj, uj, S, M, 8, 4, v.certx2);
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
  if (!RHO2 && f.stash) { v.x[j] = xn; v.kty[j] = kn; }
  const double xtn = fmin(fmax(xn - tau * (cj - kn), lj), uj);
  v.xt[j] = xtn;
  const double dx = xn - xtn;
  S.s[0] += dx * dx;
  const double xa = xtn - x0j;
  S.s[1] += xa * xa;
}

}  // namespace rh
