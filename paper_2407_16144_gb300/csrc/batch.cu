// Batched solver: many small LPs advance in one persistent launch, one CTA per LP.
//
// Each LP owns a region of a device arena (CSR of K and its transpose, the vectors of the FP64
// path, its control block and constants) described by a slot-table entry.  One launch of
// k_batch advances every active slot by up to `iters` PDHG evaluations; a slot that is new first
// runs the whole set-up in its CTA (Ruiz and Pock-Chambolle scaling, power iteration for the step
// size, primal weight, initial point), so admitting an LP costs no extra launches.  The
// iteration is the FP64 method of the single-LP path (same epilogues, same restart rule, same
// termination and certificate tests) with the two products computed by groups of G threads per
// row and the reductions done inside the CTA.  Nothing in a CTA depends on other slots, so an LP
// gives bit-identical results alone and in any mix.  The slot table lives on the device and is
// read by the kernel, so one captured graph is replayed while slots come and go.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rhpdhg.h"
#include "internal.h"
#include "iter_common.cuh"
#include "iter_mx_common.cuh"

namespace rh {

namespace {

constexpr int kBT = 256;   // threads per CTA of the batched kernel

struct BatchDesc {
  int active;              // 1 = slot in use
  int m, m_eq, n, nnz;
  int gr, gc;              // threads per row for K x~ (gr) and K^T y~ (gc)
  int ruiz_iters, power_iters;
  double pc_alpha, step_size, step_safety, primal_weight;
  const int *rp, *ci;      // CSR of K (m+1, nnz)
  double *rv;              // values, scaled in place during set-up
  const int *cp, *ri;      // CSC of K (n+1, nnz)
  double *cv;
  double *tmp_m, *tmp_n;   // set-up scratch
  RowVecs rv_;             // y, y~, y0, Kx, Kx~, Kx0, certy, q (scaled in place), D, Dinv
  ColVecs cv_;             // x, x~, x0, K^T y, K^T y0, xout, certx, c, l, u (scaled), E, Einv
  Ctl *ctl;
  IterConsts *ic;          // per-slot constants (eta, norms filled by set-up); ic->mixed is the
                           // slot's current mode (a mixed slot that escalates turns it to 0)
  double *setup_out;       // sigma_max, omega0 (for inspection)
  // mixed precision (precision 1): FP32 copies of the scaled values and the FP32-offset state
  int mixed;
  float *rv32, *cv32;
  RowVecsMx rvm;
  ColVecsMx cvm;
};

template <typename T>
__device__ __forceinline__ T group_sum(T v, int g) {
  for (int o = g >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, g);
  return v;
}
__device__ __forceinline__ double group_max(double v, int g) {
  for (int o = g >> 1; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o, g));
  return v;
}

// Block reduction of the NS sums and NM maxima selected by the masks into out (valid in thread
// 0; other slots 0); deterministic.  Sum slots set in prewarp already hold their warp's sum.
template <int NS, int NM>
__device__ void block_reduce(const Acc<NS, NM> &a, double *out, double *sh,
                             unsigned smask = 0xFFFFu, unsigned mmask = 0xFFFFu,
                             unsigned prewarp = 0u) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned all = (smask & ((1u << NS) - 1u)) | ((mmask & ((1u << NM) - 1u)) << NS);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NS + NM; ++i) {
    if (!((all >> i) & 1u)) continue;
    double v = i < NS ? a.s[i] : a.mx[i - NS];
    if (i >= NS) v = warp_max(v);
    else if (!((prewarp >> i) & 1u)) v = warp_sum(v);
    if (lane == 0) sh[warp * (NS + NM) + i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS + NM; ++i) {
      if (!((all >> i) & 1u)) { out[i] = 0.0; continue; }
      double v = sh[i];
      for (int w = 1; w < kBT / 32; ++w)
        v = i < NS ? v + sh[w * (NS + NM) + i] : fmax(v, sh[w * (NS + NM) + i]);
      out[i] = v;
    }
  }
  __syncthreads();
}

__device__ double block_sum1(double v, double *sh) {
  Acc<1, 0> a;
  a.s[0] = v;
  double out[1] = {0.0};
  block_reduce(a, out, sh);
  if (threadIdx.x == 0) sh[0] = out[0];
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

// For each row r of a CSR (rows, ptr, idx, val): dot = sum val * src[idx], then fn(r, dot).
// A warp owns 32 consecutive rows; groups of g lanes compute 32/g rows per pass (g passes),
// each result is handed to the lane that owns the row, and fn then runs for 32 rows at once,
// one per lane, so the epilogue keeps every lane busy.  Trip counts are warp-uniform.  VT is
// the value and sum type (FP64, or FP32 for the ordinary mixed-precision iterations).
template <typename VT, typename Src, typename Fn>
__device__ __forceinline__ void rows_apply(int nrows, const int *ptr, const int *idx,
                                           const VT *val, int g, const Src &src, Fn &fn) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpp = 32 / g, gid = lane / g, gl = lane % g;
  for (int base = warp * 32; base < nrows; base += kBT) {
    VT mine = VT(0);
    for (int pass = 0; pass < g; ++pass) {
      const int r = base + pass * rpp + gid;
      VT s = VT(0);
      if (r < nrows)
        for (int p = ptr[r] + gl; p < ptr[r + 1]; p += g) s += val[p] * VT(src(idx[p]));
      s = group_sum(s, g);
      const VT got = __shfl_sync(0xffffffffu, s, (lane % rpp) * g);
      if (lane / rpp == pass) mine = got;
    }
    const int r = base + lane;
    if (r < nrows) fn(r, mine);
  }
}

// Per-row statistic over |K^_ij| = |v| rs_r cs_j: OP 0 max, OP 1 sum of powers.
template <int OP>
__device__ void rows_stat(int nrows, const int *ptr, const int *idx, const double *val, int g,
                          const double *rs, const double *cs, double alpha, double *out) {
  const int gid = threadIdx.x / g, gl = threadIdx.x % g, ngroups = kBT / g;
  for (int base = 0; base < nrows; base += ngroups) {
    const int r = base + gid;
    double s = 0.0;
    if (r < nrows) {
      const double sr = rs[r];
      for (int p = ptr[r] + gl; p < ptr[r + 1]; p += g) {
        const double a = fabs(val[p]) * sr * cs[idx[p]];
        if (OP == 0) s = fmax(s, a);
        else s += (alpha == 1.0) ? a : pow(a, alpha);
      }
    }
    s = OP == 0 ? group_max(s, g) : group_sum(s, g);
    if (gl == 0 && r < nrows) out[r] = s;
  }
}

__device__ void scale_update(int n, const double *stat, double *scale) {
  for (int i = threadIdx.x; i < n; i += kBT) {
    const double s = stat[i];
    if (s > 0.0) scale[i] = scale[i] / sqrt(s);
  }
}

// The whole create-time pipeline of one LP, inside its CTA.
__device__ void batch_setup(const BatchDesc &d, double *sh) {
  const int m = d.m, n = d.n;
  RowVecs rvv = d.rv_;
  ColVecs cvv = d.cv_;
  double *D = const_cast<double *>(rvv.d), *E = const_cast<double *>(cvv.e);
  double *Dinv = const_cast<double *>(rvv.dinv), *Einv = const_cast<double *>(cvv.einv);
  double *q = const_cast<double *>(rvv.q), *c = const_cast<double *>(cvv.c);
  double *l = const_cast<double *>(cvv.l), *u = const_cast<double *>(cvv.u);
  // norms of the unscaled data
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < m; i += kBT) a += q[i] * q[i];
  for (int j = threadIdx.x; j < n; j += kBT) b += c[j] * c[j];
  const double qn = sqrt(block_sum1(a, sh)), cn = sqrt(block_sum1(b, sh));
  // Ruiz then Pock-Chambolle
  for (int i = threadIdx.x; i < m; i += kBT) D[i] = 1.0;
  for (int j = threadIdx.x; j < n; j += kBT) E[j] = 1.0;
  __syncthreads();
  for (int it = 0; it < d.ruiz_iters; ++it) {
    rows_stat<0>(m, d.rp, d.ci, d.rv, d.gr, D, E, 1.0, d.tmp_m);
    rows_stat<0>(n, d.cp, d.ri, d.cv, d.gc, E, D, 1.0, d.tmp_n);
    __syncthreads();
    scale_update(m, d.tmp_m, D);
    scale_update(n, d.tmp_n, E);
    __syncthreads();
  }
  if (d.pc_alpha >= 0.0) {
    rows_stat<1>(m, d.rp, d.ci, d.rv, d.gr, D, E, d.pc_alpha, d.tmp_m);
    rows_stat<1>(n, d.cp, d.ri, d.cv, d.gc, E, D, 2.0 - d.pc_alpha, d.tmp_n);
    __syncthreads();
    scale_update(m, d.tmp_m, D);
    scale_update(n, d.tmp_n, E);
    __syncthreads();
  }
  // scaled matrix values (row side: D_i K_ij E_j; column side: E_j K_ij D_i) and vectors
  {
    const int g = d.gr, gid = threadIdx.x / g, gl = threadIdx.x % g, ng = kBT / g;
    for (int r = gid; r < m; r += ng)
      for (int p = d.rp[r] + gl; p < d.rp[r + 1]; p += g) d.rv[p] = D[r] * d.rv[p] * E[d.ci[p]];
    const int g2 = d.gc, gid2 = threadIdx.x / g2, gl2 = threadIdx.x % g2, ng2 = kBT / g2;
    for (int r = gid2; r < n; r += ng2)
      for (int p = d.cp[r] + gl2; p < d.cp[r + 1]; p += g2) d.cv[p] = E[r] * d.cv[p] * D[d.ri[p]];
    if (d.mixed) {
      __syncthreads();
      for (int p = threadIdx.x; p < d.nnz; p += kBT) {
        d.rv32[p] = (float)d.rv[p];
        d.cv32[p] = (float)d.cv[p];
      }
    }
  }
  for (int i = threadIdx.x; i < m; i += kBT) {
    q[i] = D[i] * q[i];
    Dinv[i] = 1.0 / D[i];
  }
  for (int j = threadIdx.x; j < n; j += kBT) {
    c[j] = E[j] * c[j];
    l[j] = l[j] / E[j];
    u[j] = u[j] / E[j];
    Einv[j] = 1.0 / E[j];
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
  for (int i = threadIdx.x; i < m; i += kBT) a += q[i] * q[i];
  for (int j = threadIdx.x; j < n; j += kBT) b += c[j] * c[j];
  const double qhn = sqrt(block_sum1(a, sh)), chn = sqrt(block_sum1(b, sh));
  // power iteration on K^T K from 1/sqrt(n): v in x, K v in kx, K^T K v in kty
  double *v = cvv.x, *um = rvv.kx, *w = cvv.kty;
  for (int j = threadIdx.x; j < n; j += kBT) v[j] = 1.0 / sqrt((double)n);
  __syncthreads();
  double smax = 0.0;
  if (m > 0 && d.nnz > 0) {
    for (int it = 0; it < d.power_iters; ++it) {
      auto f1 = [&](int r, double s) { um[r] = s; };
      auto g1 = [&](int j) { return v[j]; };
      rows_apply(m, d.rp, d.ci, d.rv, d.gr, g1, f1);
      __syncthreads();
      auto f2 = [&](int r, double s) { w[r] = s; };
      auto g2 = [&](int i) { return um[i]; };
      rows_apply(n, d.cp, d.ri, d.cv, d.gc, g2, f2);
      __syncthreads();
      double ss = 0.0;
      for (int j = threadIdx.x; j < n; j += kBT) ss += w[j] * w[j];
      const double nrm = sqrt(block_sum1(ss, sh));
      for (int j = threadIdx.x; j < n; j += kBT) v[j] = nrm > 0.0 ? w[j] / nrm : 0.0;
      __syncthreads();
    }
    auto f1 = [&](int r, double s) { um[r] = s; };
    auto g1 = [&](int j) { return v[j]; };
    rows_apply(m, d.rp, d.ci, d.rv, d.gr, g1, f1);
    __syncthreads();
    double ss = 0.0;
    for (int i = threadIdx.x; i < m; i += kBT) ss += um[i] * um[i];
    smax = sqrt(block_sum1(ss, sh));
  }
  double eta;
  if (d.step_size > 0) eta = d.step_size;
  else if (smax > 1e-12) eta = d.step_safety / smax;
  else eta = 1.0;
  const double om0 = d.primal_weight > 0
                         ? d.primal_weight
                         : ((chn > 1e-10 && qhn > 1e-10) ? chn / qhn : 1.0);
  // initial point z^{0,0} = (proj_X(0), 0) in the PDHG-point slots, K x^{0,0} in K x~
  for (int j = threadIdx.x; j < n; j += kBT) cvv.xt[j] = fmin(fmax(0.0, l[j]), u[j]);
  for (int i = threadIdx.x; i < m; i += kBT) rvv.yt[i] = 0.0;
  __syncthreads();
  {
    auto f1 = [&](int r, double s) { rvv.kxt[r] = s; };
    auto g1 = [&](int j) { return cvv.xt[j]; };
    rows_apply(m, d.rp, d.ci, d.rv, d.gr, g1, f1);
  }
  if (d.mixed) {
    // anchors z^{0,0} and zero FP32 offsets; the set-up column pass then runs in restart mode
    const RowVecsMx &rm = d.rvm;
    const ColVecsMx &cm = d.cvm;
    for (int j = threadIdx.x; j < n; j += kBT) {
      cm.x0[j] = cvv.xt[j];
      cm.dxt[j] = 0.f;
      cm.dx[j] = 0.f;
      cm.ktdy[j] = 0.f;
    }
    for (int i = threadIdx.x; i < m; i += kBT) {
      rm.y0[i] = 0.0;
      rm.dyt[i] = 0.f;
      rm.kdxt[i] = 0.f;
      rm.dy[i] = 0.f;
      rm.kdx[i] = 0.f;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    d.ic->eta = eta;
    d.ic->qn1 = 1.0 + qn;
    d.ic->cn1 = 1.0 + cn;
    d.setup_out[0] = smax;
    d.setup_out[1] = om0;
    Ctl *ctl = d.ctl;
    ctl->t = 0; ctl->k = 0; ctl->n = 0; ctl->k_next = 0; ctl->n_next = 0;
    ctl->restart_pending = 1;
    ctl->w = 0.0;
    ctl->omega = om0;
    set_steps(ctl, eta, om0);
    ctl->eta = eta;
    ctl->stage = 1;
    ctl->check_t = -1;
  }
  __syncthreads();
}

template <int RHO2>
__device__ void batch_col_pass(const BatchDesc &d, const IterConsts &ic, int phase, double *sh) {
  Ctl *ctl = d.ctl;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const bool check = phase == 0 && (((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters));
  const bool rp = phase == 0 && (k == 0 && n_ep >= 1);
  const bool cert = rp || check;
  const int restart = ctl->restart_pending;
  const bool move = phase == 0 && restart;
  const long long tn = phase == 0 ? t + 1 : t;
  const bool stash = ((tn + 1) % ic.check_every == 0) || (tn + 1 >= ic.max_iters);
  StepFlags fl{restart, ctl->w, ctl->tau, check, cert, rp, move, stash, ic.m_eq};
  ColAcc a;
  a.zero();
  Tel tl;
  auto fn = [&](int j, double dot) { col_epilogue<RHO2>(j, dot, d.cv_, fl, a, a, tl); };
  const double *yt = d.rv_.yt;
  auto gs = [&](int i) { return yt[i]; };
  rows_apply(d.n, d.cp, d.ri, d.cv, d.gc, gs, fn);
  if (check) tel_flush(ctl, tl);
  double r[19];
  block_reduce(a, r, sh, col_smask(check, cert, move), col_mmask(cert, move));
  if (threadIdx.x == 0) col_finalize(ctl, ic, r, t, check, cert, rp, move, phase);
  __syncthreads();
}

template <int RHO2>
__device__ void batch_row_pass(const BatchDesc &d, const IterConsts &ic, double *sh) {
  Ctl *ctl = d.ctl;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const bool check = ((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters);
  const bool rp = (k == 0 && n_ep >= 1);
  const bool cert = rp || check;
  const int restart = ctl->restart_pending;
  const bool move = restart && ctl->mv_ready;
  const double sigma = ctl->sigma;
  StepFlags fl{restart, ctl->w, sigma, check, cert, rp, move, false, ic.m_eq};
  RowAcc a;
  a.zero();
  auto fn = [&](int i, double dot) { row_epilogue<RHO2>(i, dot, d.rv_, fl, a, a); };
  const double *xt = d.cv_.xt;
  auto gs = [&](int j) { return xt[j]; };
  rows_apply(d.m, d.rp, d.ci, d.rv, d.gr, gs, fn);
  double r[13];
  block_reduce(a, r, sh, row_smask(check, cert, move), row_mmask(cert, move));
  if (threadIdx.x == 0) row_finalize(ctl, ic, r, t, k, n_ep, sigma, move);
  __syncthreads();
}

// The FP32 restart-norm sums of a thread, summed over its warp in FP32 and placed in the FP64
// slots of a (lane 0 holds the warp's sum; block_reduce adds the warps in FP64).
template <int N, class A>
__device__ __forceinline__ unsigned warp_sums_to(FprSums<N, 0> &f, A &a) {
#pragma unroll
  for (int i = 0; i < N; ++i) a.s[i] = (double)warp_sum(f.v[i].hi);
  return (1u << N) - 1u;
}

// ---- mixed precision in a slot: the bodies of the tiled mixed kernels (iter_mx_common.cuh) over
// the slot's CSR copies, FP32 matrix values in ordinary iterations and FP64 at restarts and
// restart points; the restart-norm sums are FP32 within each warp and FP64 across the warps.

template <int RHO2>
__device__ void batch_row_pass_mx(const BatchDesc &d, const IterConsts &ic, double *sh) {
  Ctl *ctl = d.ctl;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const bool check = ((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters);
  const bool rp = (k == 0 && n_ep >= 1);
  const int restart = ctl->restart_pending;
  const bool move = restart && ctl->mv_ready;
  const double sigma = ctl->sigma;
  const float wf = (float)ctl->w, sigf = (float)sigma;
  const RowVecsMx &v = d.rvm;
  const int m_eq = ic.m_eq;
  Acc<7, 6> a;
  a.zero();
  unsigned prewarp = 0u;
  if (restart) {
    // K x0' with the FP64 values (and the anchor movement's row parts), then the dual step of
    // the restart point in FP64 from K dxt (dxt exact in dxt64)
    const double *x0 = d.cvm.x0;
    auto gA = [&](int j) { return x0[j]; };
    auto fA = [&](int i, double dot) {
      if (move) row_mx_move(i, dot, v, m_eq, a, a);
      v.kx0[i] = dot;
    };
    rows_apply(d.m, d.rp, d.ci, d.rv, d.gr, gA, fA);
    __syncthreads();
    const double *dxt64 = d.cvm.dxt64;
    auto gB = [&](int j) { return dxt64[j]; };
    auto fB = [&](int i, double kd) {
      row_mx_restart<RHO2>(i, kd, v, sigma, m_eq, check, rp, a, a);
    };
    rows_apply(d.m, d.rp, d.ci, d.rv, d.gr, gB, fB);
  } else {
    FprSums<3, 0> f;
    const float *dxt = d.cvm.dxt;
    auto g = [&](int j) { return dxt[j]; };
    auto fn = [&](int i, float kd) { row_mx_ordinary<RHO2>(i, kd, v, wf, sigf, m_eq, check, a, f); };
    rows_apply(d.m, d.rp, d.ci, d.rv32, d.gr, g, fn);
    prewarp = warp_sums_to(f, a);
  }
  double r[13];
  block_reduce(a, r, sh, row_smask(check, rp, move), row_mmask(rp, move), prewarp);
  if (threadIdx.x == 0) row_finalize(ctl, ic, r, t, k, n_ep, sigma, move);
  __syncthreads();
}

template <int RHO2>
__device__ void batch_col_pass_mx(const BatchDesc &d, const IterConsts &ic, int phase,
                                  double *sh) {
  Ctl *ctl = d.ctl;
  const long long t = ctl->t, k = ctl->k, n_ep = ctl->n;
  const int restart = ctl->restart_pending;
  const bool rp = phase == 0 && (k == 0 && n_ep >= 1);
  const bool move = phase == 0 && restart;
  const bool check = phase == 0 && (((t + 1) % ic.check_every == 0) || (t + 1 >= ic.max_iters));
  const double tau = ctl->tau;
  const float wf = (float)ctl->w, tauf = (float)tau;
  const ColVecsMx &v = d.cvm;
  Acc<11, 8> a;
  a.zero();
  Tel tl;
  unsigned prewarp = 0u;
  if (restart) {
    // z^{n+1,0} = T(z^{n,k}): K^T y0' with the FP64 values from the gathered y0 + dyt
    const double *y0 = d.rvm.y0;
    const float *dyt = d.rvm.dyt;
    auto g = [&](int i) { return y0[i] + (double)dyt[i]; };
    auto fn = [&](int j, double kty) {
      col_mx_restart<RHO2>(j, kty, v, tau, check, rp, move, a, a);
    };
    rows_apply(d.n, d.cp, d.ri, d.cv, d.gc, g, fn);
  } else if (rp) {
    const double *dyt64 = d.rvm.dyt64;
    auto g = [&](int i) { return dyt64[i]; };
    auto fn = [&](int j, double ktd) {
      col_mx_first<RHO2>(j, ktd, v, wf, tauf, check, rp, ic.no_upper, a, a);
    };
    rows_apply(d.n, d.cp, d.ri, d.cv, d.gc, g, fn);
  } else {
    FprSums<2, 0> f;
    const float *dyt = d.rvm.dyt;
    auto g = [&](int i) { return dyt[i]; };
    auto fn = [&](int j, float ktdyt) {
      col_mx_ordinary<RHO2>(j, ktdyt, v, wf, tauf, check, ic.no_upper, a, a, f, tl);
    };
    rows_apply(d.n, d.cp, d.ri, d.cv32, d.gc, g, fn);
    if (check) tel_flush(ctl, tl);
    prewarp = warp_sums_to(f, a);
  }
  double r[19];
  block_reduce(a, r, sh, col_smask(check, rp, move), col_mmask(rp, move), prewarp);
  if (threadIdx.x == 0)
    col_finalize(ctl, ic, r, t, check, rp, rp, move, phase, !restart && !rp);
  __syncthreads();
}

// A mixed slot whose restart-point certificate candidate came within 1e-3 of the test
// (kEscalate) continues in FP64 from that restart point, the FP64 anchor z^{n,0}: the FP64 state
// starts there as at the start of a solve, with the iteration and epoch counters, the primal
// weight and the step carried on, and the slot stays FP64.
template <int RHO2>
__device__ void batch_escalate(const BatchDesc &d, IterConsts &ic, double *sh) {
  const RowVecs &rv = d.rv_;
  const ColVecs &cv = d.cv_;
  for (int j = threadIdx.x; j < d.n; j += kBT) cv.xt[j] = cv.x0[j];
  for (int i = threadIdx.x; i < d.m; i += kBT) rv.yt[i] = rv.y0[i];
  __syncthreads();
  auto f1 = [&](int r, double s) { rv.kxt[r] = s; };
  auto g1 = [&](int j) { return cv.xt[j]; };
  rows_apply(d.m, d.rp, d.ci, d.rv, d.gr, g1, f1);
  __syncthreads();
  if (threadIdx.x == 0) {
    Ctl *ctl = d.ctl;
    ctl->status = kRunning;
    ctl->restart_pending = 1;
    ctl->stage = 1;
    ctl->k = 0;
    ctl->k_next = 0;
    ctl->n_next = ctl->n;
    ctl->mv_ready = 0;
    ctl->escalated = 1;
    d.ic->mixed = 0;
    ic.mixed = 0;
  }
  __syncthreads();
  batch_col_pass<RHO2>(d, ic, 1, sh);
}

template <int RHO2>
__device__ void batch_iterate(const BatchDesc &d, IterConsts &ic, int iters, double *sh) {
  Ctl *ctl = d.ctl;
  for (int it = 0; it < iters; ++it) {
    if (ctl->status == kEscalate) batch_escalate<RHO2>(d, ic, sh);
    if (ctl->status != kRunning) break;
    if (ic.mixed) batch_row_pass_mx<RHO2>(d, ic, sh);
    else batch_row_pass<RHO2>(d, ic, sh);
    if (ctl->status != kRunning) continue;
    if (ic.mixed) batch_col_pass_mx<RHO2>(d, ic, 0, sh);
    else batch_col_pass<RHO2>(d, ic, 0, sh);
  }
  if (ctl->status == kEscalate) batch_escalate<RHO2>(d, ic, sh);
}

__global__ void __launch_bounds__(kBT)
k_batch(const BatchDesc *__restrict__ descs, int nslots, int iters) {
  __shared__ double sh[(kBT / 32) * kMaxPartials];
  __shared__ IterConsts ics;
  const int slot = blockIdx.x;
  if (slot >= nslots) return;
  const BatchDesc d = descs[slot];
  if (!d.active) return;
  Ctl *ctl = d.ctl;
  if (ctl->status != kRunning && ctl->status != kEscalate) return;
  if (ctl->stage == 2) {            // new slot: set-up, then the set-up column step
    batch_setup(d, sh);
    if (threadIdx.x == 0) ics = *d.ic;
    __syncthreads();
    if (ics.mixed) {
      if (ics.rho2) batch_col_pass_mx<1>(d, ics, 1, sh);
      else batch_col_pass_mx<0>(d, ics, 1, sh);
    } else {
      if (ics.rho2) batch_col_pass<1>(d, ics, 1, sh);
      else batch_col_pass<0>(d, ics, 1, sh);
    }
  } else {
    if (threadIdx.x == 0) ics = *d.ic;
    __syncthreads();
  }
  if (ics.rho2) batch_iterate<1>(d, ics, iters, sh);
  else batch_iterate<0>(d, ics, iters, sh);
}

// Unscaled result of a slot: x = E x~ of the last check; y = D y~, where a slot still in mixed
// precision holds y~ as y0 + dyt.
__global__ void k_batch_unscale(const BatchDesc *__restrict__ descs, int slot, double *xo,
                                double *yo) {
  const BatchDesc d = descs[slot];
  const bool mixed = d.mixed && d.ic->mixed;
  for (int j = threadIdx.x + blockIdx.x * blockDim.x; j < d.n; j += blockDim.x * gridDim.x)
    xo[j] = d.cv_.e[j] * d.cv_.xout[j];
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < d.m; i += blockDim.x * gridDim.x)
    yo[i] = d.rv_.d[i] * (mixed ? d.rvm.y0[i] + (double)d.rvm.dyt[i] : d.rv_.yt[i]);
}

int pick_group(double avg) {
  // group size of the per-row products: the power of two nearest half the mean row length,
  // in [1, 32] (a lane then handles about two entries of an average row)
  int g = 1;
  while (g < 32 && 2 * g < avg) g *= 2;
  return g;
}

}  // namespace

}  // namespace rh

// ---------------------------------------------------------------------------------------------
// host side

struct rhpdhg_batch {
  int dev = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int max_slots = 0;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  struct Region { size_t off, size; };
  std::vector<Region> free_list;           // sorted by offset
  std::vector<Region> slot_region;
  std::vector<rh::BatchDesc> host_desc;
  std::vector<int> slot_m, slot_n, slot_status_read;
  std::vector<double> slot_off;
  std::vector<rhpdhg_params> slot_params;
  rh::BatchDesc *d_desc = nullptr;
  rh::Ctl *d_ctls = nullptr;               // every slot's control block (contiguous)
  rh::Ctl *h_ctl = nullptr;                // pinned copies of them
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = -1;
  std::string err;
  long long launches = 0;
};

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Arena bytes of one slot: both CSR copies, the FP64 vectors, and for a mixed-precision slot the
// FP32 values of both copies, six FP32 offset vectors per side and the exact FP64 offsets of the
// restart points.
size_t slot_bytes(int m, int n, long long nnz, bool mixed) {
  size_t b = 0;
  const size_t nn = (size_t)std::max(n, 1), mm = (size_t)std::max(m, 1);
  b += align256((m + 1) * sizeof(int)) + align256(nnz * sizeof(int)) + align256(nnz * 8);
  b += align256((n + 1) * sizeof(int)) + align256(nnz * sizeof(int)) + align256(nnz * 8);
  b += 15 * align256(nn * 8) + 13 * align256(mm * 8);
  b += align256(sizeof(rh::IterConsts)) + align256(16) + align256(nn);
  if (mixed)
    b += 2 * align256(nnz * 4) + 6 * align256(nn * 4) + 6 * align256(mm * 4) + align256(nn * 8) +
         align256(mm * 8);
  return b;
}

bool arena_alloc(rhpdhg_batch *b, size_t size, size_t *off) {
  for (size_t i = 0; i < b->free_list.size(); ++i) {
    auto &r = b->free_list[i];
    if (r.size >= size) {
      *off = r.off;
      r.off += size;
      r.size -= size;
      if (r.size == 0) b->free_list.erase(b->free_list.begin() + i);
      return true;
    }
  }
  return false;
}

void arena_release(rhpdhg_batch *b, size_t off, size_t size) {
  auto &fl = b->free_list;
  auto it = std::lower_bound(fl.begin(), fl.end(), off,
                             [](const rhpdhg_batch::Region &r, size_t o) { return r.off < o; });
  it = fl.insert(it, {off, size});
  // merge with neighbours
  size_t i = it - fl.begin();
  if (i + 1 < fl.size() && fl[i].off + fl[i].size == fl[i + 1].off) {
    fl[i].size += fl[i + 1].size;
    fl.erase(fl.begin() + i + 1);
  }
  if (i > 0 && fl[i - 1].off + fl[i - 1].size == fl[i].off) {
    fl[i - 1].size += fl[i].size;
    fl.erase(fl.begin() + i);
  }
}

int berr(rhpdhg_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg;
  rh::set_global_error(msg);
  return code;
}

}  // namespace

extern "C" {

int rhpdhg_batch_create(int32_t max_slots, int64_t arena_bytes, void *cuda_stream,
                        rhpdhg_batch **out) {
  if (!out) return RHPDHG_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_slots < 1 || arena_bytes < 1)
    return berr(nullptr, RHPDHG_ERR_INVALID_ARG, "batch: max_slots and arena_bytes must be > 0");
  rhpdhg_batch *b = new rhpdhg_batch();
  cudaGetDevice(&b->dev);
  b->st = (cudaStream_t)cuda_stream;
  if (!b->st) {
    cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  b->max_slots = max_slots;
  b->arena_bytes = align256((size_t)arena_bytes);
  cudaError_t e = cudaMalloc(&b->arena, b->arena_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_desc, max_slots * sizeof(rh::BatchDesc));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ctls, max_slots * sizeof(rh::Ctl));
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&b->h_ctl, max_slots * sizeof(rh::Ctl), 0);
  if (e != cudaSuccess) {
    rhpdhg_batch_free(b);
    return berr(nullptr, RHPDHG_ERR_OOM, std::string("batch: ") + cudaGetErrorString(e));
  }
  b->free_list.push_back({0, b->arena_bytes});
  b->slot_region.assign(max_slots, {0, 0});
  b->host_desc.assign(max_slots, rh::BatchDesc{});
  b->slot_m.assign(max_slots, 0);
  b->slot_n.assign(max_slots, 0);
  b->slot_off.assign(max_slots, 0.0);
  b->slot_params.assign(max_slots, rhpdhg_params{});
  std::memset(b->h_ctl, 0, max_slots * sizeof(rh::Ctl));
  cudaMemsetAsync(b->d_desc, 0, max_slots * sizeof(rh::BatchDesc), b->st);
  cudaMemsetAsync(b->d_ctls, 0, max_slots * sizeof(rh::Ctl), b->st);
  cudaStreamSynchronize(b->st);
  *out = b;
  return RHPDHG_OK;
}

int rhpdhg_batch_add(rhpdhg_batch *b, const rhpdhg_problem *lp, const rhpdhg_params *p,
                     int32_t *slot_out) {
  if (!b || !lp || !slot_out) return RHPDHG_ERR_INVALID_ARG;
  if (lp->memory != RHPDHG_MEM_HOST)
    return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: problems are taken from host memory");
  const int m = lp->m_eq + lp->m_ineq, n = lp->n;
  const long long nnz = lp->nnz;
  if (lp->m_eq < 0 || lp->m_ineq < 0 || n < 1 || nnz < 0 || nnz > INT32_MAX - 1 ||
      !lp->row_ptr || !lp->c || !lp->l || !lp->u || (m > 0 && !lp->rhs) ||
      (nnz > 0 && (!lp->col_idx || !lp->val)))
    return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: invalid problem sizes or arrays");
  rhpdhg_params P;
  if (p) P = *p;
  else rhpdhg_params_default(&P);
  if (P.precision != 0 && P.precision != 1)
    return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: precision is 0 (FP64) or 1 (mixed)");
  if (P.adaptive_step)
    return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: batched slots use the constant step");
  if (P.algorithm < 0 || P.algorithm > 1 || P.check_every < 1 || P.max_iters < 1 ||
      !(P.eps_rel_kkt > 0) || !(P.eps_infeas > 0) || P.first_epoch_len < 0 ||
      P.max_epoch_len < 0 || P.restart_scheme < 0 || P.restart_scheme > 2 ||
      (P.restart_scheme >= 1 && P.max_epoch_len < 1) ||
      !(P.restart_beta > 0 && P.restart_beta < 1))
    return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: invalid parameter");
  // host validation and transpose (the batched path serves small LPs)
  const int64_t *rp = lp->row_ptr;
  if (rp[0] != 0 || rp[m] != nnz) return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: malformed row_ptr");
  std::vector<int> rp32(m + 1), ci(nnz), cp(n + 2, 0), ri(nnz);
  std::vector<double> cv(nnz);
  for (int i = 0; i < m; ++i) {
    if (rp[i + 1] < rp[i]) return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: malformed row_ptr");
    rp32[i] = (int)rp[i];
    int prev = -1;
    for (long long q = rp[i]; q < rp[i + 1]; ++q) {
      const int j = lp->col_idx[q];
      if (j < 0 || j >= n || j <= prev || !std::isfinite(lp->val[q]))
        return berr(b, RHPDHG_ERR_INVALID_ARG,
                    "batch: column index out of range / not increasing, or non-finite value");
      prev = j;
      ci[q] = j;
      cp[j + 2]++;
    }
    if (!std::isfinite(lp->rhs[i])) return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: non-finite rhs");
  }
  rp32[m] = (int)nnz;
  bool any_upper = false;
  for (int j = 0; j < n; ++j) {
    if (!std::isfinite(lp->c[j]) || std::isnan(lp->l[j]) || std::isnan(lp->u[j]) ||
        lp->l[j] > lp->u[j] || lp->l[j] == INFINITY || lp->u[j] == -INFINITY)
      return berr(b, RHPDHG_ERR_INVALID_ARG, "batch: invalid c or bounds");
    any_upper = any_upper || std::isfinite(lp->u[j]);
  }
  for (int j = 0; j < n; ++j) cp[j + 2] += cp[j + 1];
  for (int i = 0; i < m; ++i)
    for (long long q = rp[i]; q < rp[i + 1]; ++q) {
      const int j = ci[q];
      const int pos = cp[j + 1]++;
      ri[pos] = i;
      cv[pos] = lp->val[q];
    }
  cp.resize(n + 1);
  // slot and arena region
  int slot = -1;
  for (int s = 0; s < b->max_slots; ++s)
    if (!b->host_desc[s].active) { slot = s; break; }
  if (slot < 0) return berr(b, RHPDHG_BUSY, "batch: no free slot");
  const bool mixed = P.precision == 1;
  const size_t need = slot_bytes(m, n, nnz, mixed);
  size_t off = 0;
  if (!arena_alloc(b, need, &off)) return berr(b, RHPDHG_ERR_OOM, "batch: arena full");
  char *base = b->arena + off;
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    char *ptr = base + cur;
    cur += align256(bytes);
    return ptr;
  };
  rh::BatchDesc d{};
  d.active = 1;
  d.m = m; d.m_eq = lp->m_eq; d.n = n; d.nnz = (int)nnz;
  d.gr = rh::pick_group(m > 0 ? (double)nnz / m : 1.0);
  d.gc = rh::pick_group((double)nnz / n);
  d.ruiz_iters = P.ruiz_iters;
  d.power_iters = P.power_iters;
  d.pc_alpha = P.pock_chambolle_alpha;
  d.step_size = P.step_size;
  d.step_safety = P.step_safety;
  d.primal_weight = P.primal_weight;
  int *d_rp = (int *)take((m + 1) * sizeof(int));
  int *d_ci = (int *)take(nnz * sizeof(int));
  double *d_rv = (double *)take(nnz * 8);
  int *d_cp = (int *)take((n + 1) * sizeof(int));
  int *d_ri = (int *)take(nnz * sizeof(int));
  double *d_cv = (double *)take(nnz * 8);
  d.rp = d_rp; d.ci = d_ci; d.rv = d_rv; d.cp = d_cp; d.ri = d_ri; d.cv = d_cv;
  const size_t nb = (size_t)std::max(n, 1) * 8, mb = (size_t)std::max(m, 1) * 8;
  double *x = (double *)take(nb), *xt = (double *)take(nb), *x0 = (double *)take(nb),
         *kty = (double *)take(nb), *kty0 = (double *)take(nb), *xout = (double *)take(nb),
         *certx = (double *)take(nb), *c = (double *)take(nb), *l = (double *)take(nb),
         *u = (double *)take(nb), *E = (double *)take(nb), *Einv = (double *)take(nb),
         *tmp_n = (double *)take(nb), *certx2 = (double *)take(nb);
  unsigned char *act = (unsigned char *)take((size_t)std::max(n, 1));
  double *y = (double *)take(mb), *yt = (double *)take(mb), *y0 = (double *)take(mb),
         *kx = (double *)take(mb), *kxt = (double *)take(mb), *kx0 = (double *)take(mb),
         *certy = (double *)take(mb), *q = (double *)take(mb), *D = (double *)take(mb),
         *Dinv = (double *)take(mb), *tmp_m = (double *)take(mb), *certy2 = (double *)take(mb);
  rh::Ctl *ctl = b->d_ctls + slot;
  rh::IterConsts *ic = (rh::IterConsts *)take(sizeof(rh::IterConsts));
  double *setup_out = (double *)take(16);
  d.tmp_m = tmp_m;
  d.tmp_n = tmp_n;
  d.rv_ = rh::RowVecs{y, yt, y0, kx, kxt, kx0, certy, q, D, Dinv, certy2};
  d.cv_ = rh::ColVecs{x, xt, x0, kty, kty0, xout, certx, c, l, u, E, Einv, certx2, act};
  d.mixed = mixed ? 1 : 0;
  if (mixed) {
    // the FP64 anchors, their products, outputs and certificates are shared with the FP64 state
    const size_t nf = (size_t)std::max(n, 1) * 4, mf = (size_t)std::max(m, 1) * 4;
    d.rv32 = (float *)take(nnz * 4);
    d.cv32 = (float *)take(nnz * 4);
    float *fx[6], *fy[6];
    for (auto &f : fx) f = (float *)take(nf);
    for (auto &f : fy) f = (float *)take(mf);
    double *dxt64 = (double *)take(nb), *dyt64 = (double *)take(mb);
    d.rvm = rh::RowVecsMx{fy[0], fy[1], fy[2], fy[3], fy[4], fy[5], y0, kx0, certy, dyt64, q, D,
                          Dinv, certy2};
    d.cvm = rh::ColVecsMx{fx[0], fx[1], fx[2], fx[3], fx[4], fx[5], x0, kty0, xout, certx, dxt64,
                          c, l, u, E, Einv, certx2, act};
  }
  d.ctl = ctl;
  d.ic = ic;
  d.setup_out = setup_out;
  cudaStream_t st = b->st;
  cudaMemcpyAsync(d_rp, rp32.data(), (m + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
  if (nnz) {
    cudaMemcpyAsync(d_ci, ci.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_rv, lp->val, nnz * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_ri, ri.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_cv, cv.data(), nnz * 8, cudaMemcpyHostToDevice, st);
  }
  cudaMemcpyAsync(d_cp, cp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c, lp->c, n * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(l, lp->l, n * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(u, lp->u, n * 8, cudaMemcpyHostToDevice, st);
  if (m) cudaMemcpyAsync(q, lp->rhs, m * 8, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(certx, 0, nb, st);
  cudaMemsetAsync(certy, 0, mb, st);
  cudaMemsetAsync(certx2, 0, nb, st);
  cudaMemsetAsync(act, 0, (size_t)std::max(n, 1), st);
  cudaMemsetAsync(certy2, 0, mb, st);
  rh::Ctl c0{};
  c0.status = rh::kRunning;
  c0.stage = 2;                     // set-up pending
  c0.check_t = -1;
  rh::IterConsts ic0{};
  ic0.m = m; ic0.m_eq = lp->m_eq; ic0.n = n;
  ic0.rho2 = P.algorithm == 1 ? 1 : 0;
  ic0.max_iters = P.max_iters;
  ic0.check_every = P.check_every;
  ic0.first_epoch_len = P.first_epoch_len;
  ic0.max_epoch_len = P.max_epoch_len;
  ic0.restart_scheme = P.restart_scheme;
  ic0.pw_update = P.primal_weight_update;
  ic0.beta2 = P.restart_beta * P.restart_beta;
  ic0.eps_kkt = P.eps_rel_kkt;
  ic0.eps_infeas = P.eps_infeas;
  ic0.obj_offset = lp->obj_offset;
  ic0.trace_cap = 0;
  ic0.trace = nullptr;
  ic0.mixed = mixed ? 1 : 0;
  ic0.no_upper = any_upper ? 0 : 1;
  // the host copies must outlive the async copies: stage through a synchronisation
  cudaMemcpyAsync(ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(ic, &ic0, sizeof(ic0), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b->d_desc + slot, &d, sizeof(d), cudaMemcpyHostToDevice, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    arena_release(b, off, need);
    return berr(b, RHPDHG_ERR_CUDA, std::string("batch add: ") + cudaGetErrorString(e));
  }
  b->host_desc[slot] = d;
  b->slot_region[slot] = {off, need};
  b->slot_m[slot] = m;
  b->slot_n[slot] = n;
  b->slot_off[slot] = lp->obj_offset;
  b->slot_params[slot] = P;
  b->h_ctl[slot] = c0;
  *slot_out = slot;
  return RHPDHG_OK;
}

int rhpdhg_batch_step(rhpdhg_batch *b, int32_t iters) {
  if (!b || iters < 1) return RHPDHG_ERR_INVALID_ARG;
  if (b->graph_iters != iters) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return berr(b, RHPDHG_ERR_CUDA, cudaGetErrorString(e));
    rh::k_batch<<<b->max_slots, rh::kBT, 0, b->st>>>(b->d_desc, b->max_slots, iters);
    cudaMemcpyAsync(b->h_ctl, b->d_ctls, b->max_slots * sizeof(rh::Ctl), cudaMemcpyDeviceToHost,
                    b->st);
    e = cudaStreamEndCapture(b->st, &g);
    if (e != cudaSuccess) return berr(b, RHPDHG_ERR_CUDA, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return berr(b, RHPDHG_ERR_CUDA, cudaGetErrorString(e));
    b->graph_iters = iters;
  }
  // one launch advances every slot; the graph ends by copying all control blocks to the host
  cudaError_t e = cudaGraphLaunch(b->gexec, b->st);
  b->launches += 1;
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return berr(b, RHPDHG_ERR_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
  return RHPDHG_OK;
}

int rhpdhg_batch_poll(rhpdhg_batch *b, int32_t slot, rhpdhg_result *r) {
  if (!b || !r || slot < 0 || slot >= b->max_slots || !b->host_desc[slot].active)
    return RHPDHG_ERR_INVALID_ARG;
  const rh::Ctl &c = b->h_ctl[slot];
  if (c.status == rh::kRunning) return RHPDHG_BUSY;
  const rh::BatchDesc &d = b->host_desc[slot];
  r->status = c.status;
  r->iters = c.t;
  r->restarts = c.n;
  r->escalated = c.escalated;
  r->rel_p = c.rel_p;
  r->rel_d = c.rel_d;
  r->rel_gap = c.rel_gap;
  r->primal_obj = c.pobj;
  r->dual_obj = c.dobj;
  r->solve_seconds = 0.0;
  r->eta = c.eta;
  r->omega = c.omega;
  double so[2] = {0, 0};
  cudaMemcpyAsync(so, d.setup_out, 16, cudaMemcpyDeviceToHost, b->st);
  const int m = d.m, n = d.n;
  double *xo = nullptr, *yo = nullptr;
  cudaMalloc(&xo, (size_t)std::max(n, 1) * 8);
  cudaMalloc(&yo, (size_t)std::max(m, 1) * 8);
  rh::k_batch_unscale<<<4, 256, 0, b->st>>>(b->d_desc, slot, xo, yo);
  b->launches += 1;
  const cudaMemcpyKind kind =
      r->out_memory == RHPDHG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (r->x) cudaMemcpyAsync(r->x, xo, n * 8, kind, b->st);
  if (r->y && m) cudaMemcpyAsync(r->y, yo, m * 8, kind, b->st);
  const bool mv = c.cert_src == rh::kCertAnchorMove;
  r->cert_source = c.cert_src;
  if (r->cert_x) cudaMemcpyAsync(r->cert_x, mv ? d.cv_.certx2 : d.cv_.certx, n * 8, kind, b->st);
  if (r->cert_y && m)
    cudaMemcpyAsync(r->cert_y, mv ? d.rv_.certy2 : d.rv_.certy, m * 8, kind, b->st);
  cudaError_t e = cudaStreamSynchronize(b->st);
  cudaFree(xo);
  cudaFree(yo);
  r->sigma_max = so[0];
  if (e != cudaSuccess) return berr(b, RHPDHG_ERR_CUDA, cudaGetErrorString(e));
  return RHPDHG_OK;
}

int rhpdhg_batch_remove(rhpdhg_batch *b, int32_t slot) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->host_desc[slot].active)
    return RHPDHG_ERR_INVALID_ARG;
  rh::BatchDesc d{};
  d.active = 0;
  cudaMemcpyAsync(b->d_desc + slot, &d, sizeof(d), cudaMemcpyHostToDevice, b->st);
  cudaMemsetAsync(b->d_ctls + slot, 0, sizeof(rh::Ctl), b->st);
  cudaStreamSynchronize(b->st);
  arena_release(b, b->slot_region[slot].off, b->slot_region[slot].size);
  b->host_desc[slot] = d;
  b->slot_region[slot] = {0, 0};
  std::memset(&b->h_ctl[slot], 0, sizeof(rh::Ctl));
  return RHPDHG_OK;
}

int rhpdhg_batch_slot_status(const rhpdhg_batch *b, int32_t slot) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->host_desc[slot].active) return -1;
  return b->h_ctl[slot].status;
}

int64_t rhpdhg_batch_free_bytes(const rhpdhg_batch *b) {
  if (!b) return -1;
  size_t t = 0;
  for (auto &r : b->free_list) t += r.size;
  return (int64_t)t;
}

int64_t rhpdhg_batch_bytes_needed(const rhpdhg_problem *lp, int32_t precision) {
  if (!lp || (precision != 0 && precision != 1)) return -1;
  return (int64_t)slot_bytes(lp->m_eq + lp->m_ineq, lp->n, lp->nnz, precision == 1);
}

int64_t rhpdhg_batch_launch_count(const rhpdhg_batch *b) { return b ? b->launches : -1; }

void rhpdhg_batch_free(rhpdhg_batch *b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  cudaFree(b->arena);
  cudaFree(b->d_desc);
  cudaFree(b->d_ctls);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
  delete b;
}

}  // extern "C"
