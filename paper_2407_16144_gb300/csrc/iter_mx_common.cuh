// Per-row and per-column bodies of the mixed-precision iteration (FP32 offsets from FP64
// anchors; see iterate_mx.cu for the representation), shared by the tiled single-LP kernels and
// the CTA-resident batched kernel.  Each body handles one row of K^ (dual side) or one column
// (primal side) given its product from the SpMV; sums go to S (the caller's accumulator for the
// row), maxima to M, and the restart-norm sums of the ordinary bodies to F (FprSums).
#pragma once

#include "common.cuh"
#include "internal.h"
#include "iter_common.cuh"

namespace rh {

// Sums of the restart test's norms in the ordinary mixed iterations (||dy||^2, dy^T K dx,
// ||y~ - y0||^2; ||dx||^2, ||x~ - x0||^2), chosen per solve (IterConsts::df_sums, the DFS
// template argument), in the packed reduction slots of common.cuh:
//   DFS = 0: FP32 throughout: each lane sums its rows' FP32 products with FMA, and the warp, the
//            CTA and the grid add in FP32 with fixed trees (relative error of order 1e-6);
//   DFS = 1: double-float sums of exact products from the lane up: FP64-grade sums on the FP32
//            pipe, at the cost of longer dependent chains in the reductions.
template <int N, int DFS>
struct FprSums {
  DF v[N];
  __device__ __forceinline__ FprSums() {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = DF{0.f, 0.f};
  }
  __device__ __forceinline__ void add(int i, float a, float b) {
    if constexpr (DFS) v[i] = df_add(v[i], df_prod(a, b));
    else v[i].hi = __fmaf_rn(a, b, v[i].hi);
  }
  // into the packed slots of an accumulator (at the end of the walk, or for a long-row group
  // before its warp sum), then cleared
  template <class A>
  __device__ __forceinline__ void flush(A &acc) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      acc.d[i] = v[i];
      v[i] = DF{0.f, 0.f};
    }
  }
};

// ---- dual side (rows of K^) ------------------------------------------------------------------

// Restart with the anchor-movement test (move): row i's parts of z^{n+1,0} - z^{n,0}, with
// y0' = y0 + dyt and dot = (K x0')_i, against the old anchor, in FP64.
template <class AS, class AM>
__device__ __forceinline__ void row_mx_move(int i, double dot, const RowVecsMx &v, int m_eq,
                                            AS &S, AM &M) {
  const double y0i = v.y0[i];
  const double dyb = (y0i + (double)v.dyt[i]) - y0i;
  const double kdb = (dot - v.kx0[i]) * v.dinv[i];
  const double di = v.d[i];
  S.s[6] += v.q[i] * dyb;
  if (i >= m_eq) M.mx[3] = fmax(M.mx[3], fmax(-dyb * di, 0.0));
  if (i < m_eq) M.mx[4] = fmax(M.mx[4], fabs(kdb));
  else M.mx[5] = fmax(M.mx[5], fmax(-kdb, 0.0));
  v.certy2[i] = dyb * di;
}

// Restart point z^{n+1,0} = T(z^{n,k}), row i, in FP64: the new anchor y0' = y0 + dyt, its FP32
// images (r0, ylo), the dual step from the restart point with kd = (K dxt)_i (dxt exact in
// dxt64) and K x0' already in kx0, and the restart point's check and certificate parts.
template <int RHO2, class AS, class AM>
__device__ __forceinline__ void row_mx_restart(int i, double kd, const RowVecsMx &v, double sigma,
                                               int m_eq, bool check, bool rp, AS &A, AM &M) {
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
    if (i >= m_eq) M.mx[0] = fmax(M.mx[0], fmax(-nd * di, 0.0));
    const double kdd = kd * v.dinv[i];
    if (i < m_eq) M.mx[1] = fmax(M.mx[1], fabs(kdd));
    else M.mx[2] = fmax(M.mx[2], fmax(-kdd, 0.0));
    v.certy[i] = nd * di;
  }
}

// Ordinary iteration, row i, in FP32: the pending blend of the offsets (eq. hpdhg / eq. hrpdhg)
// and the dual step with kd = (K dxt)_i; FP64 check parts on check iterations.
template <int RHO2, class AS, class F>
__device__ __forceinline__ void row_mx_ordinary(int i, float kd, const RowVecsMx &v, float wf,
                                                float sigf, int m_eq, bool check, AS &A, F &Fs) {
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
  Fs.add(0, ddy, ddy);
  Fs.add(1, ddy, kdx - kd);
  Fs.add(2, nd, nd);
  if (check) {
    const double qi = v.q[i];
    double r = (qi - v.kx0[i] - (double)kd) * v.dinv[i];
    if (i >= m_eq) r = fmax(r, 0.0);
    A.s[3] += r * r;
    A.s[4] += qi * (v.y0[i] + (double)nd);
  }
}

// ---- primal side (columns of K^, rows of K^T) ---------------------------------------------------

// Checks and certificates at (x~_t, y~_t) of column j given x0j, x~_t - x0 (xo), K^T y~_t (kty)
// and K^T (y~_t - y_t) (ktd), all FP64: the dual residual, objective and bound terms on check
// iterations, and at restart points (rp) the column parts of T(z) - z.
template <class AS, class AM>
__device__ __forceinline__ void col_mx_checks(int j, double x0j, double xo, double kty,
                                              double ktd, const ColVecsMx &v, bool check,
                                              bool rp, AS &A, AM &M) {
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
  if (rp) col_cert_parts(j, xo, ktd, v, cj, lj, uj, A, M, 5, 0, v.certx);
}

// Restart z^{n+1,0} = T(z^{n,k}), column j, in FP64 with kty = (K^T y0')_j: the checks of the
// restart iteration, the anchor-movement parts against the old anchor (move), the new anchor
// x0' = x0 + dxt and its FP32 images (s0, xlo, xhi), and the next PDHG point x~_{t+1} - x0'
// (kept exactly in dxt64 for the restart point's certificate test).
template <int RHO2, class AS, class AM>
__device__ __forceinline__ void col_mx_restart(int j, double kty, const ColVecsMx &v, double tau,
                                               bool check, bool rp, bool move, AS &A, AM &M) {
  const double x0j = v.x0[j];
  const float dxtj = v.dxt[j];
  const double ktd = kty - v.kty0[j];
  col_mx_checks(j, x0j, (double)dxtj, kty, ktd, v, check, rp, A, M);
  const double x0n = x0j + (double)dxtj;
  if (move) col_cert_parts(j, x0n - x0j, ktd, v, v.c[j], v.l[j], v.u[j], A, M, 8, 4, v.certx2);
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
}

// First iteration of an epoch (restart point), column j, with ktd = (K^T (y~ - y0))_j in FP64
// from the exact dyt64: the checks at the restart point, then the blend and primal step in FP32.
// no_upper: every u is +inf, so the upper-bound offset (+inf) is not read.
template <int RHO2, class AS, class AM>
__device__ __forceinline__ void col_mx_first(int j, double ktd, const ColVecsMx &v, float wf,
                                             float tauf, bool check, bool rp, bool no_upper,
                                             AS &A, AM &M) {
  const double xo = v.dxt64[j];
  const double x0j = check ? v.x0[j] : 0.0;
  const double kty = check ? v.kty0[j] + ktd : 0.0;
  col_mx_checks(j, x0j, xo, kty, ktd, v, check, rp, A, M);
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
  const float hi = no_upper ? INFINITY : v.xhi[j];
  const float nt = fminf(fmaxf(dxn + v.s0[j] + tauf * ktn, v.xlo[j]), hi);
  v.dxt[j] = nt;
  const float ddx = dxn - nt;
  A.s[0] += (double)ddx * (double)ddx;
  A.s[1] += (double)nt * (double)nt;
}

// Ordinary iteration, column j, in FP32 with ktdyt = (K^T dyt)_j: checks and active-set
// telemetry on check iterations, then the pending blend and the primal step of eq. pdhg.
// no_upper: every u is +inf, so the upper-bound offset (+inf) is not read.
template <int RHO2, class AS, class AM, class F>
__device__ __forceinline__ void col_mx_ordinary(int j, float ktdyt, const ColVecsMx &v, float wf,
                                                float tauf, bool check, bool no_upper, AS &A,
                                                AM &M, F &Fs, Tel &tl) {
  const float dxtj = v.dxt[j];
  const float hi = no_upper ? INFINITY : v.xhi[j];
  if (check) {
    tel_column(j, dxtj == v.xlo[j] || dxtj == hi, v.act, tl);
    const double x0j = v.x0[j];
    col_mx_checks(j, x0j, (double)dxtj, v.kty0[j] + (double)ktdyt, (double)ktdyt, v, check,
                  false, A, M);
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
  const float nt = fminf(fmaxf(dxn + v.s0[j] + tauf * ktn, v.xlo[j]), hi);
  v.dxt[j] = nt;
  const float ddx = dxn - nt;
  Fs.add(0, ddx, ddx);
  Fs.add(1, nt, nt);
}

}  // namespace rh
