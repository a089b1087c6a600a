// C ABI (include/rhpdhg.h): problem upload and preprocessing, the host driver of the device
// iteration (CUDA-graph replays of C iterations, two in flight), polling and inspection.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rhpdhg.h"
#include "bufcache.h"
#include "plan.h"
#include "internal.h"

using namespace rh;

namespace {

thread_local std::string g_create_error;

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double s() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

}  // namespace

namespace rh {
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace rh

struct rhpdhg_handle {
  int dev = 0;
  int sm_count = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int m = 0, m_eq = 0, m_ineq = 0, n = 0;
  long long nnz = 0;
  double obj_offset = 0.0;
  rhpdhg_params p{};
  std::vector<double> h_x0, h_y0;

  SideStore rows, cols;
  double *D = nullptr, *E = nullptr, *Dinv = nullptr, *Einv = nullptr;
  double *c = nullptr, *q = nullptr, *l = nullptr, *u = nullptr;
  double *x = nullptr, *xt = nullptr, *x0 = nullptr, *kty = nullptr, *kty0 = nullptr,
         *xout = nullptr, *certx = nullptr, *certx2 = nullptr;
  double *y = nullptr, *yt = nullptr, *y0 = nullptr, *kx = nullptr, *kxt = nullptr,
         *kx0 = nullptr, *certy = nullptr, *certy2 = nullptr;
  double *x_init = nullptr, *y_init = nullptr, *xres = nullptr, *yres = nullptr;
  unsigned char *act = nullptr;   // on-bound flags of the previous check (telemetry)
  // mixed precision: FP32 offsets and anchor images
  bool mixed = false;
  float *dxt = nullptr, *dx = nullptr, *ktdy = nullptr, *s0 = nullptr, *xlo = nullptr,
        *xhi = nullptr;
  float *dyt = nullptr, *kdxt = nullptr, *dy = nullptr, *kdx = nullptr, *r0 = nullptr,
        *ylo = nullptr;
  double *dxt64 = nullptr, *dyt64 = nullptr;
  RowVecsMx rvm{};
  ColVecsMx cvm{};
  Ctl *ctl = nullptr;
  Ctl *h_mirror = nullptr;   // two pinned host mirrors of the control block
  double *part_row = nullptr, *part_col = nullptr;
  TraceRec *trace = nullptr;
  IterConsts ic{};
  RowVecs rv{};
  ColVecs cv{};
  int grid_row = 1, grid_col = 1, smem_row = 0, smem_col = 0;
  int grid_row1 = 1, grid_col1 = 1;   // restart-mode mixed kernels: at most one resident wave
  int col_rows_last = 1;              // CTA rows the last column launch wrote (see DeferredCol)
  double eta = 1.0, omega0 = 1.0, sigma_max = 0.0;

  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  std::thread th;
  std::atomic<int> running{0};
  std::atomic<int> cancel{0};
  bool solved = false;
  int final_status = 0;
  double solve_seconds = 0.0;
  long long final_iters = 0;
  Ctl final_ctl{};
  std::string err;
  int drive_err = 0;

  double ms_row = 0, ms_col = 0;
  long long n_row = 0, n_col = 0;
  long long launches = 0;      // kernels launched by create and solves
  bool escalated = false;      // this solve switched from mixed precision to FP64
  bool created_mixed = false;  // precision requested at create
  double bytes_row = 0, bytes_col = 0;
  // autotuner: structure signature, outcome (0 = rule, 1 = timed at create, 2 = taken from the
  // cache of an earlier handle with the same signature), and the per-iteration times (us) of
  // the rule's geometry and of the chosen one
  std::string tune_sig;
  int tuned = 0;
  double tune_us_rule = 0.0, tune_us_best = 0.0;
};

namespace {

int set_err(rhpdhg_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      return set_err(h, e_ == cudaErrorMemoryAllocation ? RHPDHG_ERR_OOM : RHPDHG_ERR_CUDA, \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    }                                                                                     \
  } while (0)

// Device buffers of a handle come from the buffer cache (buf_alloc); each is released only after
// the handle's stream has been synchronised.
template <typename T>
cudaError_t dalloc(T **p, size_t count) {
  return buf_alloc((void **)p, (count > 0 ? count : 1) * sizeof(T));
}

void destroy(rhpdhg_handle *h) {
  if (!h) return;
  if (h->th.joinable()) h->th.join();
  if (h->st) cudaStreamSynchronize(h->st);
  for (auto &g : h->gexec)
    if (g) cudaGraphExecDestroy(g);
  free_side(&h->rows);
  free_side(&h->cols);
  double *bufs[] = {h->D, h->E, h->Dinv, h->Einv, h->c, h->q, h->l, h->u, h->x, h->xt, h->x0,
                    h->kty, h->kty0, h->xout, h->certx, h->y, h->yt, h->y0, h->kx, h->kxt,
                    h->kx0, h->certy, h->x_init, h->y_init, h->xres, h->yres, h->part_row,
                    h->part_col, h->dxt64, h->dyt64, h->certx2, h->certy2};
  for (double *b : bufs) buf_release(b);
  float *fbufs[] = {h->dxt, h->dx, h->ktdy, h->s0, h->xlo, h->xhi,
                    h->dyt, h->kdxt, h->dy, h->kdx, h->r0, h->ylo};
  for (float *b : fbufs) buf_release(b);
  buf_release(h->act);
  buf_release(h->ctl);
  buf_release(h->trace);
  if (h->h_mirror) cudaFreeHost(h->h_mirror);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  delete h;
}

// Algorithmic bytes one launch of each iteration kernel moves (FP64, reflected or not): the
// side's values and indices, row pointers, the gathered vector once, and the streamed vectors.
void algorithmic_bytes(rhpdhg_handle *h) {
  const double ib = 4.0;
  const int rho2 = h->ic.rho2;
  const double nnz = (double)h->nnz;
  if (h->mixed) {
    // FP32 values; row kernel reads dyt, kdxt, r0, ylo (+ dy, kdx), writes dyt, kdxt (+ dy, kdx),
    // gathers dxt; column kernel reads dxt, s0, xlo, xhi (not when every u is +inf) (+ dx, ktdy),
    // writes dxt (+ dx, ktdy), gathers dyt.  (Restart iterations add the FP64 anchor products;
    // not counted here.)
    const double fb = 4.0, vb = h->ic.bf16 ? 2.0 : 4.0;   // offsets FP32; values FP32 or BF16
    h->bytes_row = nnz * (vb + ib) + (h->m + 1) * ib + h->n * fb +
                   h->m * fb * ((4 + 2 * rho2) + (2 + 2 * rho2));
    h->bytes_col = nnz * (vb + ib) + (h->n + 1) * ib + h->m * fb +
                   h->n * fb * ((4 + 2 * rho2 - h->ic.no_upper) + (1 + 2 * rho2));
    return;
  }
  const double vb = 8.0;
  // row kernel: reads y~, y0, Kx~, Kx0, q (+ y, Kx for rho=2), writes y~, Kx~ (+ y, Kx)
  const double row_vec = (5 + 2 * rho2) + (2 + 2 * rho2);
  h->bytes_row = nnz * (vb + ib) + (h->m + 1) * ib + h->n * vb + h->m * vb * row_vec;
  // column kernel: reads x~, x0, K^Ty0, c, l, u (+ x, K^Ty), writes x~ (+ x, K^Ty)
  const double col_vec = (6 + 2 * rho2) + (1 + 2 * rho2);
  h->bytes_col = nnz * (vb + ib) + (h->n + 1) * ib + h->m * vb + h->n * vb * col_vec;
}

// Launch shape of one side's iteration kernels: warps per CTA, short tiles per work item (0 = the
// layout rule's), the ordinary mixed row kernel's wide staging round (1 = on, 0 = off, -1 = the
// rule below), and the grid as a percentage of the resident CTAs (100 = all).
struct SideShape {
  int warps = kBlockWarps;
  int mult = 0;
  int wide = -1;
  int cap = 100;
};

// Launch geometry of the iteration kernels for the row-side shape r and the column-side shape c:
// tiles per work item, dynamic shared memory for each warp's staging area, the walk
// instantiation of the ordinary mixed kernels, and grids of one work item per warp within the
// resident CTAs (times the shape's cap).
void set_geometry(rhpdhg_handle *h, const SideShape &r, const SideShape &c) {
  apply_mult(h->rows, r.mult > 0 && mult_ok(h->rows, r.mult) ? r.mult : h->rows.rule_mult);
  apply_mult(h->cols, c.mult > 0 && mult_ok(h->cols, c.mult) ? c.mult : h->cols.rule_mult);
  SideLayout &lr = h->rows.lay, &lc = h->cols.lay;
  const int wr = r.warps, wc = c.warps;
  lr.cta_warps = wr;
  lc.cta_warps = wc;
  h->smem_row = wr * lr.seg * (int)sizeof(double);
  h->smem_col = wc * lc.seg * (int)sizeof(double);
  auto capped = [](int b, int cap) { return std::max(1, b * cap / 100); };
  if (h->mixed) {
    lr.walk = lr.tile_mult > 1 ? kWalkGrouped : kWalkPlain;
    lc.walk = lc.tile_mult > 1 ? kWalkGrouped : kWalkPlain;
    // The row kernels stage twice as many groups per round (fewer dependent rounds, more
    // registers) when their tiles are long and the grid stays set by the tile count at the
    // wider kernel's residency, so that the registers cost no CTAs.
    if (lr.walk == kWalkPlain && lr.n_short_tiles > 0) {
      bool wide = r.wide == 1;
      if (r.wide < 0 &&
          h->rows.nnz_short > (long long)lr.n_short_tiles * kWarp * kStageUnroll * 4) {
        const int bw =
            iter_mx_blocks_per_sm(h->smem_row, true, kWalkWide, wr * kWarp, h->ic.df_sums,
                                  h->ic.bf16);
        const long long need = ((long long)lr.total_items() + wr - 1) / wr;
        wide = bw > 0 && need <= (long long)bw * h->sm_count;
      }
      if (wide) lr.walk = kWalkWide;
    }
    h->grid_row = tile_grid(lr, h->sm_count,
                            capped(iter_mx_blocks_per_sm(h->smem_row, true, lr.walk, wr * kWarp,
                                                         h->ic.df_sums, h->ic.bf16),
                                   r.cap));
    h->grid_col = tile_grid(lc, h->sm_count,
                            capped(iter_mx_blocks_per_sm(h->smem_col, false, lc.walk, wc * kWarp,
                                                         h->ic.df_sums, h->ic.bf16),
                                   c.cap));
    const int br = iter_mx_restart_blocks_per_sm(h->smem_row, true, wr * kWarp);
    const int bc = iter_mx_restart_blocks_per_sm(h->smem_col, false, wc * kWarp);
    h->grid_row1 = std::max(1, std::min(h->grid_row, h->sm_count * std::max(br, 1)));
    h->grid_col1 = std::max(1, std::min(h->grid_col, h->sm_count * std::max(bc, 1)));
  } else {
    h->grid_row = tile_grid(lr, h->sm_count,
                            capped(row_iter_blocks_per_sm(h->smem_row, wr * kWarp), r.cap));
    h->grid_col = tile_grid(lc, h->sm_count,
                            capped(col_iter_blocks_per_sm(h->smem_col, wc * kWarp), c.cap));
  }
}

// The shape set_geometry applied last, as a candidate (wide as resolved by the rule).
SideShape current_shape(const rhpdhg_handle *h, bool row) {
  const SideLayout &l = row ? h->rows.lay : h->cols.lay;
  SideShape s;
  s.warps = l.cta_warps;
  s.mult = l.tile_mult;
  s.wide = (row && l.walk == kWalkWide) ? 1 : 0;
  s.cap = 100;
  return s;
}

void launch_row(rhpdhg_handle *h) {
  // the column stage that precedes this row stage, for the case that it deferred its reduction:
  // an ordinary column launch (grid_col CTAs; the mixed ordinary kernel's long-row groups use
  // the second walk scratch, the FP64 kernel's the first)
  DeferredCol dc;
  dc.part = h->part_col;
  dc.gpart = h->mixed ? h->cols.wb.group_part : h->cols.wa.group_part;
  dc.nb = h->col_rows_last;   // the column launch before this one (the autotuner varies grids)
  dc.ngroups = h->cols.lay.n_long_tiles;
  if (h->mixed)
    launch_row_iter_mx(h->st, h->rows, h->rvm, h->dxt, h->dxt64, h->x0, h->ctl, h->part_row,
                       h->ic, h->grid_row, h->grid_row1, h->smem_row, dc);
  else
    launch_row_iter(h->st, h->rows, h->xt, h->rv, h->ctl, h->part_row, h->ic, h->grid_row,
                    h->smem_row, dc);
}

void launch_col(rhpdhg_handle *h, int phase) {
  h->col_rows_last = h->grid_col;   // a deferring (ordinary) column launch has grid_col CTAs
  if (h->mixed)
    launch_col_iter_mx(h->st, h->cols, h->cvm, h->dyt, h->dyt64, h->y0, h->ctl, h->part_col,
                       h->ic, h->grid_col, h->grid_col1, h->smem_col, phase);
  else
    launch_col_iter(h->st, h->cols, h->yt, h->cv, h->ctl, h->part_col, h->ic, h->grid_col,
                    h->smem_col, phase);
}

void launch_iteration(rhpdhg_handle *h) {
  launch_row(h);
  launch_col(h, 0);
}

// Iterations per host chunk (one captured graph, one read of the control block): the check
// cadence, at most kMaxChunk, so that a large check_every does not make a graph of that many
// launches (the device makes every decision; the host only polls between chunks).
constexpr int kMaxChunk = 256;
int chunk_iters(const rhpdhg_handle *h) { return std::min(h->p.check_every, kMaxChunk); }

int capture_graphs(rhpdhg_handle *h) {
  for (int g = 0; g < 2; ++g) {
    if (h->gexec[g]) continue;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk_iters(h); ++i) launch_iteration(h);
    cudaMemcpyAsync(h->h_mirror + g, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st);
    CK(cudaStreamEndCapture(h->st, &graph));
    cudaError_t e = cudaGraphInstantiate(&h->gexec[g], graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
  }
  return RHPDHG_OK;
}

int reset_state(rhpdhg_handle *h) {
  Ctl c{};
  c.t = 0; c.k = 0; c.n = 0; c.k_next = 0; c.n_next = 0;
  c.status = kRunning;
  c.restart_pending = 1;
  c.stage = 1;           // the set-up column kernel runs first
  c.w = 0.0;
  c.omega = h->omega0;
  set_steps(&c, h->eta, h->omega0);
  c.eta = h->eta;
  CK(cudaMemcpyAsync(h->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemsetAsync(h->act, 0, (size_t)std::max(h->n, 1), h->st));
  if (h->mixed) {
    // anchors z^{0,0}, zero offsets; the set-up column kernel runs in restart mode and forms
    // K^T y0, the anchor images and dxt_0; the first row kernel forms K x0 likewise
    CK(cudaMemcpyAsync(h->x0, h->x_init, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (h->m > 0)
      CK(cudaMemcpyAsync(h->y0, h->y_init, h->m * sizeof(double), cudaMemcpyDeviceToDevice,
                         h->st));
    float *zn[] = {h->dxt, h->dx, h->ktdy};
    for (float *z : zn) zero_f32(h->st, h->n, z);
    float *zm[] = {h->dyt, h->kdxt, h->dy, h->kdx};
    for (float *z : zm) zero_f32(h->st, h->m, z);
    launch_col(h, 1);
    return RHPDHG_OK;
  }
  CK(cudaMemcpyAsync(h->xt, h->x_init, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  if (h->m > 0)
    CK(cudaMemcpyAsync(h->yt, h->y_init, h->m * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  // K x^{0,0} into the PDHG-point product slot; the first row kernel takes it as K x_0
  side_spmv(h->st, h->rows, h->x_init, h->kxt, h->grid_row);
  // the column kernel in set-up phase forms x_0 = x^{0,0}, K^T y_0 and x~_0
  launch_col(h, 1);
  CK(cudaGetLastError());
  return RHPDHG_OK;
}

// Mixed precision -> FP64 for the rest of the solve, from the current restart point (the FP64
// anchor z^{n,0}): the FP64 state is set up as at the start of a solve with that point as the
// initial point, and the iteration and epoch counters, the primal weight and the step carry on.
int escalate_to_fp64(rhpdhg_handle *h) {
  Ctl c{};
  CK(cudaMemcpy(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  h->mixed = false;
  h->ic.mixed = 0;
  for (auto &g : h->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  CK(cudaMemcpyAsync(h->xt, h->x0, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  if (h->m)
    CK(cudaMemcpyAsync(h->yt, h->y0, h->m * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  c.status = kRunning;
  c.restart_pending = 1;
  c.stage = 1;
  c.k = 0;
  c.k_next = 0;
  c.n_next = c.n;
  c.cnt_row = c.cnt_col = 0;
  c.mv_ready = 0;
  c.col_deferred = 0;
  c.escalated = 1;
  CK(cudaMemcpyAsync(h->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->st));
  side_spmv(h->st, h->rows, h->xt, h->kxt, h->grid_row);
  launch_col(h, 1);
  h->launches += 2;
  CK(cudaStreamSynchronize(h->st));
  CK(cudaGetLastError());
  h->escalated = true;
  return RHPDHG_OK;
}

// ---- autotuner ------------------------------------------------------------------------------
// The launch geometry of the iteration kernels (warps per CTA of each side; for the mixed row
// kernel also the plain or the wide staging walk) is chosen by timing candidates on the
// handle's own stream: the solve's iteration kernels run on its state, every candidate
// interleaved with the others, and each side keeps the candidate with the smallest median time
// per launch.  The choice is cached for the process by a signature of the LP's structure, so
// later handles of the same shape take it without timing.

struct TuneChoice {
  SideShape r, c;
  double us_rule = 0.0, us_best = 0.0;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;

// Candidate shapes of one side: 4- or 8-warp CTAs; 1, 2 or 4 tiles per work item where the
// group fits the staging area; on the mixed row side with one tile per item, the plain or the
// wide staging walk; the full resident grid or three quarters of it.
std::vector<SideShape> side_candidates(const rhpdhg_handle *h, bool row) {
  const SideStore &sd = row ? h->rows : h->cols;
  std::vector<SideShape> c;
  for (int w : {4, 8})
    for (int m : {1, 2, 4}) {
      if (!mult_ok(sd, m)) continue;
      const bool can_widen = row && h->mixed && m == 1 && sd.lay.n_short_tiles > 0;
      for (int wide = 0; wide <= (can_widen ? 1 : 0); ++wide)
        for (int cap : {100, 75}) c.push_back(SideShape{w, m, wide, cap});
    }
  return c;
}

bool same_shape(const SideShape &a, const SideShape &b) {
  return a.warps == b.warps && a.mult == b.mult && a.wide == b.wide && a.cap == b.cap;
}

// Largest grid of each side over all candidates (the partial buffers are sized for it).
void candidate_grids(rhpdhg_handle *h, int *max_row, int *max_col) {
  const SideShape r0 = current_shape(h, true), c0 = current_shape(h, false);
  *max_row = h->grid_row;
  *max_col = h->grid_col;
  const std::vector<SideShape> rs = side_candidates(h, true), cs = side_candidates(h, false);
  const size_t k = std::max(rs.size(), cs.size());
  for (size_t i = 0; i < k; ++i) {
    set_geometry(h, rs[i % rs.size()], cs[i % cs.size()]);
    *max_row = std::max(*max_row, h->grid_row);
    *max_col = std::max(*max_col, h->grid_col);
  }
  set_geometry(h, r0, c0);
}

// Signature of the LP's structure for the cache: precision, algorithm, sum mode, sizes, SM
// count, and the histograms (log2 buckets) of the row lengths of K and of K^T.
std::string shape_signature(const rhpdhg_handle *h, const std::vector<int> &rp,
                            const std::vector<int> &cp) {
  std::string sig = std::to_string(h->mixed + h->ic.bf16) + "/" + std::to_string(h->ic.rho2) + "/" +
                    std::to_string(h->ic.df_sums) + "/" + std::to_string(h->m_eq) + "/" +
                    std::to_string(h->m_ineq) + "/" + std::to_string(h->n) + "/" +
                    std::to_string(h->nnz) + "/" + std::to_string(h->sm_count);
  for (const std::vector<int> *v : {&rp, &cp}) {
    long long hist[33] = {0};
    for (size_t i = 0; i + 1 < v->size(); ++i) {
      const int len = (*v)[i + 1] - (*v)[i];
      int b = 0;
      while (b < 32 && (1 << b) <= len) ++b;
      hist[b]++;
    }
    sig += "|";
    for (long long c : hist) sig += std::to_string(c) + ",";
  }
  return sig;
}

double median(std::vector<float> v) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  return 0.5 * (v[(v.size() - 1) / 2] + v[v.size() / 2]);
}

// Times the candidates (see above) and applies the fastest.  The state the timing leaves
// behind is discarded: every solve starts with reset_state.
int autotune(rhpdhg_handle *h) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(h->tune_sig);
    if (it != g_tune_cache.end()) {
      set_geometry(h, it->second.r, it->second.c);
      h->tuned = 2;
      h->tune_us_rule = it->second.us_rule;
      h->tune_us_best = it->second.us_best;
      return RHPDHG_OK;
    }
  }
  const std::vector<SideShape> rows = side_candidates(h, true), cols = side_candidates(h, false);
  const int nr = (int)rows.size(), nc = (int)cols.size();
  const SideShape rule_r = current_shape(h, true), rule_c = current_shape(h, false);
  // ordinary iterations only: no check, no restart, no trace while timing
  const IterConsts saved = h->ic;
  h->ic.check_every = INT_MAX;
  h->ic.max_iters = LLONG_MAX / 4;
  h->ic.restart_scheme = 0;
  h->ic.first_epoch_len = INT_MAX / 2;
  h->ic.max_epoch_len = 0;
  h->ic.trace_cap = 0;
  int rc = reset_state(h);
  // iteration i runs row candidate i mod nr and column candidate i mod nc; each stage is timed
  // on its own, so every candidate of either side gets at least `reps` samples
  const int warm = 2, reps = 3;
  const int K = warm + reps * std::max(nr, nc);
  std::vector<cudaEvent_t> ev(3 * K);
  for (auto &e : ev) cudaEventCreate(&e);
  for (int i = 0; i < K && rc == RHPDHG_OK; ++i) {
    set_geometry(h, rows[i % nr], cols[i % nc]);
    cudaEventRecord(ev[3 * i], h->st);
    launch_row(h);
    cudaEventRecord(ev[3 * i + 1], h->st);
    launch_col(h, 0);
    cudaEventRecord(ev[3 * i + 2], h->st);
  }
  h->launches += (h->mixed ? 8 : 2) + (long long)K * (h->mixed ? 4 : 2);
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  std::vector<std::vector<float>> tr(nr), tc(nc);
  for (int i = warm; i < K && e == cudaSuccess; ++i) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]);
    cudaEventElapsedTime(&b, ev[3 * i + 1], ev[3 * i + 2]);
    tr[i % nr].push_back(a);
    tc[i % nc].push_back(b);
  }
  for (auto &ev_ : ev) cudaEventDestroy(ev_);
  h->ic = saved;
  if (rc != RHPDHG_OK) return rc;
  if (e != cudaSuccess)
    return set_err(h, RHPDHG_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  int br = 0, bc = 0, ir = -1, icr = -1;
  for (int i = 0; i < nr; ++i) {
    if (median(tr[i]) < median(tr[br])) br = i;
    if (same_shape(rows[i], rule_r)) ir = i;
  }
  for (int i = 0; i < nc; ++i) {
    if (median(tc[i]) < median(tc[bc])) bc = i;
    if (same_shape(cols[i], rule_c)) icr = i;
  }
  TuneChoice ch;
  ch.r = rows[br];
  ch.c = cols[bc];
  // the rule's shape is a candidate whenever the CTA width is 4 or 8 (the default is 4)
  ch.us_rule = 1e3 * ((ir >= 0 ? median(tr[ir]) : 0.0) + (icr >= 0 ? median(tc[icr]) : 0.0));
  ch.us_best = 1e3 * (median(tr[br]) + median(tc[bc]));
  set_geometry(h, ch.r, ch.c);
  h->tuned = 1;
  h->tune_us_rule = ch.us_rule;
  h->tune_us_best = ch.us_best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[h->tune_sig] = ch;
  return RHPDHG_OK;
}

// Runs the solve to completion (in the caller's thread or the handle's thread).
void drive(rhpdhg_handle *h) {
  cudaSetDevice(h->dev);
  Timer timer;
  if (h->created_mixed && !h->mixed) {      // a previous solve escalated: back to mixed
    h->mixed = true;
    h->ic.mixed = 1;
    for (auto &g : h->gexec)
      if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  }
  h->escalated = false;
  int rc = reset_state(h);
  h->launches += h->mixed ? 8 : 2;   // set-up kernels of the solve
  const bool graphs = h->p.use_graphs && !h->p.profile;
  if (rc == RHPDHG_OK && graphs) rc = capture_graphs(h);
  if (rc != RHPDHG_OK) {
    h->drive_err = rc;
    h->final_status = kNumericalError;
    h->running = 0;
    return;
  }
  cudaEvent_t ev[2];
  cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  std::vector<cudaEvent_t> pev;
  const int chunk = chunk_iters(h);
  if (h->p.profile) {
    pev.resize(3 * chunk);
    for (auto &e : pev) cudaEventCreate(&e);
  }
  h->ms_row = h->ms_col = 0.0;
  h->n_row = h->n_col = 0;
  // Up to two chunks of C iterations in flight (one while profiling, so the per-launch events
  // of a chunk can be read back).  Each chunk ends with a copy of the control block into its
  // own pinned mirror; the host reads mirror g only after chunk g's event, and relaunches g
  // only after that read.
  const long long depth = h->p.profile ? 1 : 2;
  long long last_t = 0;
  int host_status = kRunning;
  for (;;) {
    long long launched = 0, done = 0;
    bool stop = false;
    int dev_status = kRunning;
    while (true) {
      while (!stop && launched - done < depth) {
        if (h->cancel.load()) { host_status = kCancelled; stop = true; break; }
        if (timer.s() > h->p.time_limit_s) { host_status = kTimeLimit; stop = true; break; }
        const int g = (int)(launched & 1);
        if (graphs) {
          cudaGraphLaunch(h->gexec[g], h->st);
        } else {
          for (int i = 0; i < chunk; ++i) {
            if (h->p.profile) cudaEventRecord(pev[3 * i], h->st);
            launch_row(h);
            if (h->p.profile) cudaEventRecord(pev[3 * i + 1], h->st);
            launch_col(h, 0);
            if (h->p.profile) cudaEventRecord(pev[3 * i + 2], h->st);
          }
          cudaMemcpyAsync(h->h_mirror + g, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st);
        }
        cudaEventRecord(ev[g], h->st);
        ++launched;
        h->launches += (h->mixed ? 4LL : 2LL) * chunk;
      }
      if (done >= launched) break;
      const int g = (int)(done & 1);
      cudaError_t e = cudaEventSynchronize(ev[g]);
      ++done;
      if (e != cudaSuccess) {
        h->drive_err = RHPDHG_ERR_CUDA;
        h->err = std::string("solve: ") + cudaGetErrorString(e);
        stop = true;
        continue;
      }
      const Ctl &mc = h->h_mirror[g];
      if (h->p.profile) {
        // count only the launches that did work (the rest returned at entry)
        long long ran = mc.t - last_t;
        if (mc.status == kNumericalError) ran += 1;
        last_t = mc.t;
        for (long long i = 0; i < ran && i < chunk; ++i) {
          float a = 0, b = 0;
          cudaEventElapsedTime(&a, pev[3 * i], pev[3 * i + 1]);
          cudaEventElapsedTime(&b, pev[3 * i + 1], pev[3 * i + 2]);
          h->ms_row += a;
          h->ms_col += b;
          h->n_row++;
          h->n_col++;
        }
      }
      if (mc.status != kRunning) {
        stop = true;
        dev_status = mc.status;
      }
    }
    cudaStreamSynchronize(h->st);
    if (dev_status == kEscalate && host_status == kRunning && !h->drive_err) {
      if (escalate_to_fp64(h) == RHPDHG_OK && (!graphs || capture_graphs(h) == RHPDHG_OK)) {
        Ctl c{};
        cudaMemcpy(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
        last_t = c.t;
        continue;
      }
      h->drive_err = RHPDHG_ERR_CUDA;
    }
    break;
  }
  cudaStreamSynchronize(h->st);
  Ctl fin{};
  cudaMemcpy(&fin, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
  h->final_ctl = fin;
  h->final_status = fin.status != kRunning ? fin.status : host_status;
  if (h->final_status == kRunning || h->final_status == kEscalate)
    h->final_status = kNumericalError;
  if (h->mixed)
    launch_unscale_mx(h->st, h->n, h->m, h->E, h->xout, h->D, h->y0, h->dyt, h->xres, h->yres,
                      h->yt);
  else
    launch_unscale(h->st, h->n, h->m, h->E, h->xout, h->D, h->yt, h->xres, h->yres);
  h->launches += 1;
  // time / cancel stops happen at a chunk boundary, right after a check iteration, so xout
  // and y~ hold the PDHG point of that check
  cudaStreamSynchronize(h->st);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess && !h->drive_err) {
    h->drive_err = RHPDHG_ERR_CUDA;
    h->err = std::string("solve: ") + cudaGetErrorString(le);
  }
  h->solve_seconds = timer.s();
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  for (auto &e : pev) cudaEventDestroy(e);
  h->solved = true;
  h->running = 0;
}

}  // namespace

extern "C" {

int rhpdhg_params_default(rhpdhg_params *p) {
  if (!p) return RHPDHG_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->algorithm = 1;
  p->precision = 0;
  p->eps_rel_kkt = 1e-4;
  p->eps_infeas = 1e-8;
  p->max_iters = 10000000;
  p->time_limit_s = 3600.0;
  p->ruiz_iters = 10;
  p->pock_chambolle_alpha = 1.0;
  p->step_size = 0.0;
  p->step_safety = 0.9;
  p->power_iters = 100;
  p->primal_weight = 0.0;
  p->primal_weight_update = 1;
  p->first_epoch_len = 64;
  p->max_epoch_len = 1000;
  p->restart_scheme = 0;
  p->restart_beta = std::exp(-1.0);
  p->check_every = 64;
  p->use_graphs = 1;
  p->trace = 0;
  p->profile = 0;
  p->trace_capacity = 4096;
  p->adaptive_step = 0;
  p->x0 = nullptr;
  p->y0 = nullptr;
  return RHPDHG_OK;
}

const char *rhpdhg_last_error(const rhpdhg_handle *h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

int rhpdhg_create(const rhpdhg_problem *lp, const rhpdhg_params *params, void *cuda_stream,
                  rhpdhg_handle **out) {
  rhpdhg_handle *h = nullptr;
  if (!out) return set_err(nullptr, RHPDHG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!lp || !params) return set_err(nullptr, RHPDHG_ERR_INVALID_ARG, "lp or params is NULL");
  const rhpdhg_params &P = *params;
  if (lp->m_eq < 0 || lp->m_ineq < 0 || lp->n < 1 || lp->nnz < 0)
    return set_err(nullptr, RHPDHG_ERR_INVALID_ARG, "negative size or n < 1");
  if ((long long)lp->m_eq + lp->m_ineq > INT_MAX - 1 || lp->nnz > INT_MAX - 1)
    return set_err(nullptr, RHPDHG_ERR_INVALID_ARG, "m or nnz exceeds the 32-bit index range");
  if (lp->memory != RHPDHG_MEM_HOST && lp->memory != RHPDHG_MEM_DEVICE)
    return set_err(nullptr, RHPDHG_ERR_INVALID_ARG, "unknown memory kind");
  const int m = lp->m_eq + lp->m_ineq;
  if (!lp->row_ptr || !lp->c || !lp->l || !lp->u || (m > 0 && !lp->rhs) ||
      (lp->nnz > 0 && (!lp->col_idx || !lp->val)))
    return set_err(nullptr, RHPDHG_ERR_INVALID_ARG, "missing problem array");
  if (P.algorithm < 0 || P.algorithm > 1 || P.precision < 0 || P.precision > 2 || P.check_every < 1 ||
      P.max_iters < 1 || !(P.eps_rel_kkt > 0) || !(P.eps_infeas > 0) || P.ruiz_iters < 0 ||
      P.power_iters < 1 || P.step_size < 0 || !(P.step_safety > 0) || P.primal_weight < 0 ||
      P.first_epoch_len < 0 || P.max_epoch_len < 0 || P.restart_scheme < 0 ||
      P.restart_scheme > 2 || (P.restart_scheme >= 1 && P.max_epoch_len < 1) ||
      !(P.restart_beta > 0 && P.restart_beta < 1) || P.trace_capacity < 0 ||
      P.pock_chambolle_alpha > 2.0 || P.adaptive_step < 0 || P.adaptive_step > 1 ||
      (P.cta_warps != 0 && P.cta_warps != 4 && P.cta_warps != 8 && P.cta_warps != 16) ||
      P.df_sums < 0 || P.df_sums > 1 || P.autotune < 0 || P.autotune > 1 ||
      P.pow2_scaling < 0 || P.pow2_scaling > 1 || (P.precision == 2 && P.df_sums != 0) ||
      (P.tile_mult != 0 && P.tile_mult != 1 && P.tile_mult != 2 && P.tile_mult != 4))
    return set_err(nullptr, RHPDHG_ERR_INVALID_ARG, "invalid parameter");
  if ((P.dev_alloc == nullptr) != (P.dev_free == nullptr))
    return set_err(nullptr, RHPDHG_ERR_INVALID_ARG,
                   "invalid parameter: dev_alloc and dev_free are given together or not at all");
  if (P.adaptive_step && P.precision != 0)
    return set_err(nullptr, RHPDHG_ERR_INVALID_ARG,
                   "the adaptive step rule runs with precision 0 (FP64) only");

  h = new rhpdhg_handle();
  h->p = P;
  h->mixed = P.precision >= 1;
  h->ic.bf16 = P.precision == 2 ? 1 : 0;
  h->created_mixed = h->mixed;
  h->m = m;
  h->m_eq = lp->m_eq;
  h->m_ineq = lp->m_ineq;
  h->n = lp->n;
  h->nnz = lp->nnz;
  h->obj_offset = lp->obj_offset;
  h->st = (cudaStream_t)cuda_stream;
  if (P.x0) h->h_x0.assign(P.x0, P.x0 + h->n);
  if (P.y0) h->h_y0.assign(P.y0, P.y0 + m);
  h->p.x0 = nullptr;
  h->p.y0 = nullptr;

  auto fail = [&](int code) {
    std::string msg = h->err;
    destroy(h);
    g_create_error = msg;
    return code;
  };
#define CKC(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                             \
      return fail(e_ == cudaErrorMemoryAllocation ? RHPDHG_ERR_OOM : RHPDHG_ERR_CUDA);          \
    }                                                                                          \
  } while (0)

  const long long launches0 = launches_so_far();
  CKC(cudaGetDevice(&h->dev));
  if (!h->st) {
    // stream capture is not allowed on the legacy default stream: use a private stream
    CKC(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  CKC(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->dev));
  // every device buffer of this create comes from the caller's allocator when one is given
  DevAllocator hook;
  hook.alloc = P.dev_alloc;
  hook.free = P.dev_free;
  hook.ctx = P.alloc_ctx;
  hook.stream = (void *)h->st;
  AllocScope alloc_scope(hook);
  const int n = h->n;
  const int nnz = (int)h->nnz;
  const cudaStream_t st = h->st;
  const cudaMemcpyKind kind =
      lp->memory == RHPDHG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;

  // ---- upload + validate ----
  long long *rp64 = nullptr;
  int *rp = nullptr, *col = nullptr, *cp = nullptr, *ridx = nullptr;
  double *val = nullptr, *cval = nullptr, *c_in = nullptr, *q_in = nullptr, *l_in = nullptr,
         *u_in = nullptr, *tmp = nullptr;
  unsigned int *flags = nullptr;
  auto free_tmp = [&]() {
    cudaStreamSynchronize(st);
    for (void *b : {(void *)rp64, (void *)rp, (void *)col, (void *)cp, (void *)ridx, (void *)val,
                    (void *)cval, (void *)c_in, (void *)q_in, (void *)l_in, (void *)u_in,
                    (void *)tmp, (void *)flags})
      buf_release(b);
    rp64 = nullptr; rp = col = cp = ridx = nullptr; val = cval = c_in = q_in = l_in = u_in = tmp = nullptr;
    flags = nullptr;
  };
#define CKT(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      free_tmp();                                                                              \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                             \
      return fail(e_ == cudaErrorMemoryAllocation ? RHPDHG_ERR_OOM : RHPDHG_ERR_CUDA);          \
    }                                                                                          \
  } while (0)

  CKT(dalloc(&rp64, m + 1));
  CKT(dalloc(&rp, m + 1));
  CKT(dalloc(&col, nnz));
  CKT(dalloc(&val, nnz));
  CKT(dalloc(&c_in, n));
  CKT(dalloc(&q_in, m));
  CKT(dalloc(&l_in, n));
  CKT(dalloc(&u_in, n));
  CKT(dalloc(&flags, 1));
  CKT(dalloc(&tmp, 1024));
  CKT(cudaMemcpyAsync(rp64, lp->row_ptr, (m + 1) * sizeof(long long), kind, st));
  if (nnz > 0) {
    CKT(cudaMemcpyAsync(col, lp->col_idx, (size_t)nnz * sizeof(int), kind, st));
    CKT(cudaMemcpyAsync(val, lp->val, (size_t)nnz * sizeof(double), kind, st));
  }
  CKT(cudaMemcpyAsync(c_in, lp->c, n * sizeof(double), kind, st));
  if (m > 0) CKT(cudaMemcpyAsync(q_in, lp->rhs, m * sizeof(double), kind, st));
  CKT(cudaMemcpyAsync(l_in, lp->l, n * sizeof(double), kind, st));
  CKT(cudaMemcpyAsync(u_in, lp->u, n * sizeof(double), kind, st));
  unsigned int vf = validate_problem(st, m, n, h->nnz, rp64, col, val, c_in, q_in, l_in, u_in,
                                     flags);
  CKT(cudaGetLastError());
  h->ic.no_upper = (vf & kHasFiniteUpper) ? 0 : 1;
  vf &= ~kHasFiniteUpper;
  if (vf) {
    std::string msg = "invalid problem:";
    if (vf & 1u) msg += " malformed row_ptr;";
    if (vf & 2u) msg += " column index out of range or not strictly increasing in a row;";
    if (vf & 4u) msg += " non-finite matrix value;";
    if (vf & 8u) msg += " non-finite c or rhs;";
    if (vf & 16u) msg += " NaN bound or l > u;";
    if (vf & 32u) msg += " l = +inf or u = -inf;";
    free_tmp();
    h->err = msg;
    return fail(RHPDHG_ERR_INVALID_ARG);
  }
  convert_row_ptr(st, m, rp64, rp);

  // ---- transpose + scaling ----
  CKT(dalloc(&cp, n + 1));
  CKT(dalloc(&ridx, nnz));
  CKT(dalloc(&cval, nnz));
  CKT(build_transpose(st, m, n, nnz, rp, col, val, cp, ridx, cval));
  CKT(dalloc(&h->D, m));
  CKT(dalloc(&h->E, n));
  CKT(dalloc(&h->Dinv, m));
  CKT(dalloc(&h->Einv, n));
  {
    double *tm = nullptr, *tn = nullptr;
    CKT(dalloc(&tm, m));
    CKT(dalloc(&tn, n));
    compute_scaling(st, m, n, rp, col, val, cp, ridx, cval, P.ruiz_iters, P.pock_chambolle_alpha,
                    h->D, h->E, tm, tn);
    if (P.pow2_scaling || P.precision == 2) {
      round_pow2(st, m, h->D);
      round_pow2(st, n, h->E);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    buf_release(tm);
    buf_release(tn);
    CKT(e);
    CKT(cudaGetLastError());
  }
  // ---- layouts ----
  {
    std::vector<int> hrp(m + 1), hcp(n + 1);
    CKT(cudaMemcpy(hrp.data(), rp, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    CKT(cudaMemcpy(hcp.data(), cp, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    // precision 2 keeps BF16 values of K^, exact when every value of K has at most 8
    // significant bits (the scaling factors are powers of two)
    if (P.precision == 2 && !values_exact_in_bf16(st, h->nnz, val, flags)) {
      free_tmp();
      h->err = "precision 2 needs matrix values exactly representable in BF16 (at most 8 "
               "significant bits, within the FP32 exponent range)";
      return fail(RHPDHG_ERR_INVALID_ARG);
    }
    const int lowp = P.precision;
    h->ic.rho2 = P.algorithm == 1 ? 1 : 0;
    h->ic.df_sums = P.df_sums;
    if (P.autotune) h->tune_sig = shape_signature(h, hrp, hcp);
    CKT(build_side(st, m, nnz, rp, col, val, h->D, h->E, lowp, &h->rows));
    CKT(build_side(st, n, nnz, cp, ridx, cval, h->E, h->D, lowp, &h->cols));
  }
  // ---- scaled vectors ----
  CKT(dalloc(&h->c, n));
  CKT(dalloc(&h->q, m));
  CKT(dalloc(&h->l, n));
  CKT(dalloc(&h->u, n));
  vmul(st, n, h->E, c_in, h->c, 0);
  vmul(st, m, h->D, q_in, h->q, 0);
  vmul(st, n, h->E, l_in, h->l, 1);
  vmul(st, n, h->E, u_in, h->u, 1);
  fill(st, m, 1.0, h->Dinv);
  fill(st, n, 1.0, h->Einv);
  vmul(st, m, h->D, h->Dinv, h->Dinv, 1);
  vmul(st, n, h->E, h->Einv, h->Einv, 1);
  // norms: ||c||, ||rhs|| (unscaled) and ||c^||, ||q^|| (scaled)
  double *dn = nullptr;
  CKT(dalloc(&dn, 8));
  sumsq(st, n, c_in, dn + 0, tmp);
  sumsq(st, m, q_in, dn + 1, tmp);
  sumsq(st, n, h->c, dn + 2, tmp);
  sumsq(st, m, h->q, dn + 3, tmp);
  double hn[8] = {0};
  CKT(cudaMemcpyAsync(hn, dn, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CKT(cudaStreamSynchronize(st));
  const double cn = std::sqrt(hn[0]), qn = std::sqrt(hn[1]);
  const double chn = std::sqrt(hn[2]), qhn = std::sqrt(hn[3]);
  free_tmp();

  // ---- launch geometry ----
  allow_large_smem(kMaxTileSmem);
  allow_large_smem_setup(kMaxTileSmem);
  allow_large_smem_mx(kMaxTileSmem);
  // the rule's geometry for the power iteration, so that the step size does not depend on the
  // launch shape asked for (which is applied after it)
  set_geometry(h, SideShape{}, SideShape{});

  // ---- power iteration for sigma_max(K^) ----
  // v <- K^T K^ v / ||K^T K^ v|| from v = 1/sqrt(n); each step is two fused products (the
  // normalisation rides on the next product's input scale), then sigma = ||K^ v||.
  {
    double *v = nullptr, *w = nullptr, *um = nullptr, *pp = nullptr, *ss = nullptr;
    unsigned int *tk = nullptr;
    // FP64 handles in FP64; mixed-precision handles in their own value precision with FP32
    // products and row sums (the step keeps its 10% margin: eta sigma_max = 0.9 (1 + O(1e-6)))
    const int lowp = P.precision;
    const int gr = side_spmv_pw_grid(h->rows, lowp, h->sm_count);
    const int gc = side_spmv_pw_grid(h->cols, lowp, h->sm_count);
    const int gmax = std::max(gr, gc);
    CKT(dalloc(&v, n));
    CKT(dalloc(&w, n));
    CKT(dalloc(&um, m));
    CKT(dalloc(&pp, (size_t)gmax * kMaxPartials));
    CKT(dalloc(&ss, 8));
    CKT(dalloc(&tk, 1));
    CKT(cudaMemsetAsync(tk, 0, sizeof(unsigned int), st));
    fill(st, n, 1.0 / std::sqrt((double)n), v);
    const double *scale = nullptr;       // v is already normalised
    for (int it = 0; it < P.power_iters; ++it) {
      side_spmv_pw(st, h->rows, lowp, v, scale, um, pp, tk, ss + 2, gr);
      side_spmv_pw(st, h->cols, lowp, um, nullptr, w, pp, tk, ss + 4, gc);
      std::swap(v, w);
      scale = ss + 5;                    // 1 / ||K^T K^ v||
    }
    side_spmv_pw(st, h->rows, lowp, v, scale, um, pp, tk, ss + 6, gr);
    double s2 = 0;
    CKT(cudaMemcpyAsync(&s2, ss + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
    CKT(cudaStreamSynchronize(st));
    CKT(cudaGetLastError());
    buf_release(v);
    buf_release(w);
    buf_release(um);
    buf_release(pp);
    buf_release(ss);
    buf_release(tk);
    h->sigma_max = (m > 0 && h->nnz > 0) ? std::sqrt(s2) : 0.0;
  }
  buf_release(dn);
  {
    SideShape r, c;
    r.warps = c.warps = P.cta_warps > 0 ? P.cta_warps : kBlockWarps;
    r.mult = c.mult = P.tile_mult;   // 0 = the rule; a side whose group does not fit keeps it
    set_geometry(h, r, c);
  }
  if (P.step_size > 0) h->eta = P.step_size;
  else if (h->sigma_max > 1e-12) h->eta = P.step_safety / h->sigma_max;
  else h->eta = 1.0;
  if (P.primal_weight > 0) h->omega0 = P.primal_weight;
  else h->omega0 = (chn > 1e-10 && qhn > 1e-10) ? chn / qhn : 1.0;

  // ---- iteration state ----
  double **nv[] = {&h->x, &h->xt, &h->x0, &h->kty, &h->kty0, &h->xout, &h->certx, &h->certx2,
                   &h->x_init,
                   &h->xres};
  for (double **b : nv) CKC(dalloc(b, n));
  double **mv[] = {&h->y, &h->yt, &h->y0, &h->kx, &h->kxt, &h->kx0, &h->certy, &h->certy2,
                   &h->y_init,
                   &h->yres};
  for (double **b : mv) CKC(dalloc(b, m));
  if (h->mixed) {
    float **fn[] = {&h->dxt, &h->dx, &h->ktdy, &h->s0, &h->xlo, &h->xhi};
    for (float **b : fn) CKC(dalloc(b, n));
    float **fm[] = {&h->dyt, &h->kdxt, &h->dy, &h->kdx, &h->r0, &h->ylo};
    for (float **b : fm) CKC(dalloc(b, m));
    CKC(dalloc(&h->dxt64, n));
    CKC(dalloc(&h->dyt64, m));
  }
  CKC(dalloc(&h->act, n));
  CKC(cudaMemsetAsync(h->certx, 0, n * sizeof(double), st));
  CKC(cudaMemsetAsync(h->certx2, 0, n * sizeof(double), st));
  if (m) CKC(cudaMemsetAsync(h->certy, 0, m * sizeof(double), st));
  if (m) CKC(cudaMemsetAsync(h->certy2, 0, m * sizeof(double), st));
  CKC(dalloc(&h->ctl, 1));
  CKC(cudaHostAlloc((void **)&h->h_mirror, 2 * sizeof(Ctl), cudaHostAllocDefault));
  std::memset(h->h_mirror, 0, 2 * sizeof(Ctl));
  {
    int gr = h->grid_row, gc = h->grid_col;
    if (P.autotune && P.cta_warps == 0 && P.tile_mult == 0) candidate_grids(h, &gr, &gc);
    CKC(dalloc(&h->part_row, (size_t)gr * kMaxPartials));
    CKC(dalloc(&h->part_col, (size_t)gc * kMaxPartials));
  }
  if (P.trace && P.trace_capacity > 0) CKC(dalloc(&h->trace, (size_t)P.trace_capacity));
  CKC(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), st));

  // initial point z^{0,0}: the projection of 0 onto [l, u], or the warm start (scaled)
  if (!h->h_x0.empty()) {
    CKC(cudaMemcpyAsync(h->x_init, h->h_x0.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    vmul(st, n, h->E, h->x_init, h->x_init, 1);
  } else {
    fill(st, n, 0.0, h->x_init);
    vclamp(st, n, h->x_init, h->l, h->u);
  }
  if (m) {
    if (!h->h_y0.empty()) {
      CKC(cudaMemcpyAsync(h->y_init, h->h_y0.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
      vmul(st, m, h->D, h->y_init, h->y_init, 1);
    } else {
      fill(st, m, 0.0, h->y_init);
    }
  }

  IterConsts &ic = h->ic;
  ic.m = m; ic.m_eq = h->m_eq; ic.n = n;
  ic.rho2 = P.algorithm == 1 ? 1 : 0;
  ic.max_iters = P.max_iters;
  ic.check_every = P.check_every;
  ic.first_epoch_len = P.first_epoch_len;
  ic.max_epoch_len = P.max_epoch_len;
  ic.restart_scheme = P.restart_scheme;
  ic.pw_update = P.primal_weight_update;
  ic.beta2 = P.restart_beta * P.restart_beta;
  ic.eta = h->eta;
  ic.eps_kkt = P.eps_rel_kkt;
  ic.eps_infeas = P.eps_infeas;
  ic.qn1 = 1.0 + qn;
  ic.cn1 = 1.0 + cn;
  ic.obj_offset = h->obj_offset;
  ic.trace_cap = h->trace ? P.trace_capacity : 0;
  ic.trace = h->trace;
  ic.mixed = h->mixed ? 1 : 0;
  ic.df_sums = P.df_sums;
  ic.adaptive = P.adaptive_step ? 1 : 0;
  h->rv = RowVecs{h->y, h->yt, h->y0, h->kx, h->kxt, h->kx0, h->certy, h->q, h->D, h->Dinv,
                  h->certy2};
  h->cv = ColVecs{h->x, h->xt, h->x0, h->kty, h->kty0, h->xout, h->certx, h->c, h->l, h->u,
                  h->E, h->Einv, h->certx2, h->act};
  h->rvm = RowVecsMx{h->dyt, h->kdxt, h->dy, h->kdx, h->r0, h->ylo, h->y0, h->kx0, h->certy,
                     h->dyt64, h->q, h->D, h->Dinv, h->certy2};
  h->cvm = ColVecsMx{h->dxt, h->dx, h->ktdy, h->s0, h->xlo, h->xhi, h->x0, h->kty0, h->xout,
                     h->certx, h->dxt64, h->c, h->l, h->u, h->E, h->Einv, h->certx2, h->act};
  algorithmic_bytes(h);
  {
    // the ordinary mixed kernels read the matrix stream evict-first where one iteration's
    // bytes exceed L2 (see Vec4 in common.cuh)
    int l2 = 0;
    CKC(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->dev));
    h->ic.l2_first = h->mixed && h->bytes_row + h->bytes_col > (double)l2 ? 1 : 0;
  }
  h->launches = launches_so_far() - launches0;
  CKC(cudaStreamSynchronize(st));
  CKC(cudaGetLastError());
  if (P.autotune && P.cta_warps == 0 && P.tile_mult == 0) {
    const int rc = autotune(h);
    if (rc != RHPDHG_OK) return fail(rc);
  }
  *out = h;
  return RHPDHG_OK;
#undef CKC
#undef CKT
}

int rhpdhg_solve(rhpdhg_handle *h, int blocking) {
  if (!h) return set_err(nullptr, RHPDHG_ERR_INVALID_ARG, "handle is NULL");
  if (h->running.load()) return set_err(h, RHPDHG_ERR_STATE, "a solve is already running");
  if (h->th.joinable()) h->th.join();
  h->cancel = 0;
  h->drive_err = 0;
  h->solved = false;
  h->running = 1;
  if (blocking) {
    drive(h);
    return h->drive_err ? h->drive_err : RHPDHG_OK;
  }
  h->th = std::thread(drive, h);
  return RHPDHG_OK;
}

int rhpdhg_poll(rhpdhg_handle *h, rhpdhg_result *r) {
  if (!h || !r) return set_err(h, RHPDHG_ERR_INVALID_ARG, "handle or result is NULL");
  if (h->running.load()) return RHPDHG_BUSY;
  if (h->th.joinable()) h->th.join();
  if (!h->solved) return set_err(h, RHPDHG_ERR_STATE, "no solve has run");
  if (h->drive_err) return h->drive_err;
  const Ctl &c = h->final_ctl;
  r->status = h->final_status;
  r->iters = c.t;
  r->restarts = c.n;
  r->rel_p = c.rel_p;
  r->rel_d = c.rel_d;
  r->rel_gap = c.rel_gap;
  r->primal_obj = c.pobj;
  r->dual_obj = c.dobj;
  r->solve_seconds = h->solve_seconds;
  r->eta = h->p.adaptive_step ? c.eta : h->eta;
  r->omega = c.omega;
  r->sigma_max = h->sigma_max;
  const cudaMemcpyKind kind =
      r->out_memory == RHPDHG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (r->x) CK(cudaMemcpyAsync(r->x, h->xres, h->n * sizeof(double), kind, h->st));
  if (r->y && h->m) CK(cudaMemcpyAsync(r->y, h->yres, h->m * sizeof(double), kind, h->st));
  r->cert_source = c.cert_src;
  r->escalated = h->escalated ? 1 : 0;
  const bool mv = c.cert_src == kCertAnchorMove;
  if (r->cert_x)
    CK(cudaMemcpyAsync(r->cert_x, mv ? h->certx2 : h->certx, h->n * sizeof(double), kind, h->st));
  if (r->cert_y && h->m)
    CK(cudaMemcpyAsync(r->cert_y, mv ? h->certy2 : h->certy, h->m * sizeof(double), kind, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RHPDHG_OK;
}

int rhpdhg_cancel(rhpdhg_handle *h) {
  if (!h) return RHPDHG_ERR_INVALID_ARG;
  h->cancel = 1;
  return RHPDHG_OK;
}

void rhpdhg_free(rhpdhg_handle *h) {
  if (!h) return;
  h->cancel = 1;
  if (h->th.joinable()) h->th.join();
  destroy(h);
}

int rhpdhg_get_state(const rhpdhg_handle *hc, int which, double *x, double *y) {
  rhpdhg_handle *h = const_cast<rhpdhg_handle *>(hc);
  if (!h) return RHPDHG_ERR_INVALID_ARG;
  if (h->running.load()) return set_err(h, RHPDHG_ERR_STATE, "solve running");
  const double *xs = nullptr, *ys = nullptr;
  if (which == 1) { xs = h->xout; ys = h->yt; }
  else if (which == 2) { xs = h->x0; ys = h->y0; }
  else return set_err(h, RHPDHG_ERR_INVALID_ARG, "which must be 1 (PDHG point) or 2 (anchor)");
  if (x) CK(cudaMemcpyAsync(x, xs, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (y && h->m) CK(cudaMemcpyAsync(y, ys, h->m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RHPDHG_OK;
}

int rhpdhg_get_scaling(const rhpdhg_handle *hc, double *D, double *E, double *eta,
                       double *omega0, double *sigma_max) {
  rhpdhg_handle *h = const_cast<rhpdhg_handle *>(hc);
  if (!h) return RHPDHG_ERR_INVALID_ARG;
  if (h->running.load()) return set_err(h, RHPDHG_ERR_STATE, "solve running");
  if (D && h->m) CK(cudaMemcpyAsync(D, h->D, h->m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (E) CK(cudaMemcpyAsync(E, h->E, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (eta) *eta = h->eta;
  if (omega0) *omega0 = h->omega0;
  if (sigma_max) *sigma_max = h->sigma_max;
  return RHPDHG_OK;
}

int rhpdhg_get_layout(const rhpdhg_handle *h, int64_t *out, int32_t capacity) {
  if (!h || !out || capacity < RHPDHG_LAYOUT_FIELDS) return RHPDHG_ERR_INVALID_ARG;
  const SideLayout &r = h->rows.lay, &c = h->cols.lay;
  const int64_t v[RHPDHG_LAYOUT_FIELDS] = {h->grid_row,  h->grid_col,  r.tile_mult, c.tile_mult,
                                           r.n_long,     c.n_long,     r.n_chunks,  c.n_chunks,
                                           r.seg,        c.seg,        r.walk,      c.walk,
                                           r.cta_warps,  c.cta_warps,  h->tuned,
                                           (int64_t)std::llround(1e3 * h->tune_us_rule),
                                           (int64_t)std::llround(1e3 * h->tune_us_best),
                                           r.wide_rows,  c.wide_rows};
  for (int i = 0; i < RHPDHG_LAYOUT_FIELDS; ++i) out[i] = v[i];
  return RHPDHG_OK;
}

int64_t rhpdhg_release_cached_memory(void) { return (int64_t)buf_drop_cache(); }

int rhpdhg_plan_layout(const int64_t *row_ptr, int32_t nrows, int64_t *out, int32_t capacity) {
  if (!row_ptr || !out || nrows < 0 || capacity < RHPDHG_PLAN_FIELDS || row_ptr[0] != 0)
    return RHPDHG_ERR_INVALID_ARG;
  std::vector<int> hp((size_t)nrows + 1);
  for (int32_t i = 0; i <= nrows; ++i) {
    if (row_ptr[i] > INT_MAX || (i > 0 && row_ptr[i] < row_ptr[i - 1]))
      return RHPDHG_ERR_INVALID_ARG;
    hp[i] = (int)row_ptr[i];
  }
  SidePlan P;
  if (!plan_side(hp.data(), nrows, &P)) return RHPDHG_ERR_INVALID_ARG;
  const int64_t v[RHPDHG_PLAN_FIELDS] = {P.ntiles,
                                         P.mult,
                                         (int64_t)P.long_rows.size(),
                                         (int64_t)P.chunk_row.size(),
                                         ((P.maxseg + 3) & ~3LL) + 4,
                                         P.nnz_s,
                                         P.nnz_l,
                                         P.wide_rows};
  for (int i = 0; i < RHPDHG_PLAN_FIELDS; ++i) out[i] = v[i];
  return RHPDHG_OK;
}

int rhpdhg_get_trace(const rhpdhg_handle *hc, rhpdhg_trace_rec *recs, int64_t capacity,
                     int64_t *count) {
  rhpdhg_handle *h = const_cast<rhpdhg_handle *>(hc);
  if (!h || !count) return RHPDHG_ERR_INVALID_ARG;
  if (h->running.load()) return set_err(h, RHPDHG_ERR_STATE, "solve running");
  if (!h->trace) { *count = 0; return RHPDHG_OK; }
  long long iters = h->final_ctl.t;
  long long cnt = std::min<long long>(iters, h->ic.trace_cap);
  *count = cnt;
  long long ncopy = std::min<long long>(cnt, capacity);
  static_assert(sizeof(TraceRec) == sizeof(rhpdhg_trace_rec), "trace record layout");
  if (recs && ncopy > 0)
    CK(cudaMemcpy(recs, h->trace, ncopy * sizeof(TraceRec), cudaMemcpyDeviceToHost));
  return RHPDHG_OK;
}

int rhpdhg_kernel_times(const rhpdhg_handle *hc, double *ms_row, double *ms_col,
                        int64_t *launches_row, int64_t *launches_col, double *bytes_row,
                        double *bytes_col) {
  const rhpdhg_handle *h = hc;
  if (!h) return RHPDHG_ERR_INVALID_ARG;
  if (ms_row) *ms_row = h->n_row ? h->ms_row / h->n_row : 0.0;
  if (ms_col) *ms_col = h->n_col ? h->ms_col / h->n_col : 0.0;
  if (launches_row) *launches_row = h->n_row;
  if (launches_col) *launches_col = h->n_col;
  if (bytes_row) *bytes_row = h->bytes_row;
  if (bytes_col) *bytes_col = h->bytes_col;
  return RHPDHG_OK;
}

int64_t rhpdhg_launch_count(const rhpdhg_handle *h) { return h ? h->launches : -1; }

}  // extern "C"
