// Launch wrappers shared between the translation units of the library (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "common.cuh"
#include "../../include/rhpdhg.h"

namespace rh {

// Owning device buffers of one side: the split-CSR structure, its FP64 values, optionally an
// FP32 copy of the values (mixed precision), and two sets of walk scratch.
struct SideStore {
  SideLayout lay;
  SideVals<double> v64;
  SideVals<float> v32;
  SideVals<__nv_bfloat16> v16;
  WalkScratch wa, wb;
  int *ptr_s = nullptr, *tile_end = nullptr, *idx_s = nullptr, *long_rows = nullptr,
      *beg_l = nullptr, *end_l = nullptr, *idx_l = nullptr;
  uint32_t *long_mask = nullptr;
  int *chunk_ptr = nullptr, *chunk_row = nullptr;
  int4 *chunk_desc = nullptr;
  double *val64_s = nullptr, *val64_l = nullptr;
  float *val32_s = nullptr, *val32_l = nullptr;
  __nv_bfloat16 *val16_s = nullptr, *val16_l = nullptr;
  double *part_a = nullptr, *part_b = nullptr;
  unsigned int *done_a = nullptr, *done_b = nullptr;
  double *gpart_a = nullptr, *gpart_b = nullptr;
  long long nnz_short = 0, nnz_long = 0;
  int rule_mult = 1;                    // tiles per work item by the layout rule
  long long maxseg_mult[3] = {0, -1, -1};  // longest group segment with 1, 2, 4 tiles per item
                                           // (-1: over the staging budget)
};

// Tiles per work item m usable on a side (its longest group of m tiles fits the staging area).
inline bool mult_ok(const SideStore &sd, int m) {
  const int k = m == 4 ? 2 : (m == 2 ? 1 : 0);
  return (m == 1 || m == 2 || m == 4) && sd.maxseg_mult[k] >= 0;
}
// Sets the side's walk to m tiles per work item (mult_ok): item count and staging stride.
inline void apply_mult(SideStore &sd, int m) {
  const int k = m == 4 ? 2 : (m == 2 ? 1 : 0);
  sd.lay.tile_mult = m;
  sd.lay.n_tile_groups = (sd.lay.n_short_tiles + m - 1) / m;
  sd.lay.seg = (int)((sd.maxseg_mult[k] + 3) & ~3LL) + 4;
}

struct RowVecs {      // m-vectors used by the row kernel (K^ x~ and the dual step)
  double *y, *yt, *y0, *kx, *kxt, *kx0, *certy;
  const double *q, *d, *dinv;
  double *certy2;     // y-part of the anchor-movement candidate
};

struct ColVecs {      // n-vectors used by the column kernel (K^T y~ and the primal step)
  double *x, *xt, *x0, *kty, *kty0, *xout, *certx;
  const double *c, *l, *u, *e, *einv;
  double *certx2;     // x-part of the anchor-movement candidate
  unsigned char *act; // 1 where x~ was on a bound at the previous check
};

struct RowVecsMx {    // mixed precision, m-vectors (offsets from the FP64 anchor y0)
  float *dyt, *kdxt, *dy, *kdx, *r0, *ylo;
  double *y0, *kx0, *certy, *dyt64;
  const double *q, *d, *dinv;
  double *certy2;
};

struct ColVecsMx {    // mixed precision, n-vectors (offsets from the FP64 anchor x0)
  float *dxt, *dx, *ktdy, *s0, *xlo, *xhi;
  double *x0, *kty0, *xout, *certx, *dxt64;
  const double *c, *l, *u, *e, *einv;
  double *certx2;
  unsigned char *act;
};

// Message for rhpdhg_last_error(NULL) (calls without a handle).
void set_global_error(const std::string &msg);

// Launch through cudaLaunchKernelEx: the return value is this launch's own error (an error left
// by earlier, unrelated work of the process is neither reported nor cleared).
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), int grid, int block, size_t smem,
                          cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Process-wide count of kernels launched by this library's wrappers (for launch accounting).
void count_launches(long long n);
long long launches_so_far();

// ---- setup (setup.cu) ------------------------------------------------------------------------
// Validation of a device-resident problem: returns a bit mask of problems found (0 = valid),
// plus the information bit kHasFiniteUpper (not an error) when some u_j is finite.
unsigned int validate_problem(cudaStream_t st, int m, int n, long long nnz, const long long *row_ptr,
                              const int *col, const double *val, const double *c, const double *q,
                              const double *l, const double *u, unsigned int *d_flags);
// int64 -> int32 row pointers
void convert_row_ptr(cudaStream_t st, int m, const long long *rp64, int *rp32);
// CSR (m x n) -> CSC (column pointers, row indices, values), stable (rows ascending).
// Returns cudaSuccess or an error.
cudaError_t build_transpose(cudaStream_t st, int m, int n, int nnz, const int *rp, const int *col,
                            const double *val, int *cp, int *ridx, double *cval);
// Ruiz (ruiz_iters passes) then Pock-Chambolle (alpha; skipped when alpha < 0): fills D (m),
// E (n) so that D K E is the scaled matrix.
void compute_scaling(cudaStream_t st, int m, int n, const int *rp, const int *col,
                     const double *val, const int *cp, const int *ridx, const double *cval,
                     int ruiz_iters, double alpha, double *D, double *E, double *tmp_m,
                     double *tmp_n);
// Build a split-CSR side from a CSR (nrows rows) with values scaled as
// val * rscale[row] * cscale[col] (FP64, plus an FP32 copy for lowp 1 or a BF16 copy for lowp 2).
// Rows longer than kShortMax, and the longest rows of any tile whose short segment would exceed
// kSegBudget, go to the long CSR.  Device buffers come from buf_alloc.
cudaError_t build_side(cudaStream_t st, int nrows, int nnz, const int *ptr, const int *idx,
                       const double *val, const double *rscale, const double *cscale,
                       int lowp, SideStore *out);
// Each entry of v (n positive factors) rounded to the nearest power of two on a log scale.
void round_pow2(cudaStream_t st, int n, double *v);
// True when every value has at most 8 significant bits and fits the FP32 exponent range (is
// exact in BF16); d_flag is a device word of scratch.  Synchronises the stream.
unsigned int values_exact_in_bf16(cudaStream_t st, long long nnz, const double *val,
                                  unsigned int *d_flag);
void free_side(SideStore *s);
// Launch geometry of the tile kernels for a side with L: enough CTAs of lay.cta_warps warps for
// one work item per warp, at most blocks_per_sm resident CTAs per SM.
int tile_grid(const SideLayout &lay, int sm_count, int blocks_per_sm);
// out = side * src   (plain product, FP64)
void side_spmv(cudaStream_t st, const SideStore &side, const double *src, double *out, int grid);
// Power-iteration product: out = side * (src * in_scale[0]) and ss = (||out||^2, 1/||out||);
// lowp 0: FP64 values, products and sums; 1 / 2: the side's FP32 / BF16 values with FP32 products
// and row sums (mixed-precision handles); the norm is an FP64 sum in every case.
// part holds grid * kMaxPartials doubles, ticket a zeroed counter.
void side_spmv_pw(cudaStream_t st, const SideStore &side, int lowp, const double *src,
                  const double *in_scale, double *out, double *part, unsigned int *ticket,
                  double *ss, int grid);
int side_spmv_pw_grid(const SideStore &side, int lowp, int sm_count);
// deterministic sum of squares -> *out (device scalar); tmp holds >= 1024 doubles
void sumsq(cudaStream_t st, int n, const double *x, double *out, double *tmp);
// v = w / sqrt(*ss)
void fill(cudaStream_t st, int n, double v, double *x);
// y = a .* x (elementwise), optionally y = x ./ a when div = 1
void vmul(cudaStream_t st, int n, const double *a, const double *x, double *y, int div);
// x = clamp(x, l, u)
void vclamp(cudaStream_t st, int n, double *x, const double *l, const double *u);

// ---- iteration (iterate.cu) -----------------------------------------------------------------
// dc: the column stage's partials, which the row kernel reduces when that stage deferred them
void launch_row_iter(cudaStream_t st, const SideStore &side, const double *xt, const RowVecs &v,
                     Ctl *ctl, double *part, const IterConsts &ic, int grid, int smem,
                     const DeferredCol &dc);
void launch_col_iter(cudaStream_t st, const SideStore &side, const double *yt, const ColVecs &v,
                     Ctl *ctl, double *part, const IterConsts &ic, int grid, int smem,
                     int phase);
// x_out = E .* xout ; y_out = D .* yt
void launch_unscale(cudaStream_t st, int n, int m, const double *e, const double *xs,
                    const double *d, const double *ys, double *xo, double *yo);
int row_iter_blocks_per_sm(int smem, int threads);

// ---- standalone KKT evaluation (kkt.cu) --------------------------------------------------------
constexpr int kKktMaxBlocks = 1024;   // block partials of the evaluation kernels
constexpr int kKktSlotCount = 8;
int kkt_blocks(int m, int n);
// scratch: kty (n doubles), part (kKktMaxBlocks * kKktSlotCount doubles), dout (8 doubles);
// *bad_index is set when the CSR held a row offset or column index out of range
cudaError_t kkt_eval_with_scratch(const rhpdhg_problem *lp, const double *x, const double *y,
                                  cudaStream_t st, double *kty, double *part, double *dout,
                                  double *out, bool *bad_index);

// ---- mixed-precision iteration (iterate_mx.cu) -------------------------------------------------
// grid: CTAs of the ordinary kernel; grid1: CTAs of the restart-mode kernel (at most one wave)
void launch_row_iter_mx(cudaStream_t st, const SideStore &side, const RowVecsMx &v,
                        const float *dxt, const double *dxt64, const double *x0, Ctl *ctl,
                        double *part, const IterConsts &ic, int grid, int grid1, int smem,
                        const DeferredCol &dc);
void launch_col_iter_mx(cudaStream_t st, const SideStore &side, const ColVecsMx &v,
                        const float *dyt, const double *dyt64, const double *y0, Ctl *ctl,
                        double *part, const IterConsts &ic, int grid, int grid1, int smem,
                        int phase);
// Resident CTAs per SM of the restart-mode mixed kernels of one side (FP64 staging smem).
int iter_mx_restart_blocks_per_sm(int smem, bool row, int threads);
void launch_unscale_mx(cudaStream_t st, int n, int m, const double *e, const double *xs,
                       const double *d, const double *y0, const float *dyt, double *xo,
                       double *yo, double *yt64);
void zero_f32(cudaStream_t st, int n, float *x);
void allow_large_smem_mx(int bytes);
// Resident CTAs per SM of the ordinary mixed kernels of one side (row: K^, else K^T) in one
// walk instantiation (kWalk*), one kind of restart-norm sums (IterConsts::df_sums) and one value
// type (lp: 0 = FP32, 1 = BF16), for CTAs of `threads` threads.
int iter_mx_blocks_per_sm(int smem, bool row, int walk, int threads, int dfs, int lp);
// opt in to dynamic shared memory above 48 KB for the tile kernels
void allow_large_smem(int bytes);
void allow_large_smem_setup(int bytes);
int col_iter_blocks_per_sm(int smem, int threads);

}  // namespace rh
