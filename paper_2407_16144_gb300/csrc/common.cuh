// Internal definitions shared by the kernels and the C-ABI layer of the rHPDHG library.
//
// Data layout in device memory (one LP):
//   * Each side of the bilinear form is one "row operator": the row side is K^ (m rows, used
//     for K^ x~) and the column side is K^T (n rows, used for K^T y~).  Each is stored in a
//     tiled split-CSR layout (SideLayout): rows with at most L entries live in a short CSR
//     (long rows have zero length there) processed 32 rows per warp, one lane per row; rows
//     with more than L entries live in a long CSR processed by a whole warp per row.  Both kinds
//     end in the same per-row epilogue, executed by one lane per row so the FP64 work of the
//     epilogue (the method's elementwise part) runs with all 32 lanes active.
//   * Vectors are plain arrays indexed by row (m) or column (n) in the original order.
//   * A small control block (Ctl) holds the iteration counters, the restart decision, the step
//     data and the staged reduction results; kernels read it at entry and the last CTA of each
//     kernel updates it, so the restart test and the termination test never leave the device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace rh {

constexpr int kWarp = 32;
constexpr int kTileRows = 32;          // rows per tile = lanes per warp
constexpr int kBlockWarps = 4;         // warps per CTA of the tile kernels
constexpr int kBlockThreads = kBlockWarps * kWarp;
constexpr int kMaxPartials = 16;       // reduction slots per CTA
constexpr int kMaxTileL = 64;          // largest short-row threshold
constexpr int kMaxTileSmem = kBlockWarps * kTileRows * kMaxTileL * 8;   // bytes

enum Status : int {
  kRunning = 0, kOptimal = 1, kPrimalInfeasible = 2, kDualInfeasible = 3, kIterLimit = 4,
  kTimeLimit = 5, kNumericalError = 6, kCancelled = 7
};

// Split-CSR layout of one side (see file comment).  Values are the scaled matrix entries.
template <typename VT>
struct SideLayout {
  int nrows = 0;
  int L = 32;                // short-row threshold: rows with <= L entries are short
  int n_short_tiles = 0;     // ceil(nrows / 32)
  int n_long = 0;            // number of long rows
  int n_long_tiles = 0;      // ceil(n_long / 32)
  const int *ptr_s = nullptr;       // nrows + 1
  const int *idx_s = nullptr;       // nnz_short
  const VT *val_s = nullptr;        // nnz_short
  const uint32_t *long_mask = nullptr;  // n_short_tiles words: bit r set if row 32t+r is long
  const int *long_rows = nullptr;   // n_long row ids (ascending)
  const int *ptr_l = nullptr;       // n_long + 1
  const int *idx_l = nullptr;       // nnz_long
  const VT *val_l = nullptr;        // nnz_long
  __host__ __device__ int total_tiles() const { return n_short_tiles + n_long_tiles; }
};

// Device control block.  Written only by the last CTA of a kernel (or by the host while no
// kernel of the handle runs); read by every CTA at kernel entry.
struct Ctl {
  long long t;           // index of the current iteration (PDHG evaluation)
  long long k;           // inner index of the current iterate z^{n,k}
  long long n;           // outer index (epoch)
  long long k_next, n_next;
  int status;
  int restart_pending;   // 1: iterate t+1 is the restart point T(z^{n,k})
  double w;              // Halpern weight (k+1)/(k+2) of the pending blend
  double omega, tau, sigma, eta;
  double fpr0_sq;        // ||z^{n,0} - T(z^{n,0})||_P^2
  double fpr_sq;         // last ||z - T(z)||_P^2
  double dx_sq;          // ||x_t - x~_t||^2          (column kernel -> next row kernel)
  double xa_sq;          // ||x~_t - x^{n,0}||^2      (primal-weight update)
  // row-side parts of the termination and infeasibility tests of iteration t
  double rp_sq, qy, inf_qv, inf_yneg, inf_kd_eq, inf_kd_in;
  // last termination check
  double rel_p, rel_d, rel_gap, pobj, dobj;
  long long check_t;
  long long restarts;
  unsigned int cnt_row, cnt_col;   // last-CTA tickets
  int pad;
};

struct TraceRec {      // mirrors rhpdhg_trace_rec
  long long t, epoch, k;
  double fpr_sq, omega;
  int restart, pad;
};

// Per-solve constants passed by value to the iteration kernels.
struct IterConsts {
  int m, m_eq, n;
  int rho2;                   // 1 = reflected (r2HPDHG)
  long long max_iters;
  int check_every;
  int first_epoch_len;
  long long max_epoch_len;
  int restart_scheme;
  int pw_update;
  double beta2;
  double eta;
  double eps_kkt, eps_infeas;
  double qn1, cn1;            // 1 + ||rhs||_2, 1 + ||c||_2 (unscaled)
  double obj_offset;
  long long trace_cap;
  TraceRec *trace;
};

// ---------------------------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per-thread accumulators of NS sums and NM maxima, reduced per CTA in a fixed order.
template <int NS, int NM>
struct Acc {
  double s[NS > 0 ? NS : 1];
  double mx[NM > 0 ? NM : 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = 0.0;
#pragma unroll
    for (int i = 0; i < NM; ++i) mx[i] = 0.0;
  }
};

// Reduce Acc over the CTA (deterministic: fixed shuffle tree, warps summed in index order) and
// write the CTA's partials to part[blockIdx.x * kMaxPartials + slot].  Returns true in every
// thread of the last CTA to finish (after a fence), which then owns the grid-level reduction.
template <int NS, int NM>
__device__ bool cta_reduce_and_ticket(Acc<NS, NM> &a, double *part, unsigned int *ticket) {
  __shared__ double red[kBlockWarps][kMaxPartials];
  __shared__ bool last;
  static_assert(NS + NM <= kMaxPartials, "too many partial slots");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    double v = warp_sum(a.s[i]);
    if (lane == 0) red[warp][i] = v;
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    double v = warp_max(a.mx[i]);
    if (lane == 0) red[warp][NS + i] = v;
  }
  __syncthreads();
  if (threadIdx.x < NS + NM) {
    const int i = threadIdx.x;
    double v = red[0][i];
    for (int w = 1; w < kBlockWarps; ++w) v = (i < NS) ? v + red[w][i] : fmax(v, red[w][i]);
    part[(size_t)blockIdx.x * kMaxPartials + i] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int tk = atomicAdd(ticket, 1u);
    last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the last CTA: reduce the grid's partials in block order.  out[i] valid in all threads.
template <int NS, int NM>
__device__ void grid_finish(const double *part, double *out) {
  __shared__ double red[kBlockWarps][kMaxPartials];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = gridDim.x;
  double v[NS + NM];
#pragma unroll
  for (int i = 0; i < NS + NM; ++i) v[i] = 0.0;
  // thread t sums blocks t, t + blockDim, ... (fixed order)
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NS + NM; ++i) {
      double p = __ldcg(part + (size_t)b * kMaxPartials + i);
      v[i] = (i < NS) ? v[i] + p : fmax(v[i], p);
    }
  }
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    double r = warp_sum(v[i]);
    if (lane == 0) red[warp][i] = r;
  }
#pragma unroll
  for (int i = NS; i < NS + NM; ++i) {
    double r = warp_max(v[i]);
    if (lane == 0) red[warp][i] = r;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NS + NM; ++i) {
    double r = red[0][i];
    for (int w = 1; w < kBlockWarps; ++w) r = (i < NS) ? r + red[w][i] : fmax(r, red[w][i]);
    out[i] = r;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// The tile walker: computes dot = (row of the side operator) . src for every row and calls
// epi(row, dot) once per row, from one lane.  SrcT is the gathered vector type, VT the value
// type, PT the product/accumulator type.  smem points to this warp's staging area of at least
// 32 * L elements of PT.

template <typename VT, typename SrcT, typename PT, typename Epi>
__device__ __forceinline__ void walk_tiles(const SideLayout<VT> &lay, const SrcT *__restrict__ src,
                                           PT *smem, Epi &epi) {
  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * kBlockWarps + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * kBlockWarps;
  const int total = lay.total_tiles();
  for (int tile = gwarp; tile < total; tile += nwarps) {
    if (tile < lay.n_long_tiles) {
      // long rows: a whole warp per row, results collected one per lane
      const int base = tile * kTileRows;
      const int cnt = min(kTileRows, lay.n_long - base);
      PT mine = PT(0);
      int my_row = -1;
      for (int i = 0; i < cnt; ++i) {
        const int b = lay.ptr_l[base + i], e = lay.ptr_l[base + i + 1];
        PT s = PT(0);
        for (int p = b + lane; p < e; p += kWarp)
          s += PT(lay.val_l[p]) * PT(src[lay.idx_l[p]]);
        s = warp_sum(s);
        if (lane == i) { mine = s; my_row = lay.long_rows[base + i]; }
      }
      if (my_row >= 0) epi(my_row, mine);
    } else {
      const int st = tile - lay.n_long_tiles;
      const int row0 = st * kTileRows;
      const int nr = min(kTileRows, lay.nrows - row0);
      // row pointers: lane r holds ptr_s[row0 + r] (clamped to the tile end)
      const int pl = lay.ptr_s[row0 + min(lane, nr)];
      const int seg_e = lay.ptr_s[row0 + nr];
      const int seg_b = __shfl_sync(0xffffffffu, pl, 0);
      const int rb = pl;
      int re = __shfl_down_sync(0xffffffffu, pl, 1);
      if (lane == kWarp - 1) re = seg_e;
      // stage the products of the tile's segment (coalesced value / index loads)
      for (int p = seg_b + lane; p < seg_e; p += kWarp)
        smem[p - seg_b] = PT(lay.val_s[p]) * PT(src[lay.idx_s[p]]);
      __syncwarp();
      const uint32_t lm = lay.long_mask[st];
      if (lane < nr && !((lm >> lane) & 1u)) {
        PT s = PT(0);
        for (int p = rb; p < re; ++p) s += smem[p - seg_b];
        epi(row0 + lane, s);
      }
      __syncwarp();
    }
  }
}

}  // namespace rh
