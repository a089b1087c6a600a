// Internal definitions shared by the kernels and the C-ABI layer of the rHPDHG library.
//
// Data layout in device memory (one LP):
//   * Each side of the bilinear form is one "row operator": the row side is K^ (m rows, used
//     for K^ x~) and the column side is K^T (n rows, used for K^T y~).  Each is stored in a
//     tiled split-CSR layout (SideLayout): each tile of 32 consecutive rows keeps its rows of
//     at most kShortMax entries in a short CSR segment of at most kSegBudget entries (the
//     tile's longest rows move out until it fits), processed by one warp, one lane per row;
//     the other rows live in a long CSR cut into chunks that are whole-warp tasks.  Both kinds
//     end in the same per-row epilogue, executed by one lane per row so the FP64 work of the
//     epilogue (the method's elementwise part) runs with all 32 lanes active.
//   * Vectors are plain arrays indexed by row (m) or column (n) in the original order.
//   * A small control block (Ctl) holds the iteration counters, the restart decision, the step
//     data and the staged reduction results; kernels read it at entry and the last CTA of each
//     kernel updates it, so the restart test and the termination test never leave the device.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace rh {

constexpr int kWarp = 32;
constexpr int kTileRows = 32;          // rows per tile = lanes per warp
constexpr int kBlockWarps = 4;         // default warps per CTA of the tile kernels
constexpr int kBlockThreads = kBlockWarps * kWarp;
constexpr int kMaxBlockWarps = 16;     // widest CTA of the tile kernels (the width is a launch
                                       // parameter: walk and reductions read blockDim.x)
constexpr int kMaxBlockThreads = kMaxBlockWarps * kWarp;
constexpr int kMaxPartials = 20;       // reduction slots per CTA
constexpr int kShortMax = 128;         // rows with more entries are always long
constexpr int kSegBudget = 1024;       // entries of one tile's short segment (staging area)
constexpr int kMaxTileSmem = kMaxBlockWarps * (kSegBudget + 8) * 8;   // bytes, FP64 staging
                                                                      // at the widest CTA
constexpr int kChunk = 256;            // entries per long-row chunk (8 per lane)
constexpr int kStageUnroll = 2;        // 4-entry groups staged per lane per round
constexpr int kMaxTileMult = 4;        // most short tiles walked as one work item

// Walk instantiations of the ordinary mixed kernels: one tile per item; one tile per item with
// twice the staging unroll (row side only: long tiles, grid set by the tile count); groups of
// tiles per item (any layout).
enum WalkKind : int { kWalkPlain = 0, kWalkWide = 1, kWalkGrouped = 2 };
__host__ __device__ constexpr int walk_unroll(int walk) {
  return walk == kWalkWide ? 2 * kStageUnroll : kStageUnroll;
}

// Information bit of the problem validation: some upper bound u_j is finite.
constexpr unsigned int kHasFiniteUpper = 0x100u;

// Infeasibility certificate candidates (rhpdhg_result.cert_source).
enum CertSource : int { kCertNone = 0, kCertRestartPoint = 1, kCertCheck = 2, kCertAnchorMove = 3 };

enum Status : int {
  kRunning = 0, kOptimal = 1, kPrimalInfeasible = 2, kDualInfeasible = 3, kIterLimit = 4,
  kTimeLimit = 5, kNumericalError = 6, kCancelled = 7,
  kEscalate = 100   // internal: the mixed-precision solve continues in FP64 (never returned)
};

// Split-CSR structure of one side (see file comment).  The values live in separate arrays
// (FP64 and, for the mixed-precision path, FP32 copies share this structure).  Every short-row
// tile and every long row starts on a 4-entry (16-byte) boundary; the gaps are zero-filled
// padding that no row's range covers, so tiles and chunks can be read with 128-bit loads.  Long
// rows are further cut into chunks of at most kChunk entries; a chunk is one warp task.
struct SideLayout {
  int nrows = 0;
  int seg = 8;               // per-warp staging stride (entries): longest segment of a work
                             // item's tile group, rounded up to 4, plus 4
  int n_short_tiles = 0;     // ceil(nrows / 32)
  int n_long = 0;            // number of long rows
  int n_long_tiles = 0;      // ceil(n_long / 32): groups of 32 long rows sharing an epilogue
  int n_chunks = 0;          // chunks of the long rows
  const int *ptr_s = nullptr;       // nrows: start of each row in the short arrays (long: empty)
  const int *tile_end = nullptr;    // n_short_tiles: end of the last row of each tile (unpadded)
  const int *idx_s = nullptr;       // short entries (padded)
  const uint32_t *long_mask = nullptr;  // n_short_tiles words: bit r set if row 32t+r is long
  const int *long_rows = nullptr;   // n_long row ids (ascending)
  const int *beg_l = nullptr;       // n_long: start of each long row (4-aligned)
  const int *end_l = nullptr;       // n_long: end of each long row
  const int *idx_l = nullptr;       // long entries (padded, plus kChunk slack at the end)
  const int *chunk_ptr = nullptr;   // n_long + 1: chunks of long row i are [chunk_ptr[i], ..[i+1])
  const int *chunk_row = nullptr;   // n_chunks: long-row index of each chunk
  const int4 *chunk_desc = nullptr; // n_chunks: (long-row index, first entry, end entry, chunks
                                    // of its group of 32 long rows): one load per chunk item
  int tile_mult = 1;         // consecutive short tiles per work item (1 .. kMaxTileMult)
  int walk = 0;              // instantiation of the ordinary mixed kernels' walk (kWalk*)
  int cta_warps = kBlockWarps;  // warps per CTA of this side's iteration kernels (host only)
  int wide_rows = 0;         // FP64 walks sum a tile's longest rows warp-wide (tile_rows_fp64)
  int n_tile_groups = 0;     // ceil(n_short_tiles / tile_mult)
  __host__ __device__ int total_items() const { return n_chunks + n_tile_groups; }
};

// Values of one side in one precision.
template <typename VT>
struct SideVals {
  const VT *s = nullptr;     // nnz_short
  const VT *l = nullptr;     // nnz_long
};

// Per-walk scratch: chunk partial sums and group tickets (kept at zero between launches).  Two
// walks in the same kernel use two disjoint scratch sets.
struct WalkScratch {
  double *chunk_part = nullptr;       // n_chunks
  unsigned int *group_done = nullptr; // n_long_tiles
  double *group_part = nullptr;       // n_long_tiles * kMaxPartials: reduction slots of the
                                      // long-row epilogues of each group (see walk_tiles)
};

// An ordinary column stage that left its grid reduction to the next row kernel (see
// col_defers): its CTA rows of partials, its long-row groups' partials, and their counts.
struct DeferredCol {
  const double *part = nullptr;
  const double *gpart = nullptr;
  int nb = 0;
  int ngroups = 0;
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
  int col_deferred;      // 1: the last column stage left its reduction to the next row kernel
                         // (set by every CTA of that stage, which no column kernel reads;
                         // cleared by the row finaliser that applies it)
  double w;              // Halpern weight (k+1)/(k+2) of the pending blend
  double omega, tau, sigma, eta;
  double tau_inv, sigma_inv;   // 1 / tau, 1 / sigma (set with tau and sigma: the restart test
                               // multiplies instead of dividing on the narrow FP64 pipe)
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
  // column parts of the anchor-movement certificate candidate z^{n+1,0} - z^{n,0}, staged by
  // the column kernel of a restart decision (mv_ready = 1) for the row kernel that applies the
  // restart, which completes the test
  double mv_cd, mv_u, mv_l, mv_dlb, mv_dub, mv_au, mv_al;
  int mv_ready;
  int cert_src;          // candidate that certified infeasibility (kCert*)
  int near_cert;         // mixed precision: consecutive restart points whose candidate came
                         // within 1e-3 of certifying (two move the solve to FP64)
  int escalated;         // 1 once a mixed-precision solve continued in FP64
  // adaptive step rule: redo = 1 while iteration t is being recomputed with a smaller step
  // (the kernels then take z_t from the stored x, K^T y, y, K x); retries counts the attempts
  int redo, retries;
  double eta_next;
  // active-set telemetry of check iterations: columns with x~ on a bound, and columns whose
  // on-bound status changed since the previous check (integer atomics, reset by col_finalize)
  unsigned long long tel_act, tel_chg;
  long long act_last, chg_last;
  unsigned int cnt_row, cnt_col;   // last-CTA tickets
  int stage;             // 0: the row stage of iteration t is next; 1: the column stage is next
                         // (each finalisation advances it, so of two kernels launched for the
                         // same stage only the first one whose mode matches does the work)
};

// Primal and dual steps tau = eta / omega, sigma = eta omega and their reciprocals.
__host__ __device__ __forceinline__ void set_steps(Ctl *ctl, double eta, double omega) {
  ctl->tau = eta / omega;
  ctl->sigma = eta * omega;
  ctl->tau_inv = 1.0 / ctl->tau;
  ctl->sigma_inv = 1.0 / ctl->sigma;
}

struct TraceRec {      // mirrors rhpdhg_trace_rec
  long long t, epoch, k;
  double fpr_sq, omega;
  int restart, retries;        // retries: rejected step sizes before this iteration's step
  long long active, changed;   // check iterations: active-set telemetry, else -1
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
  int mixed;                  // 1 = FP32-offset iterates (certificates escalate to FP64)
  int bf16;                   // mixed: 1 = BF16 matrix values in the ordinary kernels
  int no_upper;               // 1 = every u_j is +inf: the mixed kernels do not read the
                              // FP32 upper-bound offsets (all +inf)
  int df_sums;                // mixed: 1 = double-float restart-norm sums from the lane up,
                              // 0 = FP32 sums at every level
  int adaptive;               // 1 = adaptive step rule (inadmissible steps are redone)
  int l2_first;               // mixed: 1 = the ordinary kernels read the matrix stream with the
                              // L2 evict-first policy (one iteration's bytes exceed L2)
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

// ---------------------------------------------------------------------------------------------
// Double-float sums.  The FP64 pipe of this part is narrow (about 2 FP64 operations per clock per
// SM, against 128 FP32), so the per-iteration sums of the mixed-precision kernels are carried as
// double-floats: an unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2), updated
// with error-free transformations on the FP32 pipe.  Products of two FP32 numbers are exact
// (FMA-based TwoProd) and a sum of double-floats has a relative error of at most 3 u^2 with
// u = 2^-24 (Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", 2017, Algorithm 6), so the sums carry about 46 bits where
// plain FP32 sums carry 24.  The _rn intrinsics keep the compiler from contracting or
// reassociating the transformations.

struct DF {
  float hi, lo;
};

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker's Fast2Sum)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ DF df_add(DF x, DF y) {
  float sh, sl, th, tl, vh, vl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  fast_two_sum(sh, __fadd_rn(sl, th), vh, vl);
  DF z;
  fast_two_sum(vh, __fadd_rn(tl, vl), z.hi, z.lo);
  return z;
}

// a * b exactly (while the product neither overflows nor underflows FP32)
__device__ __forceinline__ DF df_prod(float a, float b) {
  DF r;
  r.hi = __fmul_rn(a, b);
  r.lo = __fmaf_rn(a, b, -r.hi);
  return r;
}

__device__ __forceinline__ DF df_warp_sum(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, w);
  }
  return v;
}

// The packed slots carry either double-floats (EXACT) or plain FP32 sums in hi (lo = 0), which
// the same reductions add with single FP32 additions: the FP32 option of the mixed-precision
// restart-norm sums, whose dependent chains in the grid reduction stay short.
template <bool EXACT>
__device__ __forceinline__ DF dfx_add(DF x, DF y) {
  if constexpr (EXACT) return df_add(x, y);
  else return DF{__fadd_rn(x.hi, y.hi), 0.f};
}
template <bool EXACT>
__device__ __forceinline__ DF dfx_warp_sum(DF v) {
  if constexpr (EXACT) return df_warp_sum(v);
  else return DF{warp_sum(v.hi), 0.f};
}

// A double-float travels through the 8-byte partial slots bit-packed (no FP64 arithmetic).
__device__ __forceinline__ double df_pack(DF a) {
  return __hiloint2double(__float_as_int(a.hi), __float_as_int(a.lo));
}
__device__ __forceinline__ DF df_unpack(double v) {
  DF r;
  r.hi = __int_as_float(__double2hiint(v));
  r.lo = __int_as_float(__double2loint(v));
  return r;
}
__device__ __forceinline__ double df_value(DF a) { return (double)a.hi + (double)a.lo; }

// Per-thread accumulators of NS sums and NM maxima, reduced per CTA in a fixed order.  The first
// ND sums are packed slots (d[0 .. ND-1]; s[0 .. ND-1] are unused): double-floats when EXACT,
// plain FP32 sums otherwise; the others are FP64.
template <int NS, int NM, int ND = 0, bool EXACT = true>
struct Acc {
  double s[NS > 0 ? NS : 1];
  double mx[NM > 0 ? NM : 1];
  DF d[ND > 0 ? ND : 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = 0.0;
#pragma unroll
    for (int i = 0; i < NM; ++i) mx[i] = 0.0;
#pragma unroll
    for (int i = 0; i < ND; ++i) d[i] = DF{0.f, 0.f};
  }
};

// Per-warp results of a CTA-level reduction; cta_reduce_and_ticket and grid_finish use it one
// after the other (each ends with a barrier).
__device__ __forceinline__ double (*cta_red())[kMaxPartials] {
  __shared__ double red[kMaxBlockWarps][kMaxPartials];
  return red;
}

// Reduce Acc over the CTA (deterministic: fixed shuffle tree, warps summed in index order) and
// write the CTA's partials to part[blockIdx.x * kMaxPartials + slot] (double-float slots
// bit-packed).  Only the slots set in smask (sums) and mmask (maxima) are reduced and written;
// slots set in prewarp hold, in lane 0, a value already summed over the warp (FP64 slots only).
// Returns true in every thread of the last CTA to finish (after a fence), which then owns the
// grid-level reduction.
template <int NS, int NM, int ND, bool EXACT, bool TICKET = true>
__device__ bool cta_reduce_and_ticket(Acc<NS, NM, ND, EXACT> &a, unsigned smask, unsigned mmask,
                                      unsigned prewarp, double *part, unsigned int *ticket) {
  double (*red)[kMaxPartials] = cta_red();
  __shared__ bool last;
  static_assert(NS + NM <= kMaxPartials, "too many partial slots");
  static_assert(ND <= NS, "double-float slots are sums");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    if (!((smask >> i) & 1u)) continue;
    if (i < ND) {
      const DF v = dfx_warp_sum<EXACT>(a.d[i < ND ? i : 0]);
      if (lane == 0) red[warp][i] = df_pack(v);
    } else {
      const double v = ((prewarp >> i) & 1u) ? a.s[i] : warp_sum(a.s[i]);
      if (lane == 0) red[warp][i] = v;
    }
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    if (!((mmask >> i) & 1u)) continue;
    const double v = warp_max(a.mx[i]);
    if (lane == 0) red[warp][NS + i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double *dst = part + (size_t)blockIdx.x * kMaxPartials;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      if (!((smask >> i) & 1u)) continue;
      if (i < ND) {
        DF v = df_unpack(red[0][i]);
        for (int w = 1; w < nw; ++w) v = dfx_add<EXACT>(v, df_unpack(red[w][i]));
        dst[i] = df_pack(v);
      } else {
        double v = red[0][i];
        for (int w = 1; w < nw; ++w) v += red[w][i];
        dst[i] = v;
      }
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      if (!((mmask >> i) & 1u)) continue;
      double v = red[0][NS + i];
      for (int w = 1; w < nw; ++w) v = fmax(v, red[w][NS + i]);
      dst[NS + i] = v;
    }
    if constexpr (TICKET) {
      __threadfence();
      const unsigned int tk = atomicAdd(ticket, 1u);
      last = (tk == gridDim.x - 1);
    }
  }
  if constexpr (TICKET) {
    __syncthreads();
    if (last) __threadfence();
    return last;
  } else {
    return false;
  }
}

// The CTA-level half of cta_reduce_and_ticket: the CTA's row of partials is written and no ticket
// is taken (the row is reduced by a later kernel, after this one has completed).
template <int NS, int NM, int ND, bool EXACT>
__device__ void cta_reduce_store(Acc<NS, NM, ND, EXACT> &a, unsigned smask, unsigned mmask,
                                 double *part) {
  cta_reduce_and_ticket<NS, NM, ND, EXACT, false>(a, smask, mmask, 0u, part, nullptr);
}

// Warp-collective: reduce the long-row sums al of every lane and store them as group grp's
// partials (lane 0; double-float slots bit-packed), then clear al.  Only sums need this (their
// order decides the rounding); long-row maxima are taken into the finishing warp's own
// accumulator.
template <int NS, int ND, bool EXACT>
__device__ __forceinline__ void store_group(Acc<NS, 0, ND, EXACT> &al, unsigned smask,
                                            double *gpart, int grp) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    if (!((smask >> i) & 1u)) continue;
    if (i < ND) {
      const DF v = dfx_warp_sum<EXACT>(al.d[i < ND ? i : 0]);
      if (lane == 0) gpart[(size_t)grp * kMaxPartials + i] = df_pack(v);
    } else {
      const double v = warp_sum(al.s[i]);
      if (lane == 0) gpart[(size_t)grp * kMaxPartials + i] = v;
    }
  }
  al.zero();
}

// In the last CTA: reduce the grid's partials in block order, then the long-row groups'
// partials in group order, for the slots in the masks (others return 0; the first ND sums are
// double-floats, returned as hi + lo).  out[i] valid in all threads.
//
// Thread t sums blocks t, t + blockDim, ... of each slot in that order, then groups t,
// t + blockDim, ...; each warp reduces its lanes with a fixed shuffle tree and the warps' results
// are added in warp order, so the result does not depend on how the loads are scheduled.  The
// reads are latency-bound (a few values per thread from L2, possibly on the other die) and the
// last CTA's time is set by the number of dependent round trips.  Two schedules: block by block
// with all active slots of a block in flight (ceil(nb / blockDim) rounds), or slot by slot with
// kGridBatch blocks in flight (about one round per active slot); the one with fewer rounds runs.
// BATCH = false keeps only the first (the FP64 kernels: ALU-bound, with fewer CTAs, where the
// second gains nothing and its registers cost).
constexpr int kGridBatch = 10;
template <int NS, int NM, bool BATCH = true, int ND = 0, bool EXACT = true>
__device__ void grid_finish(const double *part, double *out, unsigned smask, unsigned mmask,
                            const double *gpart = nullptr, int ngroups = 0, int nrows = -1) {
  double (*red)[kMaxPartials] = cta_red();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = nrows >= 0 ? nrows : (int)gridDim.x;   // rows of part (default: this grid's)
  double v[NS + NM];
  DF vd[ND > 0 ? ND : 1];
#pragma unroll
  for (int i = 0; i < NS + NM; ++i) v[i] = 0.0;
#pragma unroll
  for (int i = 0; i < ND; ++i) vd[i] = DF{0.f, 0.f};
  // one partial p of slot i into the thread's running value
  auto take = [&](int i, double p) {
    if (i < ND) vd[i < ND ? i : 0] = dfx_add<EXACT>(vd[i < ND ? i : 0], df_unpack(p));
    else v[i] = (i < NS) ? v[i] + p : fmax(v[i], p);
  };
  const unsigned all = smask | (mmask << NS);
  const int rounds_by_block = (nb + (int)blockDim.x - 1) / (int)blockDim.x;
  if (!BATCH || rounds_by_block <= __popc(all)) {
#pragma unroll 4
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const double *src = part + (size_t)b * kMaxPartials;
#pragma unroll
      for (int i = 0; i < NS + NM; ++i) {
        if (!((all >> i) & 1u)) continue;
        take(i, __ldcg(src + i));
      }
    }
  } else {
    for (int b0 = threadIdx.x; b0 < nb; b0 += kGridBatch * blockDim.x) {
#pragma unroll
      for (int i = 0; i < NS + NM; ++i) {
        if (!((all >> i) & 1u)) continue;
        double p[kGridBatch];
#pragma unroll
        for (int j = 0; j < kGridBatch; ++j) {
          const int b = b0 + j * blockDim.x;
          p[j] = b < nb ? __ldcg(part + (size_t)b * kMaxPartials + i) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < kGridBatch; ++j) take(i, p[j]);
      }
    }
  }
  // groups hold sums only (long-row maxima go straight to the finishing warp's CTA partials)
  for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const double *src = gpart + (size_t)g * kMaxPartials;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      if (!((smask >> i) & 1u)) continue;
      take(i, __ldcg(src + i));
    }
  }
#pragma unroll
  for (int i = 0; i < NS + NM; ++i) {
    if (!((all >> i) & 1u)) continue;
    if (i < ND) {
      const DF r = dfx_warp_sum<EXACT>(vd[i < ND ? i : 0]);
      if (lane == 0) red[warp][i] = df_pack(r);
    } else {
      const double r = (i < NS) ? warp_sum(v[i]) : warp_max(v[i]);
      if (lane == 0) red[warp][i] = r;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NS + NM; ++i) {
    if (!((all >> i) & 1u)) { out[i] = 0.0; continue; }
    if (i < ND) {
      DF r = df_unpack(red[0][i]);
      for (int w = 1; w < nw; ++w) r = dfx_add<EXACT>(r, df_unpack(red[w][i]));
      out[i] = df_value(r);
    } else {
      double r = red[0][i];
      for (int w = 1; w < nw; ++w) r = (i < NS) ? r + red[w][i] : fmax(r, red[w][i]);
      out[i] = r;
    }
  }
  __syncthreads();
}

// The last CTA of a row kernel adds a deferred column stage's two sums (see DeferredCol) after
// its own grid reduction.  dcol_prefetch issues, before that reduction, the loads of the first
// kDcolPre column rows of each thread (t, t + blockDim, ...), so that their latency overlaps the
// row reduction's; dcol_finish adds them, any further rows and the column's long-row groups in
// the order grid_finish uses (a thread's rows in index order, then its groups; lanes by the
// shuffle tree; warps in index order), and returns the sums (the first ND double-floats) in
// every thread.
constexpr int kDcolPre = 4;
constexpr int kDcolBatch = 6;
struct DcolPre {
  double p[kDcolPre][2];
};

__device__ __forceinline__ void dcol_prefetch(const DeferredCol &dc, DcolPre &pre) {
#pragma unroll
  for (int j = 0; j < kDcolPre; ++j) {
    const int b = (int)threadIdx.x + j * (int)blockDim.x;
    const double *src = dc.part + (size_t)b * kMaxPartials;
    pre.p[j][0] = b < dc.nb ? __ldcg(src) : 0.0;
    pre.p[j][1] = b < dc.nb ? __ldcg(src + 1) : 0.0;
  }
}

template <int ND, bool EXACT>
__device__ void dcol_finish(const DeferredCol &dc, const DcolPre &pre, double *out) {
  double (*red)[kMaxPartials] = cta_red();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double v[2] = {0.0, 0.0};
  DF vd[2] = {DF{0.f, 0.f}, DF{0.f, 0.f}};
  auto take = [&](int i, double p) {
    if (i < ND) vd[i] = dfx_add<EXACT>(vd[i], df_unpack(p));
    else v[i] += p;
  };
#pragma unroll
  for (int j = 0; j < kDcolPre; ++j) {
    if ((int)threadIdx.x + j * (int)blockDim.x >= dc.nb) break;
    take(0, pre.p[j][0]);
    take(1, pre.p[j][1]);
  }
  // further rows kDcolBatch at a time, all in flight together
  const int bd = (int)blockDim.x;
  for (int b0 = (int)threadIdx.x + kDcolPre * bd; b0 < dc.nb; b0 += kDcolBatch * bd) {
    double q[kDcolBatch][2];
#pragma unroll
    for (int j = 0; j < kDcolBatch; ++j) {
      const int b = b0 + j * bd;
      const double *src = dc.part + (size_t)b * kMaxPartials;
      q[j][0] = b < dc.nb ? __ldcg(src) : 0.0;
      q[j][1] = b < dc.nb ? __ldcg(src + 1) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kDcolBatch; ++j) {
      if (b0 + j * bd >= dc.nb) break;
      take(0, q[j][0]);
      take(1, q[j][1]);
    }
  }
  for (int g = threadIdx.x; g < dc.ngroups; g += blockDim.x) {
    const double *src = dc.gpart + (size_t)g * kMaxPartials;
    take(0, __ldcg(src));
    take(1, __ldcg(src + 1));
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (i < ND) {
      const DF r = dfx_warp_sum<EXACT>(vd[i]);
      if (lane == 0) red[warp][i] = df_pack(r);
    } else {
      const double r = warp_sum(v[i]);
      if (lane == 0) red[warp][i] = r;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (i < ND) {
      DF r = df_unpack(red[0][i]);
      for (int w = 1; w < nw; ++w) r = dfx_add<EXACT>(r, df_unpack(red[w][i]));
      out[i] = df_value(r);
    } else {
      double r = red[0][i];
      for (int w = 1; w < nw; ++w) r += red[w][i];
      out[i] = r;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// The tile walker: computes dot = (row of the side operator) . src for every row and calls
// epi(row, dot, is_long) once per row, from one lane, 32 rows per warp at a time.  Work items are
// the chunks of the long rows followed by the short-row tiles (or groups of tile_mult consecutive
// tiles), distributed over all warps of the grid round robin (so two walks over the same
// structure give every row to the same warp and lane).
//   * A chunk's warp reads its (<= 256) entries as 32 contiguous bytes of indices and values per
//     lane, sums them (fixed shuffle tree) into chunk_part and takes a ticket; the warp that
//     completes the last chunk of a group of 32 long rows (no waiting) adds each row's chunk
//     partials in chunk order, runs the 32 epilogues lane-parallel and calls gdone(group).
//   * A short tile stages the products of its 16-byte-aligned entry segment in shared memory
//     (128-bit index / value loads, 4 U gathers per lane in flight), then lane r sums
//     row r's products with four interleaved accumulators.
// VT is the value type, PT the product/accumulator type; src(j) returns the gathered vector
// entry; smem is this warp's staging area of 32 * L + 4 PTs.

// Cache policy of the matrix stream (template parameter CP of the walk).  CP = 1 reads the
// entries with an L2 evict-first policy: where one iteration's bytes exceed L2 they stream through
// once per product, and the policy leaves L2 to the gathered vectors and the reduction partials.
// Where the problem fits L2 the plain loads (CP = 0) are kept: there the evict-first lines were
// measured to cost re-reads; BF16 values keep them too (the hinted 8-byte loads measured slower).  The policy is created next to each load from an immediate, which
// the compiler keeps a constant (a policy selected at run time measured slower).
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <typename VT>
struct Vec4;
template <>
struct Vec4<float> {
  float v[4];
  template <int CP = 0>
  __device__ __forceinline__ void load(const float *p) {
    if constexpr (CP == 1) {
      asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
          : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
          : "l"(p), "l"(l2_evict_first()));
    } else {
      const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
  }
};
// BF16 values (exact images of a matrix whose entries have at most 8 significant bits, scaled by
// powers of two), widened to FP32 as they are loaded: 8 bytes per 4 entries.
template <>
struct Vec4<__nv_bfloat16> {
  float v[4];
  template <int CP = 0>
  __device__ __forceinline__ void load(const __nv_bfloat16 *p) {
    static_assert(CP == 0, "BF16 values are read with plain loads");
    const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
    v[0] = __uint_as_float(t.x << 16);
    v[1] = __uint_as_float(t.x & 0xFFFF0000u);
    v[2] = __uint_as_float(t.y << 16);
    v[3] = __uint_as_float(t.y & 0xFFFF0000u);
  }
};
template <>
struct Vec4<double> {
  double v[4];
  template <int CP = 0>
  __device__ __forceinline__ void load(const double *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

template <int CP = 0>
__device__ __forceinline__ void load_idx4(const int *p, int *j) {
  if constexpr (CP == 1) {
    asm("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(j[0]), "=r"(j[1]), "=r"(j[2]), "=r"(j[3])
        : "l"(p), "l"(l2_evict_first()));
  } else {
    const int4 t = __ldg(reinterpret_cast<const int4 *>(p));
    j[0] = t.x; j[1] = t.y; j[2] = t.z; j[3] = t.w;
  }
}

// One long-row chunk (work item `item` < lay.n_chunks) of walk_tiles, by the whole warp.
template <typename VT, typename PT, int CP, typename Src, typename Epi, typename GroupDone>
__device__ __forceinline__ void walk_chunk(const SideLayout &lay, const SideVals<VT> vals,
                                           const Src &src, const WalkScratch ws, Epi &epi,
                                           GroupDone &gdone, int item) {
  const int lane = threadIdx.x & 31;
  const int4 dsc = __ldg(lay.chunk_desc + item);
  const int li = dsc.x;
  const int cb = dsc.y;                                   // 4-aligned
  const int ce = dsc.z;
  // lane reads entries [p0, p0 + 8): two 16-byte index loads, 16 or 32 bytes of values
  const int p0 = cb + 8 * lane;
  PT s = PT(0);
  if (p0 < ce) {
    int j[8];
    Vec4<VT> va, vb;
    load_idx4<CP>(lay.idx_l + p0, j);
    load_idx4<CP>(lay.idx_l + p0 + 4, j + 4);
    va.template load<CP>(vals.l + p0);
    vb.template load<CP>(vals.l + p0 + 4);
    PT x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (p0 + u < ce) ? PT(src(j[u])) : PT(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) s += PT(va.v[u]) * x[u];
#pragma unroll
    for (int u = 0; u < 4; ++u) s += PT(vb.v[u]) * x[4 + u];
  }
  s = warp_sum(s);
  const int grp = li / kTileRows;
  const int g0 = grp * kTileRows;
  const int g1 = min(g0 + kTileRows, lay.n_long);
  int fin = 0;
  if (lane == 0) {
    ws.chunk_part[item] = (double)s;
    __threadfence();
    const unsigned int need = (unsigned int)dsc.w;
    const unsigned int old = atomicAdd(ws.group_done + grp, 1u);
    fin = (old == need - 1) ? 1 : 0;
  }
  fin = __shfl_sync(0xffffffffu, fin, 0);
  if (fin) {
    __threadfence();
    const int lr = g0 + lane;
    if (lr < g1) {
      // the row's chunk partials, added in chunk order; loaded eight at a time so that a long
      // row's loads are in flight together (a row has up to 5000 / 256 chunks)
      PT d = PT(0);
      const int c1 = lay.chunk_ptr[lr + 1];
      for (int c = lay.chunk_ptr[lr]; c < c1; c += 8) {
        double p[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) p[u] = c + u < c1 ? __ldcg(ws.chunk_part + c + u) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c + u < c1) d += PT(p[u]);
      }
      epi(lay.long_rows[lr], d, true);
    }
    // the finishing warp varies from run to run: the group's reduction contributions go to the
    // group's own slots, which the last CTA adds in group order
    gdone(grp);
    if (lane == 0) ws.group_done[grp] = 0u;
  }
}

// FP64 tiles: the FP64 pipe is narrow, and lane-per-row sums issue as many FP64 adds per warp as
// the tile's longest row has entries, with the other lanes masked.  Rows longer than a threshold
// T are therefore summed by the whole warp (lane-strided partial sums and a shuffle tree, about
// len/32 + 5 adds per row), the rest lane per row as in tile_rows.  T is the candidate among 8,
// 16, 32 and the longest row that minimises the warp's FP64 adds, 4 ceil(T / 4) + the sum over
// rows longer than T of (ceil(len / 32) + 5) (one warp reduction per candidate); a tile whose rows
// have at most 16 entries keeps T = its longest row.  Rows at or below T are summed exactly as
// tile_rows sums them.  Used only on sides where the same cost model, evaluated over all tiles at
// set-up, saves FP64 adds (SideLayout::wide_rows); elsewhere tile_rows keeps lane-per-row sums.
template <typename Epi>
__device__ __forceinline__ void tile_rows_fp64(const double *smem, int row0, int nr, int rb,
                                               int re, int seg_b, uint32_t lm, Epi &epi) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool act = lane < nr && !((lm >> lane) & 1u);
  const int len = act ? re - rb : 0;           // at most kShortMax
  const int mx = (int)__reduce_max_sync(full, (unsigned)len);
  int T = mx;
  if (mx > 16) {
    int best = (mx + 3) & ~3;
    const int wadds = ((len + 31) >> 5) + 5;   // this row's adds when summed by the warp
#pragma unroll
    for (int c = 8; c <= 32; c *= 2) {
      if (c >= mx) break;
      const int cost = c + (int)__reduce_add_sync(full, len > c ? (unsigned)wadds : 0u);
      if (cost < best) {
        best = cost;
        T = c;
      }
    }
  }
  double dot = 0.0;
  if (act && len <= T) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int p = rb - seg_b;
    const int pe = re - seg_b;
    for (; p + 4 <= pe; p += 4) {
      s0 += smem[p];
      s1 += smem[p + 1];
      s2 += smem[p + 2];
      s3 += smem[p + 3];
    }
    if (p < pe) s0 += smem[p];
    if (p + 1 < pe) s1 += smem[p + 1];
    if (p + 2 < pe) s2 += smem[p + 2];
    dot = (s0 + s1) + (s2 + s3);
  }
  unsigned big = __ballot_sync(full, act && len > T);
  while (big) {
    const int r = __ffs(big) - 1;
    big &= big - 1;
    const int b = __shfl_sync(full, rb, r) - seg_b, e = __shfl_sync(full, re, r) - seg_b;
    double s = 0.0;
    for (int p = b + lane; p < e; p += 32) s += smem[p];
    s = warp_sum(s);
    if (lane == r) dot = s;
  }
  // one converged epilogue pass (split into the short rows' and the long rows' lanes, the FP64
  // epilogue issued twice and measured slower)
  if (act) epi(row0 + lane, dot, false);
}

// Lane r of a short tile sums row r's staged products smem[rb - seg_b, re - seg_b) with four
// interleaved accumulators and runs its epilogue (rows marked long in lm are skipped).  FP64
// tiles go to tile_rows_fp64.
template <typename PT, typename Epi>
__device__ __forceinline__ void tile_rows(const PT *smem, int row0, int nr, int rb, int re,
                                          int seg_b, uint32_t lm, bool wide, Epi &epi) {
  // (without the warp-wide sums each lane goes on to its epilogue as soon as its row is summed,
  // so its loads overlap the other lanes' sums)
  if constexpr (sizeof(PT) == sizeof(double)) {
    if (wide) {
      tile_rows_fp64(smem, row0, nr, rb, re, seg_b, lm, epi);
      return;
    }
  }
  {
    const int lane = threadIdx.x & 31;
    if (lane < nr && !((lm >> lane) & 1u)) {
      PT s0 = PT(0), s1 = PT(0), s2 = PT(0), s3 = PT(0);
      int p = rb - seg_b;
      const int pe = re - seg_b;
      for (; p + 4 <= pe; p += 4) {
        s0 += smem[p];
        s1 += smem[p + 1];
        s2 += smem[p + 2];
        s3 += smem[p + 3];
      }
      if (p < pe) s0 += smem[p];
      if (p + 1 < pe) s1 += smem[p + 1];
      if (p + 2 < pe) s2 += smem[p + 2];
      epi(row0 + lane, (s0 + s1) + (s2 + s3), false);
    }
  }
}


// Prefetch of the line holding *p into L1 (no register is held while it is in flight).
__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Default per-row prefetch hook of walk_tiles: none.
struct NoPrefetch {
  __device__ __forceinline__ void operator()(int) const {}
};

// Stage the products of the segment [seg_b, seg_e) (seg_b 4-aligned) in smem[0, ...): lane
// handles 4-entry groups g = lane, lane + 32, ..., U at a time (more loads in flight per round,
// more registers).
template <typename VT, typename PT, int U, int CP, typename Src>
__device__ __forceinline__ void stage_segment(const SideLayout &lay, const SideVals<VT> vals,
                                              const Src &src, PT *smem, int seg_b, int seg_e) {
  const int lane = threadIdx.x & 31;
  const int nvec = (seg_e - seg_b + 3) >> 2;             // groups of 4 entries
  constexpr int kU = U;
  for (int g0 = 0; g0 < nvec; g0 += kWarp * kU) {
    int j[kU][4];
    Vec4<VT> vv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int g = g0 + u * kWarp + lane;
      if (g < nvec) {
        load_idx4<CP>(lay.idx_s + seg_b + 4 * g, j[u]);
        vv[u].template load<CP>(vals.s + seg_b + 4 * g);
      }
    }
    PT x[kU][4];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int g = g0 + u * kWarp + lane;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        x[u][e] = (g < nvec && seg_b + 4 * g + e < seg_e) ? PT(src(j[u][e])) : PT(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int g = g0 + u * kWarp + lane;
      if (g < nvec) {
#pragma unroll
        for (int e = 0; e < 4; ++e) smem[4 * g + e] = PT(vv[u].v[e]) * x[u][e];
      }
    }
  }
}

// One short tile st of walk_tiles (tile_mult == 1): stage its segment, then lane r sums row r
// and runs its epilogue.
template <typename VT, typename PT, int U, int CP, typename Src, typename Epi, typename Pre>
__device__ __forceinline__ void walk_tile(const SideLayout &lay, const SideVals<VT> vals,
                                          const Src &src, PT *smem, Epi &epi, const Pre &pre,
                                          int st) {
  const int lane = threadIdx.x & 31;
  const int row0 = st * kTileRows;
  const int nr = min(kTileRows, lay.nrows - row0);
  if (lane < nr) pre(row0 + lane);
  const int rb = lay.ptr_s[row0 + min(lane, nr - 1)];
  const int seg_e = lay.tile_end[st];
  const int seg_b = __shfl_sync(0xffffffffu, rb, 0);     // 4-aligned
  int re = __shfl_down_sync(0xffffffffu, rb, 1);
  if (lane >= nr - 1) re = seg_e;
  stage_segment<VT, PT, U, CP>(lay, vals, src, smem, seg_b, seg_e);
  __syncwarp();
  tile_rows<PT>(smem, row0, nr, rb, re, seg_b, lay.long_mask[st], lay.wide_rows != 0, epi);
  __syncwarp();
}

// GROUPED = false is the walk of layouts with tile_mult == 1 only (one tile per item, fewer
// registers); GROUPED = true walks any layout.
// pre(row) is called by the lane of each short-tile row before the tile's entries are staged,
// so that what the row's epilogue will read can be requested while the staging round trips run.
template <typename VT, typename PT, bool GROUPED = true, int U = kStageUnroll, int CP = 0,
          typename Src, typename Epi, typename GroupDone, typename Pre = NoPrefetch>
__device__ __forceinline__ void walk_tiles(const SideLayout &lay, const SideVals<VT> vals,
                                           const Src &src, PT *smem, const WalkScratch ws,
                                           Epi &epi, GroupDone &gdone,
                                           const Pre &pre = Pre()) {
  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int total = lay.total_items();
  for (int item = gwarp; item < total; item += nwarps) {
    if (item < lay.n_chunks) {
      walk_chunk<VT, PT, CP>(lay, vals, src, ws, epi, gdone, item);
    } else if constexpr (!GROUPED) {
      walk_tile<VT, PT, U, CP>(lay, vals, src, smem, epi, pre, item - lay.n_chunks);
    } else {
      // a group of nt <= tile_mult consecutive short tiles, staged as one segment
      const int t0 = (item - lay.n_chunks) * lay.tile_mult;
      const int nt = min(lay.tile_mult, lay.n_short_tiles - t0);
      for (int r = t0 * kTileRows + lane; r < min((t0 + nt) * kTileRows, lay.nrows); r += kWarp)
        pre(r);
      // the tiles' row starts (requested into L1 for the row sums), ends and long-row masks
      for (int m = 1; m < nt; ++m) {
        const int row0 = (t0 + m) * kTileRows;
        prefetch_l1(lay.ptr_s + row0 + min(lane, lay.nrows - 1 - row0));
      }
      int te = 0;
      uint32_t lmk = 0u;
      if (lane < nt) {
        te = lay.tile_end[t0 + lane];
        lmk = lay.long_mask[t0 + lane];
      }
      const int rb0 = lay.ptr_s[t0 * kTileRows + min(lane, lay.nrows - 1 - t0 * kTileRows)];
      const int seg_b = __shfl_sync(0xffffffffu, rb0, 0);     // 4-aligned
      const int seg_e = __shfl_sync(0xffffffffu, te, nt - 1);
      stage_segment<VT, PT, U, CP>(lay, vals, src, smem, seg_b, seg_e);
      __syncwarp();
#pragma unroll 1
      for (int m = 0; m < nt; ++m) {
        const int row0 = (t0 + m) * kTileRows;
        const int nr = min(kTileRows, lay.nrows - row0);
        const int rb = m == 0 ? rb0 : lay.ptr_s[row0 + min(lane, nr - 1)];
        const int te_m = __shfl_sync(0xffffffffu, te, m);
        const uint32_t lm_m = __shfl_sync(0xffffffffu, lmk, m);
        int re = __shfl_down_sync(0xffffffffu, rb, 1);
        if (lane >= nr - 1) re = te_m;
        tile_rows<PT>(smem, row0, nr, rb, re, seg_b, lm_m, lay.wide_rows != 0, epi);
      }
      __syncwarp();
    }
  }
}

}  // namespace rh
