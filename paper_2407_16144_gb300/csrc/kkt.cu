// Standalone evaluation of the relative KKT error of a point (x, y) of an LP held in device
// memory: the termination measure of the solver (Section 7, "Termination criteria"; the l2 form
// described in include/rhpdhg.h), available to callers who want to check any point.
//
//   rel_p   = || (b - A x, (h - G x)^+) ||_2 / (1 + ||q||_2)
//   rel_d   = || c - K^T y - lambda ||_2 / (1 + ||c||_2),  lambda = proj_Lambda(c - K^T y)
//   rel_gap = |p - d| / (1 + |p| + |d|),  p = c^T x + off,  d = q^T y + sum(l lambda^+ - u lambda^-) + off
//
// K^T y is formed by scattering each row's contribution (atomic FP64 adds) into an n-vector of
// scratch, so only the CSR of K is needed; the sums are then reduced per block into scratch
// partials and finished by one block.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/rhpdhg.h"
#include "internal.h"

namespace rh {

namespace {

constexpr int kKktThreads = 256;
constexpr int kKktSlots = kKktSlotCount;   // stride of a block's partials
constexpr int kKktUsed = 7;                // 0 rp2, 1 qy, 2 qq, 3 rd2, 4 cx, 5 bnd, 6 cc
constexpr int kKktFlag = 5;                // dout[5]: 1 if the CSR held an index out of range

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kKktThreads / 32; ++w) r += sh[w];
  return r;   // valid in thread 0
}

// Rows whose offsets fall outside [0, nnz] or decrease, and entries whose column lies outside
// [0, n), are skipped and reported through flag (the caller's CSR is not validated beforehand).
__global__ void __launch_bounds__(kKktThreads)
k_kkt_rows(int m, int m_eq, int n, long long nnz, const long long *rp, const int *col,
           const double *val, const double *x, const double *y, const double *q, double *kty,
           double *part, double *flag) {
  __shared__ double sh[kKktThreads / 32];
  double s_rp2 = 0.0, s_qy = 0.0, s_qq = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const double yi = y[i], qi = q[i];
    double kx = 0.0;
    long long p0 = rp[i], p1 = rp[i + 1];
    if (p0 < 0 || p1 < p0 || p1 > nnz) {
      *flag = 1.0;
      p1 = p0;
    }
    for (long long p = p0; p < p1; ++p) {
      const int j = col[p];
      if (j < 0 || j >= n) {
        *flag = 1.0;
        continue;
      }
      kx += val[p] * x[j];
      atomicAdd(kty + j, val[p] * yi);
    }
    double r = qi - kx;
    if (i >= m_eq) r = fmax(r, 0.0);
    s_rp2 += r * r;
    s_qy += qi * yi;
    s_qq += qi * qi;
  }
  const double a = block_sum(s_rp2, sh), b = block_sum(s_qy, sh), c = block_sum(s_qq, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * kKktSlots + 0] = a;
    part[blockIdx.x * kKktSlots + 1] = b;
    part[blockIdx.x * kKktSlots + 2] = c;
  }
}

__global__ void __launch_bounds__(kKktThreads)
k_kkt_cols(int n, const double *c, const double *l, const double *u, const double *x,
           const double *kty, double *part) {
  __shared__ double sh[kKktThreads / 32];
  double s_rd2 = 0.0, s_cx = 0.0, s_bnd = 0.0, s_cc = 0.0;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const double cj = c[j], lj = l[j], uj = u[j];
    const double g = cj - kty[j];
    const bool lf = isfinite(lj), uf = isfinite(uj);
    double lam = 0.0;
    if (lf && uf) lam = g;
    else if (lf) lam = fmax(g, 0.0);
    else if (uf) lam = fmin(g, 0.0);
    const double rd = g - lam;
    s_rd2 += rd * rd;
    s_cx += cj * x[j];
    if (lam > 0.0) s_bnd += lj * lam;
    else if (lam < 0.0) s_bnd += uj * lam;
    s_cc += cj * cj;
  }
  const double a = block_sum(s_rd2, sh), b = block_sum(s_cx, sh), d = block_sum(s_bnd, sh),
               e = block_sum(s_cc, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * kKktSlots + 3] = a;
    part[blockIdx.x * kKktSlots + 4] = b;
    part[blockIdx.x * kKktSlots + 5] = d;
    part[blockIdx.x * kKktSlots + 6] = e;
  }
}

__global__ void k_kkt_final(int nb, const double *part, double off, double *out) {
  // one thread per used slot, blocks summed in order
  __shared__ double tot[kKktUsed];
  if (threadIdx.x < kKktUsed) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b * kKktSlots + threadIdx.x];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double rel_p = sqrt(tot[0]) / (1.0 + sqrt(tot[2]));
    const double rel_d = sqrt(tot[3]) / (1.0 + sqrt(tot[6]));
    const double p = tot[4] + off, d = tot[1] + tot[5] + off;
    out[0] = rel_p;
    out[1] = rel_d;
    out[2] = fabs(p - d) / (1.0 + fabs(p) + fabs(d));
    out[3] = p;
    out[4] = d;
  }
}

__global__ void k_kkt_zero(int n, double *v, double *flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0.0;
}


}  // namespace

int kkt_blocks(int m, int n) {
  const int need = ((m > n ? m : n) + kKktThreads - 1) / kKktThreads;
  return need < 1 ? 1 : (need > kKktMaxBlocks ? kKktMaxBlocks : need);
}

// Runs the evaluation with caller-provided scratch: kty (n doubles), part (kKktMaxBlocks *
// kKktSlots doubles) and dout (8 doubles), all device memory; copies the 5 results to out (host).
// *bad_index is set when the CSR held a row offset or column index out of range.
cudaError_t kkt_eval_with_scratch(const rhpdhg_problem *lp, const double *x, const double *y,
                                  cudaStream_t st, double *kty, double *part, double *dout,
                                  double *out, bool *bad_index) {
  const int m = lp->m_eq + lp->m_ineq, n = lp->n;
  const int nb = kkt_blocks(m, n);
  double *flag = dout + kKktFlag;
  cudaError_t e = launch_kernel(k_kkt_zero, nb, kKktThreads, 0, st, n, kty, flag);
  if (e == cudaSuccess)
    e = launch_kernel(k_kkt_rows, nb, kKktThreads, 0, st, m, lp->m_eq, n, (long long)lp->nnz,
               (const long long *)lp->row_ptr, lp->col_idx, lp->val, x, y, lp->rhs, kty, part,
               flag);
  if (e == cudaSuccess)
    e = launch_kernel(k_kkt_cols, nb, kKktThreads, 0, st, n, lp->c, lp->l, lp->u, x, (const double *)kty,
               part);
  if (e == cudaSuccess)
    e = launch_kernel(k_kkt_final, 1, 32, 0, st, nb, (const double *)part, lp->obj_offset, dout);
  if (e != cudaSuccess) return e;
  count_launches(4);
  double h[6] = {0};
  e = cudaMemcpyAsync(h, dout, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 5; ++i) out[i] = h[i];
  *bad_index = h[kKktFlag] != 0.0;
  return cudaSuccess;
}

// Host checks shared by both entry points; returns an empty string when the arguments are usable.
std::string kkt_arg_error(const rhpdhg_problem *lp, const double *x, const double *y,
                          const double *out) {
  if (!lp || !x || !out) return "lp, x or out is NULL";
  if (lp->memory != RHPDHG_MEM_DEVICE) return "the problem's arrays must be in device memory";
  if (lp->n < 1 || lp->m_eq < 0 || lp->m_ineq < 0 || lp->nnz < 0)
    return "negative size or n < 1";
  if ((long long)lp->m_eq + lp->m_ineq > 2147483646LL) return "m exceeds the 32-bit range";
  const bool rows = lp->m_eq + lp->m_ineq > 0;
  if (!lp->row_ptr || !lp->c || !lp->l || !lp->u || (rows && (!y || !lp->rhs)) ||
      (lp->nnz > 0 && (!lp->col_idx || !lp->val)))
    return "missing problem array or point";
  return "";
}

// Result of a finished evaluation as a return code, with the message for rhpdhg_last_error.
int kkt_finish(const char *who, cudaError_t e, bool bad_index) {
  if (e != cudaSuccess) {
    set_global_error(std::string(who) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RHPDHG_ERR_OOM : RHPDHG_ERR_CUDA;
  }
  if (bad_index) {
    set_global_error(std::string(who) +
                     ": a row offset or column index of the CSR is out of range (entries skipped)");
    return RHPDHG_ERR_INVALID_ARG;
  }
  return RHPDHG_OK;
}

}  // namespace rh

extern "C" int rhpdhg_kkt_eval(const rhpdhg_problem *lp, const double *x, const double *y,
                               void *stream, double *out) {
  using namespace rh;
  const std::string bad = kkt_arg_error(lp, x, y, out);
  if (!bad.empty()) {
    set_global_error("rhpdhg_kkt_eval: " + bad);
    return RHPDHG_ERR_INVALID_ARG;
  }
  const int n = lp->n;
  cudaStream_t st = (cudaStream_t)stream;
  double *kty = nullptr, *part = nullptr, *dout = nullptr;
  bool bad_index = false;
  cudaError_t e = cudaMalloc(&kty, (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)kKktMaxBlocks * kKktSlotCount * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dout, 8 * sizeof(double));
  if (e == cudaSuccess) e = kkt_eval_with_scratch(lp, x, y, st, kty, part, dout, out, &bad_index);
  cudaFree(kty);
  cudaFree(part);
  cudaFree(dout);
  return kkt_finish("rhpdhg_kkt_eval", e, bad_index);
}

// ---------------------------------------------------------------------------------------------
// Allocation-free variant.  Some callers may not call cudaMalloc: code that lives inside a
// framework which owns all device memory through its own pool and forbids raw allocations, code
// in latency-critical loops that must not take the allocator's device-wide synchronisation, and
// services that must keep a fixed device-memory footprint.  For them the same evaluation runs on
// a scratch array fixed at file scope: every GPU that loads this library holds it until the
// process exits.  Its host-side name is only a stand-in for the device symbol, so the device
// address is looked up once per device with cudaGetSymbolAddress and kept.

namespace {

constexpr long long kNoAllocMaxN = 1LL << 20;   // largest n accepted (8 MiB of K^T y scratch)
constexpr long long kNoAllocDoubles =
    kNoAllocMaxN + (long long)rh::kKktMaxBlocks * rh::kKktSlotCount + 8;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_kkt_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

}  // namespace

extern "C" int rhpdhg_kkt_eval_noalloc(const rhpdhg_problem *lp, const double *x,
                                       const double *y, void *stream, double *out) {
  using namespace rh;
  const std::string bad = kkt_arg_error(lp, x, y, out);
  if (!bad.empty()) {
    set_global_error("rhpdhg_kkt_eval_noalloc: " + bad);
    return RHPDHG_ERR_INVALID_ARG;
  }
  if ((long long)lp->n > kNoAllocMaxN) {
    set_global_error("rhpdhg_kkt_eval_noalloc: n = " + std::to_string(lp->n) +
                     " exceeds the fixed scratch of this entry point (n <= " +
                     std::to_string(kNoAllocMaxN) + "); use rhpdhg_kkt_eval");
    return RHPDHG_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return kkt_finish("rhpdhg_kkt_eval_noalloc: cudaGetDevice", e, false);
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_global_error("rhpdhg_kkt_eval_noalloc: device ordinal out of range");
    return RHPDHG_ERR_INVALID_ARG;
  }
  double *base = nullptr;
  {
    // one-time set-up per device, with that device current
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_kkt_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_global_error(std::string("rhpdhg_kkt_eval_noalloc: cudaGetSymbolAddress: ") +
                         cudaGetErrorString(e));
        return RHPDHG_ERR_CUDA;
      }
      g_noalloc_addr[dev] = static_cast<double *>(p);
    }
    base = g_noalloc_addr[dev];
  }
  // kty and the index flag in dout are cleared by the first kernel; the used slots of every
  // launched block's partials are written before the final sum reads them
  double *kty = base;
  double *part = base + kNoAllocMaxN;
  double *dout = part + (long long)kKktMaxBlocks * kKktSlotCount;
  bool bad_index = false;
  e = kkt_eval_with_scratch(lp, x, y, (cudaStream_t)stream, kty, part, dout, out, &bad_index);
  return kkt_finish("rhpdhg_kkt_eval_noalloc", e, bad_index);
}
