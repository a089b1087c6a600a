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
constexpr int kKktSlots = kKktSlotCount;   // 0 rp2, 1 qy, 2 qq, 3 rd2, 4 cx, 5 bnd, 6 cc

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

__global__ void __launch_bounds__(kKktThreads)
k_kkt_rows(int m, int m_eq, const long long *rp, const int *col, const double *val,
           const double *x, const double *y, const double *q, double *kty, double *part) {
  __shared__ double sh[kKktThreads / 32];
  double s_rp2 = 0.0, s_qy = 0.0, s_qq = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const double yi = y[i], qi = q[i];
    double kx = 0.0;
    for (long long p = rp[i]; p < rp[i + 1]; ++p) {
      const int j = col[p];
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
  // one thread per slot, blocks summed in order
  __shared__ double tot[kKktSlots];
  if (threadIdx.x < kKktSlots) {
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

__global__ void k_kkt_zero(int n, double *v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = 0.0;
}

}  // namespace

int kkt_blocks(int m, int n) {
  const int need = ((m > n ? m : n) + kKktThreads - 1) / kKktThreads;
  return need < 1 ? 1 : (need > kKktMaxBlocks ? kKktMaxBlocks : need);
}

// Runs the evaluation with caller-provided scratch: kty (n doubles), part (kKktMaxBlocks *
// kKktSlots doubles) and dout (8 doubles), all device memory; copies the 5 results to out (host).
cudaError_t kkt_eval_with_scratch(const rhpdhg_problem *lp, const double *x, const double *y,
                                  cudaStream_t st, double *kty, double *part, double *dout,
                                  double *out) {
  const int m = lp->m_eq + lp->m_ineq, n = lp->n;
  const int nb = kkt_blocks(m, n);
  k_kkt_zero<<<nb, kKktThreads, 0, st>>>(n, kty);
  k_kkt_rows<<<nb, kKktThreads, 0, st>>>(m, lp->m_eq, (const long long *)lp->row_ptr,
                                          lp->col_idx, lp->val, x, y, lp->rhs, kty, part);
  k_kkt_cols<<<nb, kKktThreads, 0, st>>>(n, lp->c, lp->l, lp->u, x, kty, part);
  k_kkt_final<<<1, 32, 0, st>>>(nb, part, lp->obj_offset, dout);
  count_launches(4);
  cudaMemcpyAsync(out, dout, 5 * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace rh

extern "C" int rhpdhg_kkt_eval(const rhpdhg_problem *lp, const double *x, const double *y,
                               void *stream, double *out) {
  using namespace rh;
  if (!lp || !x || !out || lp->n < 1 || lp->m_eq < 0 || lp->m_ineq < 0 ||
      lp->memory != RHPDHG_MEM_DEVICE || (lp->m_eq + lp->m_ineq > 0 && (!y || !lp->rhs)) ||
      !lp->row_ptr || !lp->c || !lp->l || !lp->u)
    return RHPDHG_ERR_INVALID_ARG;
  const int n = lp->n;
  cudaStream_t st = (cudaStream_t)stream;
  double *kty = nullptr, *part = nullptr, *dout = nullptr;
  cudaError_t e = cudaMalloc(&kty, (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)kKktMaxBlocks * kKktSlotCount * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dout, 8 * sizeof(double));
  if (e == cudaSuccess) e = kkt_eval_with_scratch(lp, x, y, st, kty, part, dout, out);
  cudaFree(kty);
  cudaFree(part);
  cudaFree(dout);
  if (e == cudaErrorMemoryAllocation) return RHPDHG_ERR_OOM;
  return e == cudaSuccess ? RHPDHG_OK : RHPDHG_ERR_CUDA;
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
  if (!lp || !x || !out || lp->n < 1 || lp->m_eq < 0 || lp->m_ineq < 0 ||
      lp->memory != RHPDHG_MEM_DEVICE || (lp->m_eq + lp->m_ineq > 0 && (!y || !lp->rhs)) ||
      !lp->row_ptr || !lp->c || !lp->l || !lp->u) {
    set_global_error("rhpdhg_kkt_eval_noalloc: missing or host-memory input");
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
  if (e != cudaSuccess) return RHPDHG_ERR_CUDA;
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
  double *kty = base;                                            // cleared by the first kernel
  double *part = base + kNoAllocMaxN;                            // fully rewritten per call
  double *dout = part + (long long)kKktMaxBlocks * kKktSlotCount;
  e = kkt_eval_with_scratch(lp, x, y, (cudaStream_t)stream, kty, part, dout, out);
  return e == cudaSuccess ? RHPDHG_OK : RHPDHG_ERR_CUDA;
}
