// Create-time kernels: validation, transpose, diagonal scaling (Ruiz + Pock-Chambolle, the
// "preprocessing" the paper's solver inherits, Section 7), split-CSR layout construction,
// plain products and small vector utilities used by the power iteration.
#include <cub/cub.cuh>

#include <algorithm>
#include <atomic>
#include <climits>
#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "bufcache.h"
#include "plan.h"
#include "internal.h"

namespace rh {

namespace {

inline int nblocks(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (1LL << 30)) b = (1LL << 30);
  return (int)b;
}

// bit 1: row_ptr malformed; 2: column index out of range / not increasing; 4: non-finite value;
// 8: non-finite c or rhs; 16: l > u or NaN bound; 32: l = +inf or u = -inf
__global__ void k_validate_rows(int m, int n, long long nnz, const long long *rp, const int *col,
                                const double *val, const double *q, unsigned int *flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (rp[0] != 0 || rp[m] != nnz)) atomicOr(flags, 1u);
  if (i >= m) return;
  long long b = rp[i], e = rp[i + 1];
  if (!(0 <= b && b <= e && e <= nnz)) { atomicOr(flags, 1u); return; }
  int prev = -1;
  unsigned int f = 0;
  for (long long p = b; p < e; ++p) {
    int j = col[p];
    if (j < 0 || j >= n || j <= prev) f |= 2u;
    prev = j;
    if (!isfinite(val[p])) f |= 4u;
  }
  if (!isfinite(q[i])) f |= 8u;
  if (f) atomicOr(flags, f);
}

__global__ void k_validate_cols(int n, const double *c, const double *l, const double *u,
                                unsigned int *flags) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  unsigned int f = 0;
  if (!isfinite(c[j])) f |= 8u;
  double lj = l[j], uj = u[j];
  if (isnan(lj) || isnan(uj) || lj > uj) f |= 16u;
  if (lj == INFINITY || uj == -INFINITY) f |= 32u;
  if (isfinite(uj)) f |= kHasFiniteUpper;
  if (f) atomicOr(flags, f);
}

__global__ void k_rp_convert(int m, const long long *rp64, int *rp32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= m) rp32[i] = (int)rp64[i];
}

__global__ void k_expand_rows(int m, const int *rp, int *rows_of) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) rows_of[p] = i;
}

__global__ void k_iota(int n, int *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = i;
}

__global__ void k_count_cols(int nnz, const int *col, int *cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) atomicAdd(cnt + col[p], 1);
}

__global__ void k_gather_csc(int nnz, const int *perm, const int *rows_of, const double *val,
                             int *ridx, double *cval) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nnz) return;
  int p = perm[s];
  ridx[s] = rows_of[p];
  cval[s] = val[p];
}

// per row r of a CSR side: OP 0 -> max_p |v_p| rs_r cs_{idx_p};  OP 1 -> sum_p (..)^alpha.
// G consecutive lanes share a row (strided over its entries, then a fixed shuffle tree), so a
// long power-law row is spread over a lane group instead of running on one thread.
template <int OP, int G>
__global__ void k_side_stat(int nrows, const int *ptr, const int *idx, const double *val,
                            const double *rs, const double *cs, double alpha, double *out) {
  const long long gid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const int sub = threadIdx.x % G;
  const bool in = gid < nrows;
  const int r = in ? (int)gid : 0;
  double acc = 0.0;
  if (in) {
    const double sr = rs[r];
    const int pe = ptr[r + 1];
#pragma unroll 4
    for (int p = ptr[r] + sub; p < pe; p += G) {
      const double a = fabs(val[p]) * sr * cs[idx[p]];
      if (OP == 0) acc = fmax(acc, a);
      else acc += (alpha == 1.0) ? a : pow(a, alpha);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, acc, o, G);
    acc = (OP == 0) ? fmax(acc, t) : acc + t;
  }
  if (in && sub == 0) out[r] = acc;
}

__global__ void k_scale_update(int n, const double *stat, double *scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = stat[i];
  if (s > 0.0) scale[i] = scale[i] / sqrt(s);
}

// copy each row's entries, scaled, to its place in the short or long arrays (warp per row),
// with an FP32 (LOWP 1) or BF16 (LOWP 2) copy of the scaled values
template <int LOWP>
__global__ void k_copy_rows(int nrows, const int *ptr, const int *idx, const double *val,
                            const double *rs, const double *cs, const int *dst,
                            const uint32_t *long_mask, int *idx_s, double *val_s, float *val32_s,
                            __nv_bfloat16 *val16_s, int *idx_l, double *val_l, float *val32_l,
                            __nv_bfloat16 *val16_l) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  const int r = (int)w;
  const bool lg = (long_mask[r >> 5] >> (r & 31)) & 1u;
  int *ix = lg ? idx_l : idx_s;
  double *vx = lg ? val_l : val_s;
  float *vf = lg ? val32_l : val32_s;
  __nv_bfloat16 *vh = lg ? val16_l : val16_s;
  const int b = ptr[r], e = ptr[r + 1], o = dst[r];
  const double sr = rs[r];
  for (int p = b + lane; p < e; p += 32) {
    const int j = idx[p];
    const double v = sr * val[p] * cs[j];
    ix[o + (p - b)] = j;
    vx[o + (p - b)] = v;
    if (LOWP == 1) vf[o + (p - b)] = (float)v;
    if (LOWP == 2) vh[o + (p - b)] = __float2bfloat16_rn((float)v);
  }
}

// each factor rounded to the power of two nearest to it on a log scale
__global__ void k_round_pow2(int n, double *v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int e = 0;
  const double f = frexp(v[i], &e);           // v = f 2^e, f in [0.5, 1)
  v[i] = ldexp(1.0, f >= 0.70710678118654752440 ? e : e - 1);
}

// flag = 1 if some value has more than 8 significant bits (not exact in BF16) or lies outside
// the FP32 exponent range
__global__ void k_check_bf16(long long nnz, const double *val, unsigned int *flag) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz;
       p += (long long)gridDim.x * blockDim.x) {
    const double v = val[p];
    const float f = (float)v;
    const float h = __bfloat162float(__float2bfloat16_rn(f));
    if ((double)h != v) atomicOr(flag, 1u);
  }
}

__global__ void k_sumsq_part(int n, const double *x, double *part) {
  // fixed grid of 256 blocks x 256 threads; deterministic
  __shared__ double sh[256];
  double s = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
    double v = x[i];
    s += v * v;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(int nparts, const double *part, double *out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_fill(int n, double v, double *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

__global__ void k_vmul(int n, const double *a, const double *x, double *y, int div) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = div ? x[i] / a[i] : a[i] * x[i];
}

__global__ void k_vclamp(int n, double *x, const double *l, const double *u) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = fmin(fmax(x[i], l[i]), u[i]);
}

__global__ void __launch_bounds__(kBlockThreads)
k_side_spmv(SideLayout lay, SideVals<double> vals, WalkScratch ws,
            const double *__restrict__ src, double *out) {
  extern __shared__ double smem[];
  double *my = smem + (threadIdx.x >> 5) * lay.seg;
  auto epi = [&](int row, double dot, bool) { out[row] = dot; };
  auto gather = [&](int j) { return src[j]; };
  auto gdone = [&](int) {};
  walk_tiles<double, double>(lay, vals, gather, my, ws, epi, gdone);
}

// One product of the power iteration on K^T K^: out = side * (src * in_scale[0]) (in_scale NULL:
// 1), plus ss[0] = ||out||^2 and ss[1] = 1 / ||out|| (0 for a zero vector) from the grid's
// deterministic ticket reduction.  The next product reads ss + 1 as its input scale, so the
// normalisation v = w / ||w|| costs no launch of its own.  PT is the product and row-sum type:
// FP64 with the FP64 values; FP32 with the FP32 or BF16 values of a mixed-precision handle, where
// the input scale is applied to each row's sum (in FP64) instead of to every gathered entry and
// the norm is still an FP64 sum.
template <typename VT, typename PT>
__global__ void __launch_bounds__(kBlockThreads)
k_side_spmv_pw(SideLayout lay, SideVals<VT> vals, WalkScratch ws,
               const double *__restrict__ src, const double *in_scale, double *out, double *part,
               unsigned int *ticket, double *ss) {
  extern __shared__ double smem[];
  PT *my = reinterpret_cast<PT *>(smem) + (threadIdx.x >> 5) * lay.seg;
  constexpr bool kF64 = sizeof(PT) == sizeof(double);
  const double sc = in_scale ? *in_scale : 1.0;
  const double post = kF64 ? 1.0 : sc;
  Acc<1, 0> a, al;
  a.zero();
  al.zero();
  auto epi = [&](int row, PT dot, bool lg) {
    const double o = (double)dot * post;
    out[row] = o;
    if (lg) al.s[0] += o * o;
    else a.s[0] += o * o;
  };
  auto gather = [&](int j) { return kF64 ? PT(src[j] * sc) : PT(src[j]); };
  auto gdone = [&](int grp) { store_group(al, 0x1u, ws.group_part, grp); };
  walk_tiles<VT, PT>(lay, vals, gather, my, ws, epi, gdone);
  if (cta_reduce_and_ticket(a, 0x1u, 0u, 0u, part, ticket)) {
    double r[1];
    grid_finish<1, 0>(part, r, 0x1u, 0u, ws.group_part, lay.n_long_tiles);
    if (threadIdx.x == 0) {
      ss[0] = r[0];
      ss[1] = r[0] > 0.0 ? 1.0 / sqrt(r[0]) : 0.0;
      *ticket = 0u;
    }
  }
}

}  // namespace

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches += n; }
long long launches_so_far() { return g_launches.load(); }

unsigned int validate_problem(cudaStream_t st, int m, int n, long long nnz,
                              const long long *row_ptr, const int *col, const double *val,
                              const double *c, const double *q, const double *l, const double *u,
                              unsigned int *d_flags) {
  cudaMemsetAsync(d_flags, 0, sizeof(unsigned int), st);
  k_validate_rows<<<nblocks(m + 1, 256), 256, 0, st>>>(m, n, nnz, row_ptr, col, val, q, d_flags);
  k_validate_cols<<<nblocks(n, 256), 256, 0, st>>>(n, c, l, u, d_flags);
  count_launches(2);
  unsigned int h = 0;
  cudaMemcpyAsync(&h, d_flags, sizeof(h), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return h;
}

void convert_row_ptr(cudaStream_t st, int m, const long long *rp64, int *rp32) {
  k_rp_convert<<<nblocks(m + 1, 256), 256, 0, st>>>(m, rp64, rp32);
  count_launches(1);
}

cudaError_t build_transpose(cudaStream_t st, int m, int n, int nnz, const int *rp, const int *col,
                            const double *val, int *cp, int *ridx, double *cval) {
  cudaError_t err;
  int *rows_of = nullptr, *iota = nullptr, *keys_out = nullptr, *perm = nullptr, *cnt = nullptr;
  void *tmp = nullptr;
  size_t tmp_bytes = 0, scan_bytes = 0;
  const size_t nz = (size_t)std::max(nnz, 1);
  if ((err = buf_alloc((void **)&rows_of, nz * sizeof(int)))) goto done;
  if ((err = buf_alloc((void **)&iota, nz * sizeof(int)))) goto done;
  if ((err = buf_alloc((void **)&keys_out, nz * sizeof(int)))) goto done;
  if ((err = buf_alloc((void **)&perm, nz * sizeof(int)))) goto done;
  if ((err = buf_alloc((void **)&cnt, (size_t)(n + 1) * sizeof(int)))) goto done;
  {
    int end_bit = 1;
    while ((1LL << end_bit) < (long long)n) ++end_bit;
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, col, keys_out, iota, perm, nnz, 0, end_bit,
                                    st);
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, cnt, cp, n + 1, st);
    tmp_bytes = std::max(tmp_bytes, scan_bytes);
    if ((err = buf_alloc(&tmp, std::max<size_t>(tmp_bytes, 16)))) goto done;
    k_expand_rows<<<nblocks(m, 256), 256, 0, st>>>(m, rp, rows_of);
    k_iota<<<nblocks(nnz, 256), 256, 0, st>>>(nnz, iota);
    if (nnz > 0)
      cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, col, keys_out, iota, perm, nnz, 0, end_bit,
                                      st);
    cudaMemsetAsync(cnt, 0, (size_t)(n + 1) * sizeof(int), st);
    k_count_cols<<<nblocks(nnz, 256), 256, 0, st>>>(nnz, col, cnt);
    cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, cnt, cp, n + 1, st);
    k_gather_csc<<<nblocks(nnz, 256), 256, 0, st>>>(nnz, perm, rows_of, val, ridx, cval);
    count_launches(4);
    err = cudaStreamSynchronize(st);
    if (err == cudaSuccess) err = cudaGetLastError();
  }
done:
  cudaStreamSynchronize(st);     // nothing in flight uses the scratch when it goes back
  buf_release(rows_of);
  buf_release(iota);
  buf_release(keys_out);
  buf_release(perm);
  buf_release(cnt);
  buf_release(tmp);
  return err;
}

// lanes per row for a side with `nnz` entries over `nrows` rows (the mean row length, rounded
// up to a power of two, 4 to 32)
static int stat_group(long long nnz, int nrows) {
  const double mean = nrows > 0 ? (double)nnz / nrows : 0.0;
  int g = 4;
  while (g < 32 && g < mean) g *= 2;
  return g;
}

template <int OP>
static void side_stat(cudaStream_t st, int nrows, long long nnz, const int *ptr, const int *idx,
                      const double *val, const double *rs, const double *cs, double alpha,
                      double *out) {
  const int g = stat_group(nnz, nrows);
  const long long threads = (long long)nrows * g;
  const int nb = (int)((threads + 255) / 256);
  if (nb <= 0) return;
  switch (g) {
    case 4: k_side_stat<OP, 4><<<nb, 256, 0, st>>>(nrows, ptr, idx, val, rs, cs, alpha, out); break;
    case 8: k_side_stat<OP, 8><<<nb, 256, 0, st>>>(nrows, ptr, idx, val, rs, cs, alpha, out); break;
    case 16: k_side_stat<OP, 16><<<nb, 256, 0, st>>>(nrows, ptr, idx, val, rs, cs, alpha, out); break;
    default: k_side_stat<OP, 32><<<nb, 256, 0, st>>>(nrows, ptr, idx, val, rs, cs, alpha, out); break;
  }
}

void compute_scaling(cudaStream_t st, int m, int n, const int *rp, const int *col,
                     const double *val, const int *cp, const int *ridx, const double *cval,
                     int ruiz_iters, double alpha, double *D, double *E, double *tmp_m,
                     double *tmp_n) {
  long long nnz = 0;
  {
    int last = 0;
    if (m > 0) cudaMemcpyAsync(&last, rp + m, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    nnz = last;
  }
  k_fill<<<nblocks(m, 256), 256, 0, st>>>(m, 1.0, D);
  k_fill<<<nblocks(n, 256), 256, 0, st>>>(n, 1.0, E);
  count_launches(2 + 4LL * ruiz_iters + (alpha >= 0.0 ? 4 : 0));
  for (int it = 0; it < ruiz_iters; ++it) {
    // both norms from the same current matrix, then both updates
    side_stat<0>(st, m, nnz, rp, col, val, D, E, 1.0, tmp_m);
    side_stat<0>(st, n, nnz, cp, ridx, cval, E, D, 1.0, tmp_n);
    k_scale_update<<<nblocks(m, 256), 256, 0, st>>>(m, tmp_m, D);
    k_scale_update<<<nblocks(n, 256), 256, 0, st>>>(n, tmp_n, E);
  }
  if (alpha >= 0.0) {
    side_stat<1>(st, m, nnz, rp, col, val, D, E, alpha, tmp_m);
    side_stat<1>(st, n, nnz, cp, ridx, cval, E, D, 2.0 - alpha, tmp_n);
    k_scale_update<<<nblocks(m, 256), 256, 0, st>>>(m, tmp_m, D);
    k_scale_update<<<nblocks(n, 256), 256, 0, st>>>(n, tmp_n, E);
  }
}

namespace {
// Cached buffers are keyed by (device, size): a buffer is only ever reused on the device it was
// allocated on.  Buffers from a caller's allocator carry it (hook.free set) and are never cached.
struct BufInfo {
  int dev;
  size_t bytes;
  DevAllocator hook;
};

thread_local const DevAllocator *tl_alloc = nullptr;   // set by AllocScope
std::mutex g_buf_mu;
std::unordered_map<void *, BufInfo> g_buf_info;              // every buffer from buf_alloc
std::map<std::pair<int, size_t>, std::vector<void *>> g_buf_free;   // cached, by (device, size)
size_t g_buf_free_bytes = 0;

// Frees every cached buffer (on its own device); the caller holds g_buf_mu.
void buf_drop_cache_locked() {
  if (g_buf_free.empty()) return;
  int cur = -1;
  cudaGetDevice(&cur);
  for (auto &kv : g_buf_free) {
    if (kv.second.empty()) continue;
    cudaSetDevice(kv.first.first);
    for (void *p : kv.second) {
      g_buf_info.erase(p);
      cudaFree(p);
    }
  }
  if (cur >= 0) cudaSetDevice(cur);
  g_buf_free.clear();
  g_buf_free_bytes = 0;
}
}  // namespace

AllocScope::AllocScope(const DevAllocator &a) : prev_(tl_alloc), mine_(a) {
  tl_alloc = (mine_.alloc && mine_.free) ? &mine_ : nullptr;
}
AllocScope::~AllocScope() { tl_alloc = prev_; }

cudaError_t buf_alloc(void **p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 1);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (tl_alloc) {
    // 256-byte alignment covers every vector load of the kernels
    void *q = tl_alloc->alloc(bytes, tl_alloc->stream, tl_alloc->ctx);
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
      tl_alloc->free(q, tl_alloc->stream, tl_alloc->ctx);
      return cudaErrorInvalidValue;
    }
    *p = q;
    std::lock_guard<std::mutex> lk(g_buf_mu);
    g_buf_info[q] = BufInfo{dev, bytes, *tl_alloc};
    return cudaSuccess;
  }
  {
    std::lock_guard<std::mutex> lk(g_buf_mu);
    auto it = g_buf_free.find({dev, bytes});
    if (it != g_buf_free.end() && !it->second.empty()) {
      *p = it->second.back();
      it->second.pop_back();
      g_buf_free_bytes -= bytes;
      return cudaSuccess;
    }
  }
  e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    {
      std::lock_guard<std::mutex> lk(g_buf_mu);
      buf_drop_cache_locked();
    }
    e = cudaMalloc(p, bytes);
  }
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_buf_mu);
    g_buf_info[*p] = BufInfo{dev, bytes, DevAllocator()};
  }
  return e;
}

void buf_release(void *p) {
  if (!p) return;
  {
    std::unique_lock<std::mutex> lk(g_buf_mu);
    auto it = g_buf_info.find(p);
    if (it != g_buf_info.end()) {
      const BufInfo bi = it->second;
      if (bi.hook.free) {
        g_buf_info.erase(it);
        lk.unlock();
        bi.hook.free(p, bi.hook.stream, bi.hook.ctx);
        return;
      }
      if (g_buf_free_bytes + bi.bytes <= kBufferCacheBytes) {
        g_buf_free[{bi.dev, bi.bytes}].push_back(p);
        g_buf_free_bytes += bi.bytes;
        return;
      }
      g_buf_info.erase(it);
    }
  }
  cudaFree(p);
}

size_t buf_drop_cache() {
  std::lock_guard<std::mutex> lk(g_buf_mu);
  const size_t freed = g_buf_free_bytes;
  buf_drop_cache_locked();
  return freed;
}

// The cost model of tile_rows_fp64 over all short tiles of a side: FP64 adds per warp of the
// lane-per-row sums (4 ceil(longest / 4) per tile) against the best threshold's (c + the sum over
// rows longer than c of ceil(len / 32) + 5, c in 8, 16, 32).  The warp-wide sums are enabled
// when they save at least 15% of those adds (power-law sides; not sides of even row lengths,
// where the search would only cost time).
static bool wide_rows_pay(const int *hp, const std::vector<uint32_t> &mask, int nrows) {
  long long plain = 0, best = 0;
  for (int t = 0; t * kTileRows < nrows; ++t) {
    int len[kTileRows];
    int mx = 0;
    for (int r = 0; r < kTileRows; ++r) {
      const int row = t * kTileRows + r;
      len[r] = (row < nrows && !((mask[t] >> r) & 1u)) ? hp[row + 1] - hp[row] : 0;
      mx = std::max(mx, len[r]);
    }
    const int p = (mx + 3) & ~3;
    int b = p;
    if (mx > 16) {
      for (int c = 8; c <= 32 && c < mx; c *= 2) {
        int cost = c;
        for (int r = 0; r < kTileRows; ++r)
          if (len[r] > c) cost += ((len[r] + 31) >> 5) + 5;
        b = std::min(b, cost);
      }
    }
    plain += p;
    best += b;
  }
  return plain > 0 && (double)best <= 0.85 * (double)plain;
}

bool plan_side(const int *hp, int nrows, SidePlan *p) {
  SidePlan &P = *p;
  const int ntiles = (nrows + kTileRows - 1) / kTileRows;
  P = SidePlan();
  P.nrows = nrows;
  P.ntiles = ntiles;
  P.ptr_s.assign(std::max(nrows, 1), 0);
  P.tile_end.assign(std::max(ntiles, 1), 0);
  P.dst.assign(std::max(nrows, 1), 0);
  P.mask.assign(std::max(ntiles, 1), 0u);
  P.chunk_ptr.assign(1, 0);
  long long cur = 0, cl = 0, maxseg = 0;
  auto align4 = [](long long v) { return (v + 3) & ~3LL; };
  for (int t = 0; t < ntiles; ++t) {
    const int r0 = t * kTileRows, r1 = std::min(nrows, (t + 1) * kTileRows);
    // membership: rows over kShortMax are long; then, while the tile's short segment exceeds
    // kSegBudget, its longest short row (the first of equal ones) becomes long
    long long sum = 0;
    for (int r = r0; r < r1; ++r) {
      const int len = hp[r + 1] - hp[r];
      if (len > kShortMax) P.mask[t] |= 1u << (r - r0);
      else sum += len;
    }
    while (sum > kSegBudget) {
      int best = -1, blen = -1;
      for (int r = r0; r < r1; ++r) {
        const int len = hp[r + 1] - hp[r];
        if (!((P.mask[t] >> (r - r0)) & 1u) && len > blen) { best = r; blen = len; }
      }
      P.mask[t] |= 1u << (best - r0);
      sum -= blen;
    }
    cur = align4(cur);
    const long long seg_b = cur;
    for (int r = r0; r < r1; ++r) {
      const int len = hp[r + 1] - hp[r];
      P.ptr_s[r] = (int)cur;
      if (!((P.mask[t] >> (r - r0)) & 1u)) {
        P.dst[r] = (int)cur;
        cur += len;
      } else {
        cl = align4(cl);
        const int li = (int)P.long_rows.size();
        P.long_rows.push_back(r);
        P.beg_l.push_back((int)cl);
        P.end_l.push_back((int)(cl + len));
        P.dst[r] = (int)cl;
        cl += len;
        const int nc = (len + kChunk - 1) / kChunk;
        for (int c = 0; c < nc; ++c) P.chunk_row.push_back(li);
        P.chunk_ptr.push_back(P.chunk_ptr.back() + nc);
      }
      if (cur > INT_MAX - 8 || cl > INT_MAX - 2 * kChunk) return false;   // casts stay in range
    }
    P.tile_end[t] = (int)cur;
    maxseg = std::max(maxseg, cur - seg_b);
  }
  P.nnz_s = align4(cur) + 4;
  P.nnz_l = align4(cl) + kChunk;
  if (P.nnz_s > INT_MAX || P.nnz_l > INT_MAX) return false;
  // Tiles per work item: where tiles are short (a few entries per row), M consecutive tiles are
  // staged as one segment, so that each warp's chain of dependent loads carries M tiles' bytes.
  // M is the largest of kMaxTileMult, ..., 2 whose mean group segment fits one staging round
  // (128 * kStageUnroll entries) and whose longest fits the staging budget; else 1.
  P.maxseg_mult[0] = maxseg;
  for (int k = 1, cand = 2; cand <= kMaxTileMult; ++k, cand *= 2) {
    long long mx = 0;
    for (int t0 = 0; t0 < ntiles; t0 += cand) {
      const int t1 = std::min(ntiles, t0 + cand) - 1;
      mx = std::max(mx, (long long)P.tile_end[t1] - P.ptr_s[(size_t)t0 * kTileRows]);
    }
    P.maxseg_mult[k] = (ntiles > 0 && mx <= kSegBudget) ? mx : -1;
  }
  int mult = 1;
  for (int k = 2, cand = kMaxTileMult; cand >= 2 && mult == 1; --k, cand /= 2) {
    if (ntiles < 2 * cand) continue;
    if (align4(cur) * cand > (long long)ntiles * kWarp * kStageUnroll * 4) continue;
    if (P.maxseg_mult[k] >= 0) {
      mult = cand;
      maxseg = P.maxseg_mult[k];
    }
  }
  P.mult = mult;
  P.maxseg = maxseg;
  P.wide_rows = wide_rows_pay(hp, P.mask, nrows) ? 1 : 0;
  return true;
}

cudaError_t build_side(cudaStream_t st, int nrows, int nnz, const int *ptr, const int *idx,
                       const double *val, const double *rscale, const double *cscale,
                       int lowp, SideStore *out) {
  (void)nnz;
  SideStore s;
  cudaError_t err = cudaSuccess;
  // ---- structure, on the host -------------------------------------------------------------
  std::vector<int> hp(nrows + 1);
  if ((err = cudaMemcpy(hp.data(), ptr, (nrows + 1) * sizeof(int), cudaMemcpyDeviceToHost)))
    return err;
  SidePlan P;
  if (!plan_side(hp.data(), nrows, &P)) return cudaErrorInvalidValue;
  const int ntiles = P.ntiles, mult = P.mult;
  const long long nnz_s = P.nnz_s, nnz_l = P.nnz_l, maxseg = P.maxseg;
  const std::vector<int> &ptr_s = P.ptr_s, &tile_end = P.tile_end, &dst = P.dst,
                         &long_rows = P.long_rows, &beg_l = P.beg_l, &end_l = P.end_l,
                         &chunk_ptr = P.chunk_ptr, &chunk_row = P.chunk_row;
  const std::vector<uint32_t> &mask = P.mask;
  auto align4 = [](long long v) { return (v + 3) & ~3LL; };
  const int nlong = (int)long_rows.size(), nch = (int)chunk_row.size();
  s.lay.nrows = nrows;
  s.lay.seg = (int)align4(maxseg) + 4;
  s.lay.n_short_tiles = ntiles;
  s.lay.tile_mult = mult;
  s.lay.n_tile_groups = (ntiles + mult - 1) / mult;
  s.lay.n_long = nlong;
  s.lay.n_long_tiles = (nlong + kTileRows - 1) / kTileRows;
  s.lay.n_chunks = nch;
  s.lay.wide_rows = P.wide_rows;
  s.rule_mult = mult;
  for (int k = 0; k < 3; ++k) s.maxseg_mult[k] = P.maxseg_mult[k];
  s.nnz_short = nnz_s;
  s.nnz_long = nnz_l;
  const size_t ng = (size_t)std::max(s.lay.n_long_tiles, 1);
  int *d_dst = nullptr;
  auto up = [&](int **d, const std::vector<int> &h) -> cudaError_t {
    cudaError_t e = buf_alloc((void **)d, std::max<size_t>(h.size(), 1) * sizeof(int));
    if (e == cudaSuccess && !h.empty())
      e = cudaMemcpy(*d, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice);
    return e;
  };
#define TRY(x)                 \
  do {                         \
    if ((err = (x))) goto fail; \
  } while (0)
  TRY(up(&s.ptr_s, ptr_s));
  TRY(up(&s.tile_end, tile_end));
  TRY(up(&s.long_rows, long_rows));
  TRY(up(&s.beg_l, beg_l));
  TRY(up(&s.end_l, end_l));
  TRY(up(&s.chunk_ptr, chunk_ptr));
  TRY(up(&s.chunk_row, chunk_row));
  {
    // per chunk: its long row, entry range, and the chunk count of its group of 32 long rows
    std::vector<int4> desc((size_t)std::max(nch, 1));
    for (int c = 0; c < nch; ++c) {
      const int li = chunk_row[c];
      const int cb = beg_l[li] + (c - chunk_ptr[li]) * kChunk;
      const int g0 = (li / kTileRows) * kTileRows, g1 = std::min(g0 + kTileRows, nlong);
      desc[c] = make_int4(li, cb, std::min(cb + kChunk, end_l[li]), chunk_ptr[g1] - chunk_ptr[g0]);
    }
    TRY(buf_alloc((void **)&s.chunk_desc, desc.size() * sizeof(int4)));
    TRY(cudaMemcpy(s.chunk_desc, desc.data(), desc.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  TRY(up(&d_dst, dst));
  TRY(buf_alloc((void **)&s.long_mask, mask.size() * sizeof(uint32_t)));
  TRY(cudaMemcpy(s.long_mask, mask.data(), mask.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  // ---- entries (zero padding), scaled on the device ------------------------------------------
  TRY(buf_alloc((void **)&s.idx_s, nnz_s * sizeof(int)));
  TRY(buf_alloc((void **)&s.val64_s, nnz_s * sizeof(double)));
  TRY(buf_alloc((void **)&s.idx_l, nnz_l * sizeof(int)));
  TRY(buf_alloc((void **)&s.val64_l, nnz_l * sizeof(double)));
  TRY(cudaMemsetAsync(s.idx_s, 0, nnz_s * sizeof(int), st));
  TRY(cudaMemsetAsync(s.val64_s, 0, nnz_s * sizeof(double), st));
  TRY(cudaMemsetAsync(s.idx_l, 0, nnz_l * sizeof(int), st));
  TRY(cudaMemsetAsync(s.val64_l, 0, nnz_l * sizeof(double), st));
  if (lowp == 1) {
    TRY(buf_alloc((void **)&s.val32_s, nnz_s * sizeof(float)));
    TRY(buf_alloc((void **)&s.val32_l, nnz_l * sizeof(float)));
    TRY(cudaMemsetAsync(s.val32_s, 0, nnz_s * sizeof(float), st));
    TRY(cudaMemsetAsync(s.val32_l, 0, nnz_l * sizeof(float), st));
  } else if (lowp == 2) {
    TRY(buf_alloc((void **)&s.val16_s, nnz_s * sizeof(__nv_bfloat16)));
    TRY(buf_alloc((void **)&s.val16_l, nnz_l * sizeof(__nv_bfloat16)));
    TRY(cudaMemsetAsync(s.val16_s, 0, nnz_s * sizeof(__nv_bfloat16), st));
    TRY(cudaMemsetAsync(s.val16_l, 0, nnz_l * sizeof(__nv_bfloat16), st));
  }
  if (nrows > 0) {
    const int nb = nblocks((long long)nrows * 32, 256);
    auto copy = [&](auto kern) {
      kern<<<nb, 256, 0, st>>>(nrows, ptr, idx, val, rscale, cscale, d_dst, s.long_mask,
                               s.idx_s, s.val64_s, s.val32_s, s.val16_s, s.idx_l, s.val64_l,
                               s.val32_l, s.val16_l);
    };
    if (lowp == 1) copy(k_copy_rows<1>);
    else if (lowp == 2) copy(k_copy_rows<2>);
    else copy(k_copy_rows<0>);
    count_launches(1);
  }
  // ---- walk scratch ------------------------------------------------------------------------
  TRY(buf_alloc((void **)&s.part_a, (size_t)std::max(nch, 1) * sizeof(double)));
  TRY(buf_alloc((void **)&s.part_b, (size_t)std::max(nch, 1) * sizeof(double)));
  TRY(buf_alloc((void **)&s.done_a, ng * sizeof(unsigned int)));
  TRY(buf_alloc((void **)&s.done_b, ng * sizeof(unsigned int)));
  TRY(buf_alloc((void **)&s.gpart_a, ng * kMaxPartials * sizeof(double)));
  TRY(buf_alloc((void **)&s.gpart_b, ng * kMaxPartials * sizeof(double)));
  TRY(cudaMemsetAsync(s.done_a, 0, ng * sizeof(unsigned int), st));
  TRY(cudaMemsetAsync(s.done_b, 0, ng * sizeof(unsigned int), st));
  TRY(cudaStreamSynchronize(st));
  TRY(cudaGetLastError());
#undef TRY
  buf_release(d_dst);
  s.lay.ptr_s = s.ptr_s;
  s.lay.tile_end = s.tile_end;
  s.lay.idx_s = s.idx_s;
  s.lay.long_mask = s.long_mask;
  s.lay.long_rows = s.long_rows;
  s.lay.beg_l = s.beg_l;
  s.lay.end_l = s.end_l;
  s.lay.idx_l = s.idx_l;
  s.lay.chunk_ptr = s.chunk_ptr;
  s.lay.chunk_row = s.chunk_row;
  s.lay.chunk_desc = s.chunk_desc;
  s.v64.s = s.val64_s;
  s.v64.l = s.val64_l;
  s.v32.s = s.val32_s;
  s.v32.l = s.val32_l;
  s.v16.s = s.val16_s;
  s.v16.l = s.val16_l;
  s.wa.chunk_part = s.part_a;
  s.wa.group_done = s.done_a;
  s.wa.group_part = s.gpart_a;
  s.wb.chunk_part = s.part_b;
  s.wb.group_done = s.done_b;
  s.wb.group_part = s.gpart_b;
  *out = s;
  return cudaSuccess;
fail:
  cudaStreamSynchronize(st);
  buf_release(d_dst);
  free_side(&s);
  return err;
}

void round_pow2(cudaStream_t st, int n, double *v) {
  if (n <= 0) return;
  k_round_pow2<<<nblocks(n, 256), 256, 0, st>>>(n, v);
  count_launches(1);
}

unsigned int values_exact_in_bf16(cudaStream_t st, long long nnz, const double *val,
                                  unsigned int *d_flag) {
  cudaMemsetAsync(d_flag, 0, sizeof(unsigned int), st);
  if (nnz > 0) {
    k_check_bf16<<<std::min<long long>(nblocks(nnz, 256), 4096), 256, 0, st>>>(nnz, val, d_flag);
    count_launches(1);
  }
  unsigned int h = 0;
  cudaMemcpyAsync(&h, d_flag, sizeof(h), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return h == 0;
}

void free_side(SideStore *s) {
  void *bufs[] = {s->ptr_s, s->tile_end, s->idx_s, s->long_mask, s->long_rows, s->beg_l,
                  s->end_l, s->idx_l,
                  s->chunk_ptr, s->chunk_row, s->chunk_desc, s->val64_s, s->val64_l,
                  s->val32_s, s->val32_l,
                  s->val16_s, s->val16_l,
                  s->part_a, s->part_b, s->done_a, s->done_b, s->gpart_a, s->gpart_b};
  for (void *b : bufs) buf_release(b);
  *s = SideStore();
}

int tile_grid(const SideLayout &lay, int sm_count, int blocks_per_sm) {
  const int w = lay.cta_warps > 0 ? lay.cta_warps : kBlockWarps;
  long long need = ((long long)lay.total_items() + w - 1) / w;
  long long cap = (long long)sm_count * std::max(blocks_per_sm, 1);
  long long g = std::min(need, cap);
  return (int)std::max<long long>(g, 1);
}

void allow_large_smem_setup(int bytes) {
  cudaFuncSetAttribute(k_side_spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_side_spmv_pw<double, double>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_side_spmv_pw<float, float>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_side_spmv_pw<__nv_bfloat16, float>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

static int pw_smem(const SideStore &side, int lowp) {
  return kBlockWarps * side.lay.seg * (lowp ? (int)sizeof(float) : (int)sizeof(double));
}

void side_spmv_pw(cudaStream_t st, const SideStore &side, int lowp, const double *src,
                  const double *in_scale, double *out, double *part, unsigned int *ticket,
                  double *ss, int grid) {
  const int smem = pw_smem(side, lowp);
  if (lowp == 2)
    k_side_spmv_pw<__nv_bfloat16, float><<<grid, kBlockThreads, smem, st>>>(
        side.lay, side.v16, side.wa, src, in_scale, out, part, ticket, ss);
  else if (lowp == 1)
    k_side_spmv_pw<float, float><<<grid, kBlockThreads, smem, st>>>(
        side.lay, side.v32, side.wa, src, in_scale, out, part, ticket, ss);
  else
    k_side_spmv_pw<double, double><<<grid, kBlockThreads, smem, st>>>(
        side.lay, side.v64, side.wa, src, in_scale, out, part, ticket, ss);
  count_launches(1);
}

// grid of the power-iteration product on `side`: whole resident waves, at most the work items
int side_spmv_pw_grid(const SideStore &side, int lowp, int sm_count) {
  const int smem = pw_smem(side, lowp);
  int b = 0;
  if (lowp == 2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_side_spmv_pw<__nv_bfloat16, float>,
                                                  kBlockThreads, smem);
  else if (lowp == 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_side_spmv_pw<float, float>,
                                                  kBlockThreads, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_side_spmv_pw<double, double>,
                                                  kBlockThreads, smem);
  return tile_grid(side.lay, sm_count, b);
}

void side_spmv(cudaStream_t st, const SideStore &side, const double *src, double *out, int grid) {
  int smem = kBlockWarps * side.lay.seg * (int)sizeof(double);
  k_side_spmv<<<grid, kBlockThreads, smem, st>>>(side.lay, side.v64, side.wa, src, out);
  count_launches(1);
}

void sumsq(cudaStream_t st, int n, const double *x, double *out, double *tmp) {
  k_sumsq_part<<<256, 256, 0, st>>>(n, x, tmp);
  k_sum_final<<<1, 256, 0, st>>>(256, tmp, out);
  count_launches(2);
}

void fill(cudaStream_t st, int n, double v, double *x) {
  k_fill<<<nblocks(n, 256), 256, 0, st>>>(n, v, x);
  count_launches(1);
}

void vmul(cudaStream_t st, int n, const double *a, const double *x, double *y, int div) {
  k_vmul<<<nblocks(n, 256), 256, 0, st>>>(n, a, x, y, div);
  count_launches(1);
}

void vclamp(cudaStream_t st, int n, double *x, const double *l, const double *u) {
  k_vclamp<<<nblocks(n, 256), 256, 0, st>>>(n, x, l, u);
  count_launches(1);
}

}  // namespace rh
