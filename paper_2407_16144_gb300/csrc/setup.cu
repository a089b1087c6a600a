// Create-time kernels: validation, transpose, diagonal scaling (Ruiz + Pock-Chambolle, the
// "preprocessing" the paper's solver inherits, Section 7), split-CSR layout construction,
// plain products and small vector utilities used by the power iteration.
#include <cub/cub.cuh>

#include <algorithm>
#include <atomic>
#include <vector>

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

// per row r of a CSR side: OP 0 -> max_p |v_p| rs_r cs_{idx_p};  OP 1 -> sum_p (..)^alpha
template <int OP>
__global__ void k_side_stat(int nrows, const int *ptr, const int *idx, const double *val,
                            const double *rs, const double *cs, double alpha, double *out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  double acc = 0.0;
  const double sr = rs[r];
  for (int p = ptr[r]; p < ptr[r + 1]; ++p) {
    double a = fabs(val[p]) * sr * cs[idx[p]];
    if (OP == 0) acc = fmax(acc, a);
    else acc += (alpha == 1.0) ? a : pow(a, alpha);
  }
  out[r] = acc;
}

__global__ void k_scale_update(int n, const double *stat, double *scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = stat[i];
  if (s > 0.0) scale[i] = scale[i] / sqrt(s);
}

__global__ void k_short_lengths(int nrows, const int *ptr, int L, int *len_s, int *is_long) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r > nrows) return;
  if (r == nrows) { len_s[r] = 0; return; }
  int len = ptr[r + 1] - ptr[r];
  len_s[r] = len <= L ? len : 0;
  is_long[r] = len > L ? 1 : 0;
}

__global__ void k_long_lengths(int n_long, const int *long_rows, const int *ptr, int *len_l) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n_long) return;
  if (i == n_long) { len_l[i] = 0; return; }
  int r = long_rows[i];
  len_l[i] = ptr[r + 1] - ptr[r];
}

__global__ void k_copy_short(int nrows, const int *ptr, const int *idx, const double *val,
                             const double *rs, const double *cs, const int *ptr_s, int *idx_s,
                             double *val_s, float *val32_s, int L) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int b = ptr[r], e = ptr[r + 1];
  if (e - b > L) return;
  int o = ptr_s[r];
  const double sr = rs[r];
  for (int p = b; p < e; ++p, ++o) {
    int j = idx[p];
    idx_s[o] = j;
    const double v = sr * val[p] * cs[j];
    val_s[o] = v;
    if (val32_s) val32_s[o] = (float)v;
  }
}

__global__ void k_copy_long(int n_long, const int *long_rows, const int *ptr, const int *idx,
                            const double *val, const double *rs, const double *cs,
                            const int *ptr_l, int *idx_l, double *val_l, float *val32_l) {
  // one warp per long row
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n_long) return;
  int r = long_rows[w];
  int b = ptr[r], e = ptr[r + 1];
  int o = ptr_l[w];
  const double sr = rs[r];
  for (int p = b + lane; p < e; p += 32) {
    int j = idx[p];
    idx_l[o + (p - b)] = j;
    const double v = sr * val[p] * cs[j];
    val_l[o + (p - b)] = v;
    if (val32_l) val32_l[o + (p - b)] = (float)v;
  }
}

__global__ void k_long_mask(int nrows, int ntiles, const int *is_long, uint32_t *mask) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  uint32_t mk = 0;
  for (int r = 0; r < 32; ++r) {
    int row = t * 32 + r;
    if (row < nrows && is_long[row]) mk |= (1u << r);
  }
  mask[t] = mk;
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

__global__ void k_normalize(int n, const double *w, const double *ss, double *v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = sqrt(*ss);
  v[i] = s > 0.0 ? w[i] / s : 0.0;
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
  double *my = smem + (threadIdx.x >> 5) * (kTileRows * lay.L);
  auto epi = [&](int row, double dot, bool) { out[row] = dot; };
  auto gather = [&](int j) { return src[j]; };
  auto gdone = [&](int) {};
  walk_tiles<double, double>(lay, vals, gather, my, ws, epi, gdone);
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
  if ((err = cudaMalloc(&rows_of, nz * sizeof(int)))) goto done;
  if ((err = cudaMalloc(&iota, nz * sizeof(int)))) goto done;
  if ((err = cudaMalloc(&keys_out, nz * sizeof(int)))) goto done;
  if ((err = cudaMalloc(&perm, nz * sizeof(int)))) goto done;
  if ((err = cudaMalloc(&cnt, (size_t)(n + 1) * sizeof(int)))) goto done;
  {
    int end_bit = 1;
    while ((1LL << end_bit) < (long long)n) ++end_bit;
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, col, keys_out, iota, perm, nnz, 0, end_bit,
                                    st);
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, cnt, cp, n + 1, st);
    tmp_bytes = std::max(tmp_bytes, scan_bytes);
    if ((err = cudaMalloc(&tmp, std::max<size_t>(tmp_bytes, 16)))) goto done;
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
  cudaFree(rows_of);
  cudaFree(iota);
  cudaFree(keys_out);
  cudaFree(perm);
  cudaFree(cnt);
  cudaFree(tmp);
  return err;
}

void compute_scaling(cudaStream_t st, int m, int n, const int *rp, const int *col,
                     const double *val, const int *cp, const int *ridx, const double *cval,
                     int ruiz_iters, double alpha, double *D, double *E, double *tmp_m,
                     double *tmp_n) {
  k_fill<<<nblocks(m, 256), 256, 0, st>>>(m, 1.0, D);
  k_fill<<<nblocks(n, 256), 256, 0, st>>>(n, 1.0, E);
  count_launches(2 + 4LL * ruiz_iters + (alpha >= 0.0 ? 4 : 0));
  for (int it = 0; it < ruiz_iters; ++it) {
    // both norms from the same current matrix, then both updates
    k_side_stat<0><<<nblocks(m, 256), 256, 0, st>>>(m, rp, col, val, D, E, 1.0, tmp_m);
    k_side_stat<0><<<nblocks(n, 256), 256, 0, st>>>(n, cp, ridx, cval, E, D, 1.0, tmp_n);
    k_scale_update<<<nblocks(m, 256), 256, 0, st>>>(m, tmp_m, D);
    k_scale_update<<<nblocks(n, 256), 256, 0, st>>>(n, tmp_n, E);
  }
  if (alpha >= 0.0) {
    k_side_stat<1><<<nblocks(m, 256), 256, 0, st>>>(m, rp, col, val, D, E, alpha, tmp_m);
    k_side_stat<1><<<nblocks(n, 256), 256, 0, st>>>(n, cp, ridx, cval, E, D, 2.0 - alpha, tmp_n);
    k_scale_update<<<nblocks(m, 256), 256, 0, st>>>(m, tmp_m, D);
    k_scale_update<<<nblocks(n, 256), 256, 0, st>>>(n, tmp_n, E);
  }
}

cudaError_t build_side(cudaStream_t st, int nrows, int nnz, const int *ptr, const int *idx,
                       const double *val, const double *rscale, const double *cscale, int L,
                       bool with32, SideStore *out) {
  cudaError_t err;
  SideStore s;
  int *len_s = nullptr, *is_long = nullptr, *iota = nullptr, *nsel = nullptr, *len_l = nullptr;
  void *tmp = nullptr;
  size_t tb = 0, tb2 = 0, tb3 = 0;
  int h_nlong = 0, h_nnz_s = 0, h_nnz_l = 0;
  const int ntiles = (nrows + kTileRows - 1) / kTileRows;
  s.lay.nrows = nrows;
  s.lay.L = L;
  s.lay.n_short_tiles = ntiles;
  if ((err = cudaMalloc(&s.ptr_s, (size_t)(nrows + 1) * sizeof(int)))) goto fail;
  if ((err = cudaMalloc(&len_s, (size_t)(nrows + 1) * sizeof(int)))) goto fail;
  if ((err = cudaMalloc(&is_long, (size_t)std::max(nrows, 1) * sizeof(int)))) goto fail;
  if ((err = cudaMalloc(&iota, (size_t)std::max(nrows, 1) * sizeof(int)))) goto fail;
  if ((err = cudaMalloc(&nsel, sizeof(int)))) goto fail;
  if ((err = cudaMalloc(&s.long_mask, (size_t)std::max(ntiles, 1) * sizeof(uint32_t)))) goto fail;
  if ((err = cudaMalloc(&s.long_rows, (size_t)std::max(nrows, 1) * sizeof(int)))) goto fail;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, len_s, s.ptr_s, nrows + 1, st);
  cub::DeviceSelect::Flagged(nullptr, tb2, iota, is_long, s.long_rows, nsel, nrows, st);
  tb = std::max(tb, tb2);
  if ((err = cudaMalloc(&tmp, std::max<size_t>(tb, 16)))) goto fail;
  k_short_lengths<<<nblocks(nrows + 1, 256), 256, 0, st>>>(nrows, ptr, L, len_s, is_long);
  k_iota<<<nblocks(nrows, 256), 256, 0, st>>>(nrows, iota);
  cub::DeviceScan::ExclusiveSum(tmp, tb, len_s, s.ptr_s, nrows + 1, st);
  cudaMemsetAsync(nsel, 0, sizeof(int), st);
  if (nrows > 0) cub::DeviceSelect::Flagged(tmp, tb, iota, is_long, s.long_rows, nsel, nrows, st);
  k_long_mask<<<nblocks(ntiles, 128), 128, 0, st>>>(nrows, ntiles, is_long, s.long_mask);
  count_launches(3);
  cudaMemcpyAsync(&h_nlong, nsel, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&h_nnz_s, s.ptr_s + nrows, sizeof(int), cudaMemcpyDeviceToHost, st);
  if ((err = cudaStreamSynchronize(st))) goto fail;
  s.lay.n_long = h_nlong;
  s.lay.n_long_tiles = (h_nlong + kTileRows - 1) / kTileRows;
  s.nnz_short = h_nnz_s;
  if ((err = cudaMalloc(&s.idx_s, (size_t)std::max(h_nnz_s, 1) * sizeof(int)))) goto fail;
  if ((err = cudaMalloc(&s.val64_s, (size_t)std::max(h_nnz_s, 1) * sizeof(double)))) goto fail;
  if (with32 && (err = cudaMalloc(&s.val32_s, (size_t)std::max(h_nnz_s, 1) * sizeof(float))))
    goto fail;
  if ((err = cudaMalloc(&s.ptr_l, (size_t)(h_nlong + 1) * sizeof(int)))) goto fail;
  if ((err = cudaMalloc(&len_l, (size_t)(h_nlong + 1) * sizeof(int)))) goto fail;
  k_copy_short<<<nblocks(nrows, 128), 128, 0, st>>>(nrows, ptr, idx, val, rscale, cscale,
                                                     s.ptr_s, s.idx_s, s.val64_s, s.val32_s, L);
  k_long_lengths<<<nblocks(h_nlong + 1, 256), 256, 0, st>>>(h_nlong, s.long_rows, ptr, len_l);
  count_launches(2 + (h_nlong > 0 ? 1 : 0));
  cub::DeviceScan::ExclusiveSum(nullptr, tb3, len_l, s.ptr_l, h_nlong + 1, st);
  if (tb3 > tb) {
    cudaFree(tmp);
    tmp = nullptr;
    tb = tb3;
    if ((err = cudaMalloc(&tmp, tb))) goto fail;
  }
  cub::DeviceScan::ExclusiveSum(tmp, tb, len_l, s.ptr_l, h_nlong + 1, st);
  cudaMemcpyAsync(&h_nnz_l, s.ptr_l + h_nlong, sizeof(int), cudaMemcpyDeviceToHost, st);
  if ((err = cudaStreamSynchronize(st))) goto fail;
  s.nnz_long = h_nnz_l;
  if ((err = cudaMalloc(&s.idx_l, (size_t)std::max(h_nnz_l, 1) * sizeof(int)))) goto fail;
  if ((err = cudaMalloc(&s.val64_l, (size_t)std::max(h_nnz_l, 1) * sizeof(double)))) goto fail;
  if (with32 && (err = cudaMalloc(&s.val32_l, (size_t)std::max(h_nnz_l, 1) * sizeof(float))))
    goto fail;
  if (h_nlong > 0)
    k_copy_long<<<nblocks((long long)h_nlong * 32, 128), 128, 0, st>>>(
        h_nlong, s.long_rows, ptr, idx, val, rscale, cscale, s.ptr_l, s.idx_l, s.val64_l,
        s.val32_l);
  if ((err = cudaStreamSynchronize(st))) goto fail;
  if ((err = cudaGetLastError())) goto fail;
  {
    // chunks of the long rows (host-side: n_long + 1 offsets)
    std::vector<int> hpl(h_nlong + 1), hcp(h_nlong + 1), hcr;
    if ((err = cudaMemcpy(hpl.data(), s.ptr_l, (h_nlong + 1) * sizeof(int),
                          cudaMemcpyDeviceToHost)))
      goto fail;
    hcp[0] = 0;
    for (int i = 0; i < h_nlong; ++i) {
      const int len = hpl[i + 1] - hpl[i];
      const int nc = (len + kChunk - 1) / kChunk;
      hcp[i + 1] = hcp[i] + nc;
      for (int c = 0; c < nc; ++c) hcr.push_back(i);
    }
    const int nch = hcp[h_nlong];
    s.lay.n_chunks = nch;
    if ((err = cudaMalloc(&s.chunk_ptr, (size_t)(h_nlong + 1) * sizeof(int)))) goto fail;
    if ((err = cudaMalloc(&s.chunk_row, (size_t)std::max(nch, 1) * sizeof(int)))) goto fail;
    if ((err = cudaMalloc(&s.part_a, (size_t)std::max(nch, 1) * sizeof(double)))) goto fail;
    if ((err = cudaMalloc(&s.part_b, (size_t)std::max(nch, 1) * sizeof(double)))) goto fail;
    const size_t ng = (size_t)std::max(s.lay.n_long_tiles, 1);
    if ((err = cudaMalloc(&s.done_a, ng * sizeof(unsigned int)))) goto fail;
    if ((err = cudaMalloc(&s.done_b, ng * sizeof(unsigned int)))) goto fail;
    if ((err = cudaMalloc(&s.gpart_a, ng * kMaxPartials * sizeof(double)))) goto fail;
    if ((err = cudaMalloc(&s.gpart_b, ng * kMaxPartials * sizeof(double)))) goto fail;
    if ((err = cudaMemcpy(s.chunk_ptr, hcp.data(), (h_nlong + 1) * sizeof(int),
                          cudaMemcpyHostToDevice)))
      goto fail;
    if (nch > 0 && (err = cudaMemcpy(s.chunk_row, hcr.data(), nch * sizeof(int),
                                     cudaMemcpyHostToDevice)))
      goto fail;
    if ((err = cudaMemset(s.done_a, 0, ng * sizeof(unsigned int)))) goto fail;
    if ((err = cudaMemset(s.done_b, 0, ng * sizeof(unsigned int)))) goto fail;
  }
  cudaFree(len_s);
  cudaFree(is_long);
  cudaFree(iota);
  cudaFree(nsel);
  cudaFree(len_l);
  cudaFree(tmp);
  s.lay.ptr_s = s.ptr_s;
  s.lay.idx_s = s.idx_s;
  s.lay.long_mask = s.long_mask;
  s.lay.long_rows = s.long_rows;
  s.lay.ptr_l = s.ptr_l;
  s.lay.idx_l = s.idx_l;
  s.lay.chunk_ptr = s.chunk_ptr;
  s.lay.chunk_row = s.chunk_row;
  s.v64.s = s.val64_s;
  s.v64.l = s.val64_l;
  s.v32.s = s.val32_s;
  s.v32.l = s.val32_l;
  s.wa.chunk_part = s.part_a;
  s.wa.group_done = s.done_a;
  s.wa.group_part = s.gpart_a;
  s.wb.chunk_part = s.part_b;
  s.wb.group_done = s.done_b;
  s.wb.group_part = s.gpart_b;
  *out = s;
  return cudaSuccess;
fail:
  cudaFree(len_s);
  cudaFree(is_long);
  cudaFree(iota);
  cudaFree(nsel);
  cudaFree(len_l);
  cudaFree(tmp);
  free_side(&s);
  return err;
}

void free_side(SideStore *s) {
  void *bufs[] = {s->ptr_s, s->idx_s, s->long_mask, s->long_rows, s->ptr_l, s->idx_l,
                  s->chunk_ptr, s->chunk_row, s->val64_s, s->val64_l, s->val32_s, s->val32_l,
                  s->part_a, s->part_b, s->done_a, s->done_b, s->gpart_a, s->gpart_b};
  for (void *b : bufs) cudaFree(b);
  *s = SideStore();
}

int choose_short_threshold(const int *h_ptr, int nrows) {
  // Short rows are staged for a whole 32-row tile in shared memory (32 * L products per warp);
  // longer rows go to the chunked warp-per-chunk path.  Pick the smallest L in {8, 16, 32, 64}
  // that keeps at least 90% of the rows short.
  if (nrows <= 0) return 8;
  std::vector<int> len(nrows);
  for (int i = 0; i < nrows; ++i) len[i] = h_ptr[i + 1] - h_ptr[i];
  const int cands[4] = {8, 16, 32, 64};
  for (int L : cands) {
    long long nshort = 0;
    for (int i = 0; i < nrows; ++i) nshort += (len[i] <= L);
    if (nshort >= (long long)(0.90 * nrows)) return L;
  }
  return 64;
}

int tile_grid(const SideLayout &lay, int sm_count, int blocks_per_sm) {
  long long need = ((long long)lay.total_items() + kBlockWarps - 1) / kBlockWarps;
  long long cap = (long long)sm_count * std::max(blocks_per_sm, 1);
  long long g = std::min(need, cap);
  return (int)std::max<long long>(g, 1);
}

void allow_large_smem_setup(int bytes) {
  cudaFuncSetAttribute(k_side_spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void side_spmv(cudaStream_t st, const SideStore &side, const double *src, double *out, int grid) {
  int smem = kBlockWarps * kTileRows * side.lay.L * (int)sizeof(double);
  k_side_spmv<<<grid, kBlockThreads, smem, st>>>(side.lay, side.v64, side.wa, src, out);
  count_launches(1);
}

void sumsq(cudaStream_t st, int n, const double *x, double *out, double *tmp) {
  k_sumsq_part<<<256, 256, 0, st>>>(n, x, tmp);
  k_sum_final<<<1, 256, 0, st>>>(256, tmp, out);
  count_launches(2);
}

void normalize(cudaStream_t st, int n, const double *w, const double *ss, double *v) {
  k_normalize<<<nblocks(n, 256), 256, 0, st>>>(n, w, ss, v);
  count_launches(1);
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
