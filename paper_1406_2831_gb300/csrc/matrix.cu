// Sparse-matrix setup (rbicgstab_set_matrix): CSR validation, SELL-32
// re-layout, transpose, and the generic SpMV used outside the fused passes.
//
// The API takes CSR (the storage the paper's problem statement implies for a
// "large, sparse" A, Sec. 1).  On the device the matrix is kept as SELL-32:
// 32 consecutive rows per slice, entries of a slice stored column by column
// (entry j of every row of the slice is one 32-wide coalesced line), each
// slice padded to its longest row with (col = row, val = 0).  Stencil rows
// differ in length only at the boundary, so padding is small.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "device.cuh"
#include "kernels.h"

namespace rb {

namespace {
// Device scratch freed on every return path.
struct DeviceScratch {
  void* p = nullptr;
  ~DeviceScratch() {
    if (p) cudaFree(p);
  }
};
}  // namespace

__global__ void k_fill_i32(int64_t cnt, int32_t* __restrict__ p, int32_t v) {
  for (int64_t i = gtid(); i < cnt; i += gstride()) p[i] = v;
}

// ---------------------------------------------------------------- validation
__global__ void k_validate_rows(int64_t n, int64_t nnz, const int32_t* __restrict__ rp, int* flag) {
  for (int64_t i = gtid(); i <= n; i += gstride()) {
    const int32_t a = rp[i];
    bool bad = (a < 0) || ((int64_t)a > nnz);
    if (i == 0) bad |= (a != 0);
    if (i == n) bad |= ((int64_t)a != nnz);
    if (i < n) bad |= (rp[i + 1] < a);
    if (bad) atomicMax(flag, 1);
  }
}

__global__ void k_validate_entries(int64_t n, int64_t nnz, const int32_t* __restrict__ col,
                                   const double* __restrict__ val, int* flag) {
  for (int64_t e = gtid(); e < nnz; e += gstride()) {
    const int32_t c = col[e];
    if (c < 0 || (int64_t)c >= n) atomicMax(flag, 1);
    if (val && !isfinite(val[e])) atomicMax(flag, 2);
  }
}

int csr_validate(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                 const double* val, int* d_flag, int* bad, cudaStream_t s) {
  count_launches(2);
  RB_CUDA_TRY(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
  int grid = (int)std::min<int64_t>((n + kBlock) / kBlock + 1, 4096);
  k_validate_rows<<<grid, kBlock, 0, s>>>(n, nnz, row_ptr, d_flag);
  if (nnz > 0) {
    int g2 = (int)std::min<int64_t>((nnz + kBlock - 1) / kBlock, 8192);
    k_validate_entries<<<g2, kBlock, 0, s>>>(n, nnz, col, val, d_flag);
  }
  RB_CUDA_TRY(cudaGetLastError());
  int h = 0;
  RB_CUDA_TRY(cudaMemcpyAsync(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  RB_CUDA_TRY(cudaStreamSynchronize(s));
  *bad = (h & 1) ? RB_EBADCSR : (h & 2) ? RB_ENONFINITE : 0;
  return RB_OK;
}

// ---------------------------------------------------------------- SELL-32
__global__ void k_slice_width(int64_t n, int64_t nslices, const int32_t* __restrict__ rp,
                              int32_t* __restrict__ width) {
  for (int64_t sl = gtid(); sl < nslices; sl += gstride()) {
    int w = 0;
    for (int l = 0; l < kSlice; ++l) {
      const int64_t r = sl * kSlice + l;
      if (r < n) w = max(w, rp[r + 1] - rp[r]);
    }
    width[sl] = w;
  }
}

// Stencil slices (see Sell in common.cuh): the sorted union of the column
// offsets of the slice's rows, kept when it has exactly `width` members (no
// extra entries) and every row's gathers stay inside [0, n).  One thread per
// slice; the search is quadratic in the width, which is small.
__global__ void k_slice_stencil(int64_t n, int64_t nslices, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const int32_t* __restrict__ width,
                                int stride, int32_t* __restrict__ offs, unsigned long long* count) {
  for (int64_t sl = gtid(); sl < nslices; sl += gstride()) {
    const int w = width[sl];
    const int64_t r0 = sl * kSlice;
    bool ok = w > 0 && w <= stride && r0 + kSlice <= n;
    int32_t O[kMaxStencil];
    int u = 0;
    for (int l = 0; ok && l < kSlice; ++l) {
      const int64_t r = r0 + l;
      for (int64_t e = rp[r]; ok && e < rp[r + 1]; ++e) {
        const int32_t d = (int32_t)((int64_t)col[e] - r);
        int pos = 0;
        while (pos < u && O[pos] < d) ++pos;
        if (pos < u && O[pos] == d) continue;
        if (u == w) {
          ok = false;
          break;
        }
        for (int q = u; q > pos; --q) O[q] = O[q - 1];
        O[pos] = d;
        ++u;
      }
    }
    ok = ok && u == w && r0 + O[0] >= 0 && r0 + kSlice - 1 + O[u - 1] < n;
    for (int j = 0; j < stride; ++j) offs[sl * stride + j] = ok && j < w ? O[j] : 0;
    if (!ok) offs[sl * stride] = kNoStencil;
    else atomicAdd(count, 1ull);
  }
}

// SELL entries: CSR order (padding (row, 0) at the end of short rows), or,
// for a stencil slice, offset order with (r + o_j, 0) where row r lacks o_j.
__global__ void k_sell_fill(int64_t n, int64_t nslices, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ col, const int64_t* __restrict__ sp,
                            const int32_t* __restrict__ width, const int32_t* __restrict__ offs, int stride,
                            int32_t* __restrict__ scol, int64_t* __restrict__ perm) {
  const int64_t total = nslices * kSlice;
  for (int64_t r = gtid(); r < total; r += gstride()) {
    const int64_t sl = r / kSlice;
    const int lane = (int)(r % kSlice);
    const int w = width[sl];
    const int64_t b = (r < n) ? rp[r] : 0;
    const int len = (r < n) ? (int)(rp[r + 1] - b) : 0;
    const bool stencil = offs[sl * stride] != kNoStencil;
    for (int j = 0; j < w; ++j) {
      const int64_t pos = sp[sl] + (int64_t)j * kSlice + lane;
      if (stencil) {
        const int32_t c = (int32_t)(r + offs[sl * stride + j]);
        int64_t src = -1;
        for (int e = 0; e < len; ++e)
          if (col[b + e] == c) {
            src = b + e;
            break;
          }
        scol[pos] = c;
        perm[pos] = src;
      } else if (j < len) {
        scol[pos] = col[b + j];
        perm[pos] = b + j;
      } else {
        scol[pos] = (int32_t)r;
        perm[pos] = -1;
      }
    }
  }
}

template <typename T>
__global__ void k_sell_values(int64_t cap, const int64_t* __restrict__ perm,
                              const double* __restrict__ v, T* __restrict__ out) {
  for (int64_t e = gtid(); e < cap; e += gstride()) {
    const int64_t p = perm[e];
    out[e] = (p >= 0) ? (T)v[p] : T(0);
  }
}

template <typename T>
void sell_free(SellBuf<T>* b) {
  cudaFree(b->slice_ptr);
  cudaFree(b->width);
  cudaFree(b->col);
  cudaFree(b->val);
  cudaFree(b->perm);
  cudaFree(b->offs);
  *b = SellBuf<T>();
}
template void sell_free<double>(SellBuf<double>*);
template void sell_free<float>(SellBuf<float>*);

int sell_build(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
               SellBuf<double>* out, cudaStream_t s, bool allow_stencil) {
  count_launches(3);
  sell_free(out);
  const int64_t nslices = (n + kSlice - 1) / kSlice;
  out->nslices = nslices;
  RB_CUDA_TRY(cudaMalloc(&out->width, sizeof(int32_t) * std::max<int64_t>(nslices, 1)));
  RB_CUDA_TRY(cudaMalloc(&out->slice_ptr, sizeof(int64_t) * (nslices + 1)));
  int grid = (int)std::min<int64_t>((nslices + kBlock - 1) / kBlock + 1, 4096);
  k_slice_width<<<grid, kBlock, 0, s>>>(n, nslices, row_ptr, out->width);
  RB_CUDA_TRY(cudaGetLastError());
  std::vector<int32_t> w(nslices);
  std::vector<int64_t> sp(nslices + 1);
  if (nslices)
    RB_CUDA_TRY(cudaMemcpyAsync(w.data(), out->width, sizeof(int32_t) * nslices,
                                cudaMemcpyDeviceToHost, s));
  RB_CUDA_TRY(cudaStreamSynchronize(s));
  sp[0] = 0;
  for (int64_t i = 0; i < nslices; ++i) sp[i + 1] = sp[i] + (int64_t)w[i] * kSlice;
  out->cap = sp[nslices];
  RB_CUDA_TRY(cudaMemcpyAsync(out->slice_ptr, sp.data(), sizeof(int64_t) * (nslices + 1),
                              cudaMemcpyHostToDevice, s));
  const int64_t cap = std::max<int64_t>(out->cap, 1);
  RB_CUDA_TRY(cudaMalloc(&out->col, sizeof(int32_t) * cap));
  RB_CUDA_TRY(cudaMalloc(&out->val, sizeof(double) * cap));
  RB_CUDA_TRY(cudaMalloc(&out->perm, sizeof(int64_t) * cap));
  int wmax = 0;
  for (int64_t i = 0; i < nslices; ++i) wmax = std::max(wmax, w[i]);
  int stride = 1;
  while (stride < wmax && stride < kMaxStencil) stride *= 2;
  out->offs_stride = stride;
  RB_CUDA_TRY(cudaMalloc(&out->offs, sizeof(int32_t) * std::max<int64_t>(nslices * stride, 1)));
  DeviceScratch cnt;
  RB_CUDA_TRY(cudaMalloc(&cnt.p, sizeof(unsigned long long)));
  unsigned long long* dcount = static_cast<unsigned long long*>(cnt.p);
  RB_CUDA_TRY(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s));
  // RB_SELL_GENERIC in the environment keeps every slice in CSR order (the
  // stencil layout's results are bitwise equal; this switch lets tests check it)
  if (nslices && allow_stencil && getenv("RB_SELL_GENERIC") == nullptr) {
    k_slice_stencil<<<grid, kBlock, 0, s>>>(n, nslices, row_ptr, col, out->width, stride, out->offs, dcount);
    RB_CUDA_TRY(cudaGetLastError());
  } else if (nslices) {
    k_fill_i32<<<grid, kBlock, 0, s>>>(nslices * stride, out->offs, kNoStencil);
    RB_CUDA_TRY(cudaGetLastError());
  }
  int g2 = (int)std::min<int64_t>((nslices * kSlice + kBlock - 1) / kBlock + 1, 16384);
  k_sell_fill<<<g2, kBlock, 0, s>>>(n, nslices, row_ptr, col, out->slice_ptr, out->width, out->offs, stride,
                                    out->col, out->perm);
  RB_CUDA_TRY(cudaGetLastError());
  unsigned long long hcount = 0;
  RB_CUDA_TRY(cudaMemcpyAsync(&hcount, dcount, sizeof(hcount), cudaMemcpyDeviceToHost, s));
  RB_CUDA_TRY(cudaStreamSynchronize(s));  // keeps host vectors alive until copies finish
  out->stencil_slices = (int64_t)hcount;
  return RB_OK;
}

template <typename T>
int sell_fill_values(const SellBuf<T>& out, const double* csr_val, cudaStream_t s) {
  count_launches(1);
  if (out.cap == 0) return RB_OK;
  int grid = (int)std::min<int64_t>((out.cap + kBlock - 1) / kBlock, 16384);
  k_sell_values<T><<<grid, kBlock, 0, s>>>(out.cap, out.perm, csr_val, out.val);
  RB_CUDA_TRY(cudaGetLastError());
  return RB_OK;
}
template int sell_fill_values<double>(const SellBuf<double>&, const double*, cudaStream_t);
template int sell_fill_values<float>(const SellBuf<float>&, const double*, cudaStream_t);

// ---------------------------------------------------------------- transpose
__global__ void k_col_count(int64_t nnz, const int32_t* __restrict__ col, int32_t* cnt) {
  for (int64_t e = gtid(); e < nnz; e += gstride()) atomicAdd(cnt + col[e], 1);
}

__global__ void k_scatter_t(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ trp, int32_t* fill, int32_t* tcol,
                            int64_t* tsrc) {
  for (int64_t r = gtid(); r < n; r += gstride()) {
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int32_t c = col[e];
      const int64_t pos = trp[c] + atomicAdd(fill + c, 1);
      tcol[pos] = (int32_t)r;
      tsrc[pos] = e;
    }
  }
}

// Exclusive prefix sums of the column counts (the row pointers of A^T),
// out[0..n]: three passes so that every load is coalesced.  The counts are
// cut into kScanSeg segments; each block sums one segment in tiles of
// kScanThreads consecutive entries (k_scan_sums), one block scans the
// segment sums (k_scan_offsets), and each block then scans its segment tile
// by tile (warp shuffles, then the warp totals), adding the segment's offset
// and the running tile carry (k_scan_write).  Integer adds: exact, any order.
constexpr int kScanThreads = 1024;
constexpr int kScanSeg = 512;

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;   // inclusive over warps
  }
  __syncthreads();
  const int64_t r = v + (warp > 0 ? warp_tot[warp - 1] : 0);
  __syncthreads();   // warp_tot is reused by the next call
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t n, const int32_t* __restrict__ cnt,
                                                            int64_t* __restrict__ seg_sum) {
  __shared__ int64_t red[kScanThreads / 32];
  const int64_t per = (n + kScanSeg - 1) / kScanSeg;
  const int64_t lo = std::min<int64_t>(n, (int64_t)blockIdx.x * per), hi = std::min<int64_t>(n, lo + per);
  int64_t s = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kScanThreads) s += cnt[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    seg_sum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_offsets(int64_t* seg_sum) {
  __shared__ int64_t wt[kScanThreads / 32];
  const int64_t v = threadIdx.x < kScanSeg ? seg_sum[threadIdx.x] : 0;
  const int64_t incl = block_incl_scan(v, wt);
  if (threadIdx.x < kScanSeg) seg_sum[threadIdx.x] = incl - v;   // exclusive
}

__global__ void __launch_bounds__(kScanThreads) k_scan_write(int64_t n, const int32_t* __restrict__ cnt,
                                                             const int64_t* __restrict__ seg_off,
                                                             int32_t* __restrict__ out) {
  __shared__ int64_t wt[kScanThreads / 32];
  __shared__ int64_t carry;
  const int64_t per = (n + kScanSeg - 1) / kScanSeg;
  const int64_t lo = std::min<int64_t>(n, (int64_t)blockIdx.x * per), hi = std::min<int64_t>(n, lo + per);
  if (threadIdx.x == 0) carry = seg_off[blockIdx.x];
  __syncthreads();
  for (int64_t base = lo; base < hi; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < hi ? cnt[i] : 0;
    const int64_t incl = block_incl_scan(v, wt);
    const int64_t c = carry;
    if (i < hi) out[i] = (int32_t)(c + incl - v);
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = c + incl;
    __syncthreads();
  }
  if (blockIdx.x == kScanSeg - 1 && threadIdx.x == 0) out[n] = (int32_t)carry;
}

// Entries of one row of A^T arrive in arbitrary order; sort each row by its
// column index (row of A) so the result is deterministic.  Short rows (the
// stencil case) by insertion sort, longer ones by heapsort (O(m log m)).
__device__ void sift_down(int32_t* key, int64_t* val, int64_t root, int64_t len) {
  for (;;) {
    int64_t child = 2 * root + 1;
    if (child >= len) return;
    if (child + 1 < len && key[child + 1] > key[child]) ++child;
    if (key[root] >= key[child]) return;
    const int32_t k = key[root];
    key[root] = key[child];
    key[child] = k;
    const int64_t v = val[root];
    val[root] = val[child];
    val[child] = v;
    root = child;
  }
}

__global__ void k_sort_rows(int64_t n, const int32_t* __restrict__ trp, int32_t* tcol, int64_t* tsrc) {
  for (int64_t r = gtid(); r < n; r += gstride()) {
    const int64_t b = trp[r], e = trp[r + 1], len = e - b;
    if (len <= 32) {
      for (int64_t i = b + 1; i < e; ++i) {
        const int32_t c = tcol[i];
        const int64_t s = tsrc[i];
        int64_t j = i - 1;
        while (j >= b && tcol[j] > c) {
          tcol[j + 1] = tcol[j];
          tsrc[j + 1] = tsrc[j];
          --j;
        }
        tcol[j + 1] = c;
        tsrc[j + 1] = s;
      }
    } else {
      int32_t* key = tcol + b;
      int64_t* val = tsrc + b;
      for (int64_t i = len / 2 - 1; i >= 0; --i) sift_down(key, val, i, len);
      for (int64_t end2 = len - 1; end2 > 0; --end2) {
        const int32_t k = key[0];
        key[0] = key[end2];
        key[end2] = k;
        const int64_t v = val[0];
        val[0] = val[end2];
        val[end2] = v;
        sift_down(key, val, 0, end2);
      }
    }
  }
}

int csr_transpose(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                  int32_t* t_row_ptr, int32_t* t_col, int64_t* t_src, cudaStream_t s) {
  count_launches(4);
  DeviceScratch tmp;
  RB_CUDA_TRY(cudaMalloc(&tmp.p, sizeof(int32_t) * (n + 1)));
  int32_t* cnt = static_cast<int32_t*>(tmp.p);
  RB_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), s));
  if (nnz > 0) {
    int g = (int)std::min<int64_t>((nnz + kBlock - 1) / kBlock, 16384);
    k_col_count<<<g, kBlock, 0, s>>>(nnz, col, cnt);
    RB_CUDA_TRY(cudaGetLastError());
  }
  {
    DeviceScratch segs;
    RB_CUDA_TRY(cudaMalloc(&segs.p, sizeof(int64_t) * kScanSeg));
    int64_t* seg = static_cast<int64_t*>(segs.p);
    count_launches(3);
    k_scan_sums<<<kScanSeg, kScanThreads, 0, s>>>(n, cnt, seg);
    k_scan_offsets<<<1, kScanThreads, 0, s>>>(seg);
    k_scan_write<<<kScanSeg, kScanThreads, 0, s>>>(n, cnt, seg, t_row_ptr);
    RB_CUDA_TRY(cudaGetLastError());
    RB_CUDA_TRY(cudaStreamSynchronize(s));   // the scratch is freed at the end of this scope
  }
  RB_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), s));
  int g = (int)std::min<int64_t>((n + kBlock - 1) / kBlock + 1, 16384);
  k_scatter_t<<<g, kBlock, 0, s>>>(n, row_ptr, col, t_row_ptr, cnt, t_col, t_src);
  RB_CUDA_TRY(cudaGetLastError());
  k_sort_rows<<<g, kBlock, 0, s>>>(n, t_row_ptr, t_col, t_src);
  RB_CUDA_TRY(cudaGetLastError());
  RB_CUDA_TRY(cudaStreamSynchronize(s));
  return RB_OK;
}

__global__ void k_gather(int64_t nnz, const int64_t* __restrict__ src, const double* __restrict__ v,
                         double* __restrict__ out) {
  for (int64_t e = gtid(); e < nnz; e += gstride()) out[e] = v[src[e]];
}

int gather_values(int64_t nnz, const int64_t* t_src, const double* val, double* t_val,
                  cudaStream_t s) {
  count_launches(1);
  if (nnz == 0) return RB_OK;
  int g = (int)std::min<int64_t>((nnz + kBlock - 1) / kBlock, 16384);
  k_gather<<<g, kBlock, 0, s>>>(nnz, t_src, val, t_val);
  RB_CUDA_TRY(cudaGetLastError());
  return RB_OK;
}

// ---------------------------------------------------------------- SpMV
template <typename T>
__global__ void __launch_bounds__(kBlock) k_spmv(Sell<T> A, const T* __restrict__ v, T* __restrict__ y,
                                                double alpha, double beta) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = gtid() >> 5, nw = gstride() >> 5;
  for (int64_t sl = w0; sl < A.nslices; sl += nw) {
    const int64_t row = sl * kSlice + lane;
    const int w = A.width[sl];
    const int64_t base = A.slice_ptr[sl] + lane;
    T acc = T(0);
    for (int j = 0; j < w; ++j) {
      const int64_t e = base + (int64_t)j * kSlice;
      acc = fma_t(A.val[e], v[A.col[e]], acc);
    }
    const T out = (T)alpha * acc;
    y[row] = (beta == 0.0) ? out : fma_t((T)beta, y[row], out);
  }
}

template <typename T>
cudaError_t spmv(const Sell<T>& A, const T* v, T* y, double alpha, double beta, int grid,
                 cudaStream_t s) {
  count_launches(1);
  k_spmv<T><<<grid, kBlock, 0, s>>>(A, v, y, alpha, beta);
  return cudaGetLastError();
}
template cudaError_t spmv<double>(const Sell<double>&, const double*, double*, double, double, int,
                                  cudaStream_t);
template cudaError_t spmv<float>(const Sell<float>&, const float*, float*, double, double, int,
                                 cudaStream_t);

}  // namespace rb
