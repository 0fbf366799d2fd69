// Generic FP64 kernels used outside the fused iteration: the setup of a
// solve (eq. (3.5)), the end of a solve (the final correction of Alg. 2 and the true
// residual), and the recycle-space work (Gram matrices, block updates).
// All reductions are deterministic (fixed trees, no floating-point atomics).
#include <algorithm>

#include <type_traits>

#include "device.cuh"
#include "kernels.h"

namespace rb {

// ---------------------------------------------------------------- dots
template <int KMAX>
__global__ void __launch_bounds__(kBlock) k_dots(DotArgs d, int64_t npad, IterState* st, double* partials) {
  constexpr int NV = KMAX + 4;
  __shared__ ReduceSmem<NV> sm;
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  const double* __restrict__ Mp = d.M;
  const int km = d.km;
  for (int64_t i = gtid(); i < npad; i += gstride()) {
    if (Mp) {
      // every column load of the row is issued before the first FMA
      const double vi = __ldg(d.v + i);
      double mv[KMAX > 0 ? KMAX : 1];
#pragma unroll
      for (int j = 0; j < KMAX; ++j) mv[j] = j < km ? __ldg(Mp + j * d.ld + i) : 0.0;
#pragma unroll
      for (int j = 0; j < KMAX; ++j) acc[j] = fma(mv[j], vi, acc[j]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < d.nd) acc[KMAX + q] = fma(d.a[q][i], d.b[q][i], acc[KMAX + q]);
  }
  if (block_reduce_last<NV>(acc, KMAX + 4, sm, partials, &st->ticket[PGEN])) {
    if (threadIdx.x < d.km) st->red[threadIdx.x] = sm.res[threadIdx.x];
    if (threadIdx.x < d.nd) st->red[d.km + threadIdx.x] = sm.res[KMAX + threadIdx.x];
  }
}

cudaError_t dots(const DotArgs& d, int64_t npad, IterState* st, double* partials, int grid,
                 cudaStream_t s) {
  count_launches(1);
  const int km = d.M ? d.km : 0;
  DotArgs dd = d;
  dd.km = km;
  switch (kmax_bucket(km)) {
    case 0: k_dots<0><<<grid, kBlock, 0, s>>>(dd, npad, st, partials); break;
    case 8: k_dots<8><<<grid, kBlock, 0, s>>>(dd, npad, st, partials); break;
    case 16: k_dots<16><<<grid, kBlock, 0, s>>>(dd, npad, st, partials); break;
    case 24: k_dots<24><<<grid, kBlock, 0, s>>>(dd, npad, st, partials); break;
    case 32: k_dots<32><<<grid, kBlock, 0, s>>>(dd, npad, st, partials); break;
    case 48: k_dots<48><<<grid, kBlock, 0, s>>>(dd, npad, st, partials); break;
    default: k_dots<64><<<grid, kBlock, 0, s>>>(dd, npad, st, partials); break;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- y += sign M c
__global__ void k_gemv_update(double* __restrict__ y, const double* __restrict__ M, int64_t ld, int k,
                              const double* __restrict__ c, const double* __restrict__ cs,
                              double sign, int64_t npad) {
  __shared__ double cc[kMaxK];
  if (threadIdx.x < k) cc[threadIdx.x] = sign * c[threadIdx.x] * (cs ? cs[threadIdx.x] : 1.0);
  __syncthreads();
  for (int64_t i = gtid(); i < npad; i += gstride()) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(M[j * ld + i], cc[j], acc);
    y[i] += acc;
  }
}

cudaError_t gemv_update(double* y, const double* M, int64_t ld, int k, const double* c,
                        const double* c_scale, double sign, int64_t npad, int grid,
                        cudaStream_t s) {
  count_launches(1);
  if (k <= 0) return cudaSuccess;
  k_gemv_update<<<grid, kBlock, 0, s>>>(y, M, ld, k, c, c_scale, sign, npad);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- y = a y + sum_t c_t x_t
__global__ void k_lincomb(double* __restrict__ y, double a, LinComb lc, int64_t npad) {
  for (int64_t i = gtid(); i < npad; i += gstride()) {
    double acc = a == 0.0 ? 0.0 : a * y[i];
    for (int t = 0; t < lc.nx; ++t) acc = fma(lc.c[t], lc.x[t][i], acc);
    y[i] = acc;
  }
}

cudaError_t lincomb(double* y, double a, const LinComb& lc, int64_t npad, int grid, cudaStream_t s) {
  count_launches(1);
  k_lincomb<<<grid, kBlock, 0, s>>>(y, a, lc, npad);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pattern outer product
// out[e] = scale * u[i] * v[col[e]] for every entry e of row i of a CSR
// pattern (one thread per row; rows of stencil operators are short).
__global__ void k_pattern_outer(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ u, const double* __restrict__ v, double scale,
                                double* __restrict__ out) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double su = scale * u[i];
    const int32_t e1 = rp[i + 1];
    for (int32_t e = rp[i]; e < e1; ++e) out[e] = su * v[ci[e]];
  }
}

cudaError_t pattern_outer(int64_t n, const int32_t* rp, const int32_t* ci, const double* u, const double* v,
                          double scale, double* out, int grid, cudaStream_t s) {
  count_launches(1);
  if (n <= 0) return cudaSuccess;
  k_pattern_outer<<<grid, kBlock, 0, s>>>(n, rp, ci, u, v, scale, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- block GEMM
// Out(:, c) = X R(:, c): each thread owns one row, reads the m entries of
// X's row once and forms all kc <= KC outputs in registers (KC is a
// compile-time bucket so the accumulators never spill to local memory).
template <typename T, int KC>
__global__ void __launch_bounds__(kBlock) k_gemm_cols(T* const* __restrict__ out, const T* const* __restrict__ X,
                                                     int m, const double* __restrict__ R, int kc, int64_t npad) {
  extern __shared__ __align__(16) unsigned char gem_sm[];
  T* sR = (T*)gem_sm;                              // m * KC coefficients (zero-padded)
  const T** sX = (const T**)(sR + (size_t)m * KC);  // m column pointers
  for (int e = threadIdx.x; e < m * KC; e += blockDim.x) {
    const int j = e / KC, c = e % KC;
    sR[e] = c < kc ? (T)R[j + (size_t)c * m] : T(0);
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) sX[j] = X[j];
  __syncthreads();
  constexpr int JB = 8;   // column loads issued together
  if constexpr (std::is_same<T, float>::value) {
    // two consecutive rows per thread (8-byte loads); each 16-byte broadcast
    // of four coefficients serves both rows on packed FMAs (each lane rounded
    // as fma_t, the columns summed in order j = 0, 1, ..: the products of the
    // one-row form, bit for bit)
    static_assert(KC % 4 == 0, "KC must be a multiple of 4");
    using P = Pair<float>;
    const int64_t nrow2 = npad / 2;
    for (int64_t i2 = gtid(); i2 < nrow2; i2 += gstride()) {
      const int64_t i = 2 * i2;
      float2 a0[KC / 2], a1[KC / 2];
#pragma unroll
      for (int c = 0; c < KC / 2; ++c) a0[c] = a1[c] = make_float2(0.0f, 0.0f);
      for (int j0 = 0; j0 < m; j0 += JB) {
        float2 xv[JB];
#pragma unroll
        for (int u = 0; u < JB; ++u)
          xv[u] = (j0 + u < m) ? __ldg(reinterpret_cast<const float2*>(sX[j0 + u] + i)) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < JB; ++u) {
          if (j0 + u >= m) break;
          const float4* rj = reinterpret_cast<const float4*>(sR + (size_t)(j0 + u) * KC);
          const float2 x0 = P::mk(xv[u].x, xv[u].x), x1 = P::mk(xv[u].y, xv[u].y);
#pragma unroll
          for (int c4 = 0; c4 < KC / 4; ++c4) {
            const float4 r = rj[c4];
            const float2 rlo = make_float2(r.x, r.y), rhi = make_float2(r.z, r.w);
            a0[2 * c4] = P::fma(x0, rlo, a0[2 * c4]);
            a0[2 * c4 + 1] = P::fma(x0, rhi, a0[2 * c4 + 1]);
            a1[2 * c4] = P::fma(x1, rlo, a1[2 * c4]);
            a1[2 * c4 + 1] = P::fma(x1, rhi, a1[2 * c4 + 1]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < KC / 2; ++c) {
        if (2 * c < kc) *reinterpret_cast<float2*>(out[2 * c] + i) = make_float2(a0[c].x, a1[c].x);
        if (2 * c + 1 < kc) *reinterpret_cast<float2*>(out[2 * c + 1] + i) = make_float2(a0[c].y, a1[c].y);
      }
    }
  } else {
    for (int64_t i = gtid(); i < npad; i += gstride()) {
      T acc[KC];
#pragma unroll
      for (int c = 0; c < KC; ++c) acc[c] = T(0);
      for (int j0 = 0; j0 < m; j0 += JB) {
        T xv[JB];
#pragma unroll
        for (int u = 0; u < JB; ++u) xv[u] = (j0 + u < m) ? __ldg(sX[j0 + u] + i) : T(0);
#pragma unroll
        for (int u = 0; u < JB; ++u) {
          if (j0 + u >= m) break;
          const T* rj = sR + (size_t)(j0 + u) * KC;
#pragma unroll
          for (int c = 0; c < KC; ++c) acc[c] = fma_t(xv[u], rj[c], acc[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < KC; ++c)
        if (c < kc) out[c][i] = acc[c];
    }
  }
}

template <typename T, int KC>
static cudaError_t gemm_cols_k(T* const* out, const T* const* X, int m, const double* R, int kc, int64_t npad,
                               int grid, cudaStream_t s) {
  const size_t smem = sizeof(T) * (size_t)m * KC + sizeof(void*) * (size_t)m;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_gemm_cols<T, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_gemm_cols<T, KC><<<grid, kBlock, smem, s>>>(out, X, m, R, kc, npad);
  return cudaGetLastError();
}

template <typename T>
cudaError_t gemm_cols(T* const* out, const T* const* X, int m, const double* R, int kc, int64_t npad,
                      int grid, cudaStream_t s) {
  count_launches(1);
  if (kc <= 0 || m <= 0) return cudaSuccess;
  if (kc <= 8) return gemm_cols_k<T, 8>(out, X, m, R, kc, npad, grid, s);
  if (kc <= 16) return gemm_cols_k<T, 16>(out, X, m, R, kc, npad, grid, s);
  if (kc <= 24) return gemm_cols_k<T, 24>(out, X, m, R, kc, npad, grid, s);
  if (kc <= 32) return gemm_cols_k<T, 32>(out, X, m, R, kc, npad, grid, s);
  if (kc <= 48) return gemm_cols_k<T, 48>(out, X, m, R, kc, npad, grid, s);
  return gemm_cols_k<T, 64>(out, X, m, R, kc, npad, grid, s);
}
template cudaError_t gemm_cols<double>(double* const*, const double* const*, int, const double*, int,
                                       int64_t, int, cudaStream_t);
template cudaError_t gemm_cols<float>(float* const*, const float* const*, int, const double*, int,
                                      int64_t, int, cudaStream_t);

// ---------------------------------------------------------------- Gram X^T Y
// Each block walks row tiles of 32 rows, stages X and Y tiles in shared
// memory, and accumulates the (a, b) products it owns (FP64 FMA for FP64
// columns, Dot2 for FP32 columns); block partials are reduced in block order
// by a second kernel.
constexpr int kGramRows = 32;

template <typename T>
__global__ void __launch_bounds__(kBlock) k_gram(const T* const* __restrict__ X, int mx,
                                                const T* const* __restrict__ Y, int my,
                                                int64_t npad, double* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char gsm[];
  T* sx = (T*)gsm;                        // kGramRows * mx
  T* sy = sx + kGramRows * mx;            // kGramRows * my
  const int nout = mx * my;
  const int per = (nout + blockDim.x - 1) / blockDim.x;   // outputs per thread (<= 32)
  Acc<T> acc[32];
  const int64_t ntiles = (npad + kGramRows - 1) / kGramRows;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * kGramRows;
    __syncthreads();
    for (int e = threadIdx.x; e < kGramRows * mx; e += blockDim.x) {
      const int a = e / kGramRows, rr = e % kGramRows;
      sx[rr * mx + a] = (r0 + rr < npad) ? X[a][r0 + rr] : T(0);
    }
    for (int e = threadIdx.x; e < kGramRows * my; e += blockDim.x) {
      const int b = e / kGramRows, rr = e % kGramRows;
      sy[rr * my + b] = (r0 + rr < npad) ? Y[b][r0 + rr] : T(0);
    }
    __syncthreads();
    for (int u = 0; u < per; ++u) {
      const int o = threadIdx.x + u * blockDim.x;
      if (o < nout) {
        const int a = o % mx, b = o / mx;
        Acc<T> sacc = acc[u];
#pragma unroll 8
        for (int rr = 0; rr < kGramRows; ++rr) sacc.add(sx[rr * mx + a], sy[rr * my + b]);
        acc[u] = sacc;
      }
    }
  }
  for (int u = 0; u < per; ++u) {
    const int o = threadIdx.x + u * blockDim.x;
    if (o < nout) work[(size_t)blockIdx.x * nout + o] = acc[u].get();
  }
}

__global__ void k_gram_reduce(const double* __restrict__ work, int nblocks, int nout, double* out) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += work[(size_t)b * nout + o];
    out[o] = s;
  }
}

template <typename T>
cudaError_t gram(const T* const* X, int mx, const T* const* Y, int my, int64_t npad, double* out,
                 double* work, int grid, cudaStream_t s) {
  count_launches(2);
  if (mx <= 0 || my <= 0) return cudaSuccess;
  if (mx * my > 32 * kBlock) return cudaErrorInvalidValue;
  const size_t smem = sizeof(T) * kGramRows * (size_t)(mx + my);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_gram<T><<<grid, kBlock, smem, s>>>(X, mx, Y, my, npad, work);
  const int nout = mx * my;
  k_gram_reduce<<<(nout + kBlock - 1) / kBlock, kBlock, 0, s>>>(work, grid, nout, out);
  return cudaGetLastError();
}
template cudaError_t gram<double>(const double* const*, int, const double* const*, int, int64_t, double*,
                                  double*, int, cudaStream_t);
template cudaError_t gram<float>(const float* const*, int, const float* const*, int, int64_t, double*,
                                 double*, int, cudaStream_t);

// ---------------------------------------------------------------- fused Gram
// One pass over the m columns of Z and W forms G = Z^T Z (upper triangle,
// a <= b) and H = Z^T W, the two matrices of the harmonic-Ritz step.  Rows
// are staged in shared memory 64 at a time; each thread owns up to two 4x4
// output tiles and reads 4 + 4 staged values per row for 16 products.
// Accumulation: FP64 FMA for FP64 columns, Dot2 for FP32 columns.  Block
// partials (block-major) are summed in block order by k_gram_reduce.
constexpr int kGR = 64;      // rows per shared-memory chunk
constexpr int kGT = 4;       // output tile edge
constexpr int kGC = 8;       // FP32 rows summed with plain FMAs before a compensated add

// Asynchronous element copy global -> shared (4 or 8 bytes), grouped per thread.
template <typename T>
__device__ __forceinline__ void cp_async_el(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_commit_g() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_g() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage rows [r0, r0 + kGR) of the m columns of Z and W (row-major tiles
// kGR x mp) with asynchronous copies; rows past npad are zeroed.
template <typename T>
__device__ __forceinline__ void gram_stage(const T* const* __restrict__ Z, const T* const* __restrict__ W, int m,
                                           int mp, int64_t r0, int64_t npad, T* sz, T* sw) {
  for (int e = threadIdx.x; e < kGR * m; e += blockDim.x) {
    const int c = e / kGR, rr = e % kGR;
    if (r0 + rr < npad) {
      cp_async_el(sz + rr * mp + c, Z[c] + r0 + rr);
      cp_async_el(sw + rr * mp + c, W[c] + r0 + rr);
    } else {
      sz[rr * mp + c] = T(0);
      sw[rr * mp + c] = T(0);
    }
  }
}

// The rows of a block are staged in two buffers: the copies of the next
// 64-row chunk are in flight while the current one is multiplied.
template <typename T, int TPT>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 2 : 1) k_gram_gh(const T* const* __restrict__ Z,
                                                   const T* const* __restrict__ W, int m, int mp,
                                                   int ntile_g, int ntile_h, int64_t npad,
                                                   double* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char ghsm[];
  T* sbuf = (T*)ghsm;             // 2 stages x (Z tile, W tile), kGR x mp each
  const int nt = mp / kGT;        // tiles per edge
  const int ntot = ntile_g + ntile_h;
  // this thread's tiles: t = threadIdx.x + q * blockDim.x, q < TPT
  int ta[TPT], tb[TPT], isg[TPT];
  int ntl = 0;
  for (int t = threadIdx.x; t < ntot && ntl < TPT; t += blockDim.x, ++ntl) {
    if (t < ntile_g) {   // upper-triangle tile index -> (row tile, col tile)
      int r = 0, rem = t;
      while (rem >= nt - r) { rem -= nt - r; ++r; }
      ta[ntl] = r; tb[ntl] = r + rem; isg[ntl] = 1;
    } else {
      const int u = t - ntile_g;
      ta[ntl] = u / nt; tb[ntl] = u % nt; isg[ntl] = 0;
    }
  }
  // FP32: pairs of output columns on packed instructions (same per-lane
  // rounding as the scalar form); FP64: one accumulator per entry
  constexpr bool F32 = std::is_same<T, float>::value;
  Acc<T> acc[F32 ? 1 : TPT][kGT][F32 ? 1 : kGT];
  AccP<float> accp[F32 ? TPT : 1][kGT][kGT / 2];
  const int64_t nch = (npad + kGR - 1) / kGR;
  const int tile_el = kGR * mp;
  // padding columns m..mp-1 stay zero in both stages
  for (int e = threadIdx.x; e < 2 * 2 * kGR * (mp - m); e += blockDim.x) {
    const int q = e / (kGR * (mp - m)), rem = e % (kGR * (mp - m));
    sbuf[q * tile_el + (rem / (mp - m)) * mp + m + rem % (mp - m)] = T(0);
  }
  if ((int64_t)blockIdx.x < nch)
    gram_stage<T>(Z, W, m, mp, (int64_t)blockIdx.x * kGR, npad, sbuf, sbuf + tile_el);
  cp_async_commit_g();
  int it = 0;
  for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x, ++it) {
    const int64_t nx = ch + gridDim.x;
    T* nz = sbuf + ((it + 1) & 1) * 2 * tile_el;
    if (nx < nch) gram_stage<T>(Z, W, m, mp, nx * kGR, npad, nz, nz + tile_el);
    cp_async_commit_g();
    cp_async_wait_g<1>();
    __syncthreads();
    const T* sz = sbuf + (it & 1) * 2 * tile_el;
    const T* sw = sz + tile_el;
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      if (q < ntl) {
        const T* za = sz + ta[q] * kGT;
        const T* yb = (isg[q] ? sz : sw) + tb[q] * kGT;
        if constexpr (F32) {
          // FP32 products summed with plain FMAs over kGC rows, each chunk
          // then added to the compensated (hi, lo) pair: per entry the error
          // is at most gamma_kGC * sum_i |z_i w_i| (gamma_8 ~ 4.8e-7), the
          // level of the FP32 columns themselves, at a quarter of the cost
          // of compensating every product.  Columns j, j+1 of a tile row go
          // through one packed FMA / TwoSum.
          using P = Pair<float>;
#pragma unroll 1
          for (int r0c = 0; r0c < kGR; r0c += kGC) {
            float2 p[kGT][kGT / 2];
#pragma unroll
            for (int i = 0; i < kGT; ++i)
#pragma unroll
              for (int j = 0; j < kGT / 2; ++j) p[i][j] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int rr = r0c; rr < r0c + kGC; ++rr) {
              const float4 a = *reinterpret_cast<const float4*>(za + rr * mp);
              const float4 b = *reinterpret_cast<const float4*>(yb + rr * mp);
              const float av[kGT] = {a.x, a.y, a.z, a.w};
              const float2 bv[kGT / 2] = {make_float2(b.x, b.y), make_float2(b.z, b.w)};
#pragma unroll
              for (int i = 0; i < kGT; ++i)
#pragma unroll
                for (int j = 0; j < kGT / 2; ++j) p[i][j] = P::fma(P::mk(av[i], av[i]), bv[j], p[i][j]);
            }
#pragma unroll
            for (int i = 0; i < kGT; ++i)
#pragma unroll
              for (int j = 0; j < kGT / 2; ++j) accp[q][i][j].add1(p[i][j]);
          }
        } else {
#pragma unroll 1
          for (int rr = 0; rr < kGR; ++rr) {
            T a[kGT], b[kGT];
#pragma unroll
            for (int u = 0; u < kGT; ++u) {
              a[u] = za[rr * mp + u];
              b[u] = yb[rr * mp + u];
            }
#pragma unroll
            for (int i = 0; i < kGT; ++i)
#pragma unroll
              for (int j = 0; j < kGT; ++j) acc[q][i][j].add(a[i], b[j]);
          }
        }
      }
    }
    __syncthreads();   // this stage is refilled two chunks on
  }
  cp_async_wait_g<0>();
  // block partials: G tiles then H tiles, 16 values per tile
  double* wb = work + (size_t)blockIdx.x * ntot * kGT * kGT;
  for (int q = 0; q < ntl; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
#pragma unroll
    for (int i = 0; i < kGT; ++i)
#pragma unroll
      for (int j = 0; j < kGT; ++j) {
        double v;
        if constexpr (F32) v = accp[q][i][j / 2].lane(j & 1).get();
        else v = acc[q][i][j].get();
        wb[(size_t)t * kGT * kGT + i * kGT + j] = v;
      }
  }
}

// Sum block partials in block order and scatter into G (m x m, both
// triangles) and H (m x m), column-major.
__global__ void k_gram_gh_reduce(const double* __restrict__ work, int nblocks, int m, int mp, int ntile_g,
                                 int ntile_h, double* __restrict__ G, double* __restrict__ H) {
  const int nt = mp / kGT, ntot = ntile_g + ntile_h;
  const int nval = ntot * kGT * kGT;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nval; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += work[(size_t)b * nval + o];
    const int t = o / (kGT * kGT), ij = o % (kGT * kGT), i = ij / kGT, j = ij % kGT;
    int a0, b0;
    bool g;
    if (t < ntile_g) {
      int r = 0, rem = t;
      while (rem >= nt - r) { rem -= nt - r; ++r; }
      a0 = r; b0 = r + rem; g = true;
    } else {
      a0 = (t - ntile_g) / nt; b0 = (t - ntile_g) % nt; g = false;
    }
    const int a = a0 * kGT + i, b = b0 * kGT + j;
    if (a >= m || b >= m) continue;
    if (g) {
      if (a <= b) {
        G[a + (size_t)b * m] = s;
        G[b + (size_t)a * m] = s;
      }
    } else {
      H[a + (size_t)b * m] = s;
    }
  }
}

int gram_gh_work(int m) {
  const int mp = (m + kGT - 1) / kGT * kGT, nt = mp / kGT;
  return (nt * (nt + 1) / 2 + nt * nt) * kGT * kGT;
}

template <typename T>
cudaError_t gram_gh(const T* const* Z, const T* const* W, int m, int64_t npad, double* G, double* H,
                    double* work, int grid, cudaStream_t s) {
  count_launches(2);
  if (m <= 0) return cudaSuccess;
  const int mp = (m + kGT - 1) / kGT * kGT, nt = mp / kGT;
  const int ntile_g = nt * (nt + 1) / 2, ntile_h = nt * nt;
  if (ntile_g + ntile_h > 4 * kBlock) return cudaErrorInvalidValue;
  const size_t smem = sizeof(T) * 2 * 2 * kGR * (size_t)mp;
  if (ntile_g + ntile_h <= 2 * kBlock) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_gram_gh<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gram_gh<T, 2><<<grid, kBlock, smem, s>>>(Z, W, m, mp, ntile_g, ntile_h, npad, work);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_gram_gh<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gram_gh<T, 4><<<grid, kBlock, smem, s>>>(Z, W, m, mp, ntile_g, ntile_h, npad, work);
  }
  const int nval = (ntile_g + ntile_h) * kGT * kGT;
  k_gram_gh_reduce<<<(nval + kBlock - 1) / kBlock, kBlock, 0, s>>>(work, grid, m, mp, ntile_g, ntile_h, G, H);
  return cudaGetLastError();
}
template cudaError_t gram_gh<double>(const double* const*, const double* const*, int, int64_t, double*,
                                     double*, double*, int, cudaStream_t);
template cudaError_t gram_gh<float>(const float* const*, const float* const*, int, int64_t, double*, double*,
                                    double*, int, cudaStream_t);

// ---------------------------------------------------------------- column norms
// out[j] = ||M(:, j)||^2 for column pointers M[0..k), deterministic.
template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_colnorm2(const T* const* __restrict__ M, int k, int64_t npad,
                                                    IterState* st, double* partials) {
  __shared__ ReduceSmem<KMAX> sm;
  Acc<T> acc[KMAX];
  for (int64_t i = gtid(); i < npad; i += gstride()) {
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) {
        const T v = M[j][i];
        acc[j].add(v, v);
      }
  }
  if (block_reduce_last<T, KMAX>(acc, k, sm, partials, &st->ticket[PGEN])) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) st->red[j] = sm.res[j];
  }
}

template <typename T>
cudaError_t colnorm2(const T* const* M, int k, int64_t npad, IterState* st, double* partials, int grid,
                     cudaStream_t s) {
  count_launches(1);
  if (k <= 0) return cudaSuccess;
  if (k <= 32) k_colnorm2<T, 32><<<grid, kBlock, 0, s>>>(M, k, npad, st, partials);
  else k_colnorm2<T, 64><<<grid, kBlock, 0, s>>>(M, k, npad, st, partials);
  return cudaGetLastError();
}
template cudaError_t colnorm2<double>(const double* const*, int, int64_t, IterState*, double*, int, cudaStream_t);
template cudaError_t colnorm2<float>(const float* const*, int, int64_t, IterState*, double*, int, cudaStream_t);

// ---------------------------------------------------------------- shadow r~_{-1}
// SplitMix64 (Steele, Lea, Flood 2014), output i from state `seed`:
// z = seed + (i+1)*golden gamma; two xor-shift-multiply rounds; final xor-shift.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_shadow(double* rt, int64_t n, int64_t npad, uint64_t seed) {
  for (int64_t i = gtid(); i < npad; i += gstride()) {
    if (i < n) {
      const uint64_t z = splitmix64_at(seed, (uint64_t)i);
      const double u = (double)(z >> 11) * 0x1.0p-53;
      rt[i] = 2.0 * u - 1.0;
    } else {
      rt[i] = 0.0;
    }
  }
}

cudaError_t shadow(double* rt, int64_t n, int64_t npad, uint64_t seed, cudaStream_t s) {
  count_launches(1);
  int g = (int)std::min<int64_t>((npad + kBlock - 1) / kBlock, 8192);
  k_shadow<<<g, kBlock, 0, s>>>(rt, n, npad, seed);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- column scaling
template <typename T>
__global__ void k_scale_cols(T* M, int64_t ld, int k, const double* f, int64_t npad) {
  for (int64_t i = gtid(); i < npad; i += gstride())
    for (int j = 0; j < k; ++j) M[j * ld + i] = (T)((double)M[j * ld + i] * f[j]);
}

template <typename T>
cudaError_t scale_cols(T* M, int64_t ld, int k, const double* f, int64_t npad, cudaStream_t s) {
  count_launches(1);
  if (k <= 0) return cudaSuccess;
  int g = (int)std::min<int64_t>((npad + kBlock - 1) / kBlock, 8192);
  k_scale_cols<T><<<g, kBlock, 0, s>>>(M, ld, k, f, npad);
  return cudaGetLastError();
}
template cudaError_t scale_cols<double>(double*, int64_t, int, const double*, int64_t, cudaStream_t);
template cudaError_t scale_cols<float>(float*, int64_t, int, const double*, int64_t, cudaStream_t);

// ---------------------------------------------------------------- residual
__global__ void __launch_bounds__(kBlock) k_residual(Sell<double> A, const double* __restrict__ b,
                                                    const double* __restrict__ x, double* __restrict__ r,
                                                    IterState* st, double* partials) {
  __shared__ ReduceSmem<1> sm;
  double acc[1] = {0.0};
  const int lane = threadIdx.x & 31;
  const int64_t w0 = gtid() >> 5, nw = gstride() >> 5;
  for (int64_t sl = w0; sl < A.nslices; sl += nw) {
    const int64_t row = sl * kSlice + lane;
    const int w = A.width[sl];
    const int64_t base = A.slice_ptr[sl] + lane;
    double y = 0.0;
    for (int j = 0; j < w; ++j) {
      const int64_t e = base + (int64_t)j * kSlice;
      y = fma(A.val[e], x[A.col[e]], y);
    }
    const double rv = b[row] - y;
    r[row] = rv;
    acc[0] = fma(rv, rv, acc[0]);
  }
  if (block_reduce_last<1>(acc, 1, sm, partials, &st->ticket[PGEN]) && threadIdx.x == 0)
    st->red[0] = sm.res[0];
}

cudaError_t residual_norm(const Sell<double>& A, const double* b, const double* x, double* r,
                          int64_t npad, IterState* st, double* partials, int grid,
                          cudaStream_t s) {
  count_launches(1);
  k_residual<<<grid, kBlock, 0, s>>>(A, b, x, r, st, partials);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- misc
__global__ void k_finite(const double* v, int64_t n, int* flag) {
  for (int64_t i = gtid(); i < n; i += gstride())
    if (!isfinite(v[i])) atomicMax(flag, 1);
}

cudaError_t check_finite(const double* v, int64_t n, int* flag, cudaStream_t s) {
  count_launches(1);
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (n == 0) return cudaGetLastError();
  int g = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 8192);
  k_finite<<<g, kBlock, 0, s>>>(v, n, flag);
  return cudaGetLastError();
}

__global__ void k_to_float(const double* in, float* out, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) out[i] = (float)in[i];
}
cudaError_t to_float(const double* in, float* out, int64_t n, cudaStream_t s) {
  count_launches(1);
  int g = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 8192);
  if (n > 0) k_to_float<<<g, kBlock, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

__global__ void k_to_double(const float* in, double* out, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) out[i] = (double)in[i];
}
cudaError_t to_double(const float* in, double* out, int64_t n, cudaStream_t s) {
  count_launches(1);
  int g = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 8192);
  if (n > 0) k_to_double<<<g, kBlock, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

__global__ void k_add_f2d(double* x, const float* d, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) x[i] += (double)d[i];
}
cudaError_t add_float_to_double(double* x, const float* d, int64_t n, cudaStream_t s) {
  count_launches(1);
  int g = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 8192);
  if (n > 0) k_add_f2d<<<g, kBlock, 0, s>>>(x, d, n);
  return cudaGetLastError();
}

// st->red holds [C^T r~_0 (k), (r~_0, r_0), (r_0, r_0)] from the last dots()
// call; st->bnorm2 was set before.  Converged-at-start and rho_0 = 0 are
// flagged for the host.
__global__ void k_init_state(IterState* st, int k, double tol, int max_itn) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = 0; j < k; ++j) {
    st->cr[j] = st->red[j];
    st->xc[j] = 0.0;
  }
  st->k = k;
  st->rho = st->red[k];
  st->rnorm2 = st->red[k + 1];
  st->rmax2 = st->rnorm2;
  st->thresh2 = tol * tol * st->bnorm2;
  st->alpha = st->omega = st->beta = 0.0;
  st->iter = 0;
  st->half = 0;
  st->max_itn = max_itn;
  st->status = RB_OK;
  st->done = 0;
  if (!isfinite(st->rnorm2) || !isfinite(st->rho)) {
    st->status = RB_ENONFINITE;
    st->done = 1;
  } else if (st->rnorm2 <= st->thresh2) {
    st->done = 1;
  } else if (st->rho == 0.0) {
    st->status = RB_EBREAKDOWN_RHO;
    st->done = 1;
  }
}

cudaError_t init_state(IterState* st, int k, double tol, int max_itn, cudaStream_t s) {
  count_launches(1);
  k_init_state<<<1, 32, 0, s>>>(st, k, tol, max_itn);
  return cudaGetLastError();
}

}  // namespace rb
