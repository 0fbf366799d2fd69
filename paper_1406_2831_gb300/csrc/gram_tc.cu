// Gram matrices of the recycle update on the tensor cores (tcgen05, sm_103a).
//
// After every cycle of s iterations the harmonic-Ritz update (Sec. 6.2
// cycles; the harmonic-Ritz reading of the update) needs G = Z^T Z and
// H = Z^T W for the FP32 column blocks W = [Y, P, S] and Z = [AY, AP, AS]
// (n x m each, m <= k + 2s).  This is the one dense contraction of the path:
// m ~ 70 against n ~ 2e6 makes it tall and skinny, and on CUDA cores it held
// every SM for ~1.6 ms per cycle.
//
// Stacked operand.  A 32-row tile of all source columns is laid out in
// shared memory as rows of 128 bytes (one source column's 32 values per
// row): Z's blocks first (rows [0, zrows)), then W's, every block padded to
// a multiple of 8 rows, the whole tile to R >= 128 rows.  With A = rows
// [0, 128) and B = rows [0, R), one MMA of shape M = 128, N = R, K = 8 forms
// every Z-column x (Z or W)-column product of 8 rows; rows beyond the data
// give entries nobody reads.
//
// Precision.  Each FP32 value x is split into a TF32 pair, hi = rn_tf32(x)
// and lo = rn_tf32(x - hi); hi hi' + hi lo' + lo hi' differs from x x' by at
// most ~3 * 2^-22 |x x'| (the TF32 products themselves are exact in FP32).
// The tensor core accumulates in FP32 over a chunk of 4 tiles (128 rows,
// 48 accumulating MMAs per entry): measured, its accumulation is biased like
// truncation (errors grow linearly with the chunk length), so chunks are
// kept short; chunk sums are added in FP32 registers (round to nearest) and
// CTA sums in FP64.
//
// Roles in one persistent CTA per SM (14 warps):
//   warp 0    one lane: TMA loads (one 2D tensor map per source block,
//             128-byte swizzle, zero fill beyond the columns / rows) into a
//             ring of NST stages;
//   warp 1    TMEM allocation; one lane issues the MMAs (kind::tf32) into
//             one of two accumulator buffers, alternating per chunk;
//   warps 2-5 split each landed tile into hi (in place) and lo;
//   warps 6-13 drain a finished accumulator buffer with tcgen05.ld and add
//             it to registers (one D row and half its columns per thread).
// Each CTA writes its FP32 sums once; k_gram_tc_reduce adds the CTA partials
// in FP64 in CTA order and scatters G and H (deterministic).
//
// Every mbarrier wait is bounded (kWaitCycles of the SM clock, about one
// second): on expiry the CTA raises a shared abort flag, every role leaves
// its loop, the producer and the MMA issuer wait (bounded) for their own
// copies and MMAs, the TMEM is freed, and the error word tells the host,
// which reports RB_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "mbar.cuh"

namespace rb {
namespace {

constexpr int kTcThreads = 448;              // 14 warps
constexpr int kSplitWarp0 = 2, kEpiWarp0 = 6;
constexpr int kChunkTiles = 4;               // tiles (32 rows) per accumulator buffer
constexpr int kTmemCols = 512;               // two accumulator buffers of up to 256 columns

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A B^T, A and B K-major in shared memory (descriptors), FP32 D.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The mbarrier receives one arrival once every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  // the registers are valid only after wait::ld; they are passed through it
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])::"memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: rows of 128 bytes, groups of 8 rows 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (16 B; unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::tf32, FP32 accumulator, both operands
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4)                           // D format F32
         | (2u << 7) | (2u << 10)            // A, B format TF32
         | ((uint32_t)(N >> 3) << 17)        // N / 8
         | ((uint32_t)(M >> 4) << 24);       // M / 16
}

__device__ __forceinline__ uint32_t tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Launch parameters of one stacked Gram.  Blocks in order AY, AP, AS (Z),
// Y, P, S (W).
struct GramTcParams {
  int n_tiles;        // ceil(n / 32)
  int n_chunks;       // ceil(n_tiles / kChunkTiles)
  int R;              // rows of the stacked tile: multiple of 16, 128..224
  int zrows;          // rows of Z's blocks (<= 112)
  int nst;            // pipeline stages
  uint32_t tx_bytes;  // bytes the loads of one tile deliver
  int off[6];         // first tile row of each block
  int active[6];      // block has at least one column
};

// Output positions: Z column a sits in tile row z[a], W column b in w[b].
struct GramTcPos {
  int z[kMaxGramTc];
  int w[kMaxGramTc];
};

template <int CPT>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
              const __grid_constant__ CUtensorMap m2, const __grid_constant__ CUtensorMap m3,
              const __grid_constant__ CUtensorMap m4, const __grid_constant__ CUtensorMap m5,
              const GramTcParams p, float* __restrict__ work, int* __restrict__ err) {
  extern __shared__ unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[4], bar_split[4], bar_empty[4], bar_accf[2], bar_acce[2], bar_fin;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(base);
  const uint32_t stage_bytes = 2u * (uint32_t)p.R * 128u;
  volatile int* abort = &s_abort;

  if (threadIdx.x == 0) {
    for (int st = 0; st < p.nst; ++st) {
      mbar_init(smem_u32(&bar_full[st]), 1);
      mbar_init(smem_u32(&bar_split[st]), 4);
      mbar_init(smem_u32(&bar_empty[st]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_accf[b]), 1);
      mbar_init(smem_u32(&bar_acce[b]), 8);
    }
    mbar_init(smem_u32(&bar_fin), 1);
    s_abort = 0;
    fence_barrier_init();
  }
  {  // rows no load writes (blocks without columns, padding up to R) stay zero
    float4* z4 = reinterpret_cast<float4*>(base);
    const int n4 = (int)((uint32_t)p.nst * stage_bytes / 16u);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    fence_proxy_async();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(&s_tmem), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_tmem;

  if (warp == 0) {
    // ---- producer: TMA loads of every tile into the ring
    if (lane == 0) {
      const CUtensorMap* maps[6] = {&m0, &m1, &m2, &m3, &m4, &m5};
      int it = 0;
      bool ok = true;
      for (int c = blockIdx.x; ok && c < p.n_chunks; c += gridDim.x) {
        const int t1 = min((c + 1) * kChunkTiles, p.n_tiles);
        for (int t = c * kChunkTiles; t < t1; ++t, ++it) {
          const int st = it % p.nst, use = it / p.nst;
          if (use > 0 && !mbar_wait(smem_u32(&bar_empty[st]), (use - 1) & 1, abort)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&bar_full[st]);
          mbar_expect_tx(fb, p.tx_bytes);
          const uint32_t dst = sbase + (uint32_t)st * stage_bytes;
          for (int b = 0; b < 6; ++b)
            if (p.active[b]) tma_load_2d(dst + (uint32_t)p.off[b] * 128u, maps[b], t * 32, 0, fb);
        }
      }
      // copies of the last tiles may still be landing (after an abort): wait for them
      for (int j = max(0, it - p.nst); j < it; ++j) mbar_wait(smem_u32(&bar_full[j % p.nst]), (j / p.nst) & 1, nullptr);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tf32_idesc(128, p.R);
      int it = 0, cj = 0;
      bool ok = true;
      for (int c = blockIdx.x; ok && c < p.n_chunks; c += gridDim.x, ++cj) {
        const int buf = cj & 1;
        if (cj >= 2 && !mbar_wait(smem_u32(&bar_acce[buf]), ((cj >> 1) - 1) & 1, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tbase + (uint32_t)buf * 256u;
        const int t0 = c * kChunkTiles, t1 = min(t0 + kChunkTiles, p.n_tiles);
        for (int t = t0; t < t1; ++t, ++it) {
          const int st = it % p.nst, use = it / p.nst;
          if (!mbar_wait(smem_u32(&bar_split[st]), use & 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t h = sbase + (uint32_t)st * stage_bytes, l = h + (uint32_t)p.R * 128u;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t dh = sw128_desc(h + kk * 32), dl = sw128_desc(l + kk * 32);
            mma_tf32(d, dh, dh, idesc, (t > t0 || kk > 0) ? 1u : 0u);
            mma_tf32(d, dh, dl, idesc, 1u);
            mma_tf32(d, dl, dh, idesc, 1u);
          }
          mma_commit(smem_u32(&bar_empty[st]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&bar_accf[buf]));
      }
      mma_commit(smem_u32(&bar_fin));   // every MMA issued here has completed
      mbar_wait(smem_u32(&bar_fin), 0, nullptr);
    }
    __syncwarp();
  } else if (warp < kEpiWarp0) {
    // ---- split: x -> (hi, lo) TF32 pair, hi in place
    const int tid = threadIdx.x - kSplitWarp0 * 32;
    int it = 0;
    bool ok = true;
    for (int c = blockIdx.x; ok && c < p.n_chunks; c += gridDim.x) {
      const int t1 = min((c + 1) * kChunkTiles, p.n_tiles);
      for (int t = c * kChunkTiles; t < t1; ++t, ++it) {
        const int st = it % p.nst, use = it / p.nst;
        const bool got = mbar_wait(smem_u32(&bar_full[st]), use & 1, abort);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        uint4* hi = reinterpret_cast<uint4*>(base + (size_t)st * stage_bytes);
        uint4* lo = reinterpret_cast<uint4*>(base + (size_t)st * stage_bytes + (size_t)p.R * 128);
        const int n4 = p.R * 8;
        for (int i = tid; i < n4; i += 128) {
          const uint4 x = hi[i];
          uint4 a, b;
          a.x = tf32_rn(__uint_as_float(x.x));
          a.y = tf32_rn(__uint_as_float(x.y));
          a.z = tf32_rn(__uint_as_float(x.z));
          a.w = tf32_rn(__uint_as_float(x.w));
          b.x = tf32_rn(__uint_as_float(x.x) - __uint_as_float(a.x));
          b.y = tf32_rn(__uint_as_float(x.y) - __uint_as_float(a.y));
          b.z = tf32_rn(__uint_as_float(x.z) - __uint_as_float(a.z));
          b.w = tf32_rn(__uint_as_float(x.w) - __uint_as_float(a.w));
          hi[i] = a;
          lo[i] = b;
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_split[st]));
      }
    }
  } else {
    // ---- epilogue: drain finished accumulator buffers into registers
    const int e = warp - kEpiWarp0;   // 0..7
    const int q = warp & 3;           // TMEM lanes 32q..32q+31 are this warp's
    const int half = e >> 2;
    const int row = q * 32 + lane;
    float acc[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) acc[i] = 0.f;
    int cj = 0;
    for (int c = blockIdx.x; c < p.n_chunks; c += gridDim.x, ++cj) {
      const int buf = cj & 1;
      const bool got = mbar_wait(smem_u32(&bar_accf[buf]), (cj >> 1) & 1, abort);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const uint32_t ta = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * 256u + (uint32_t)(half * CPT);
#pragma unroll
      for (int g = 0; g < CPT / 16; ++g) {
        float v[16];
        tmem_ld16(ta + g * 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[g * 16 + i] += v[i];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce[buf]));
    }
    if (row < p.zrows) {
      float* out = work + ((size_t)blockIdx.x * p.zrows + row) * p.R;
#pragma unroll
      for (int i = 0; i < CPT; ++i) {
        const int col = half * CPT + i;
        if (col < p.R) out[col] = acc[i];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, kTmemCols);
  }
  if (threadIdx.x == 0 && s_abort) atomicOr(err, 1);
}

// G(a, b) = G(b, a) from the tile entry (min, max) so that G is exactly
// symmetric; H(a, b) = D(z[a], w[b]).  CTA partials summed in FP64 in CTA
// order.
__global__ void k_gram_tc_reduce(const float* __restrict__ work, int nblk, int zrows, int R, int m,
                                 const GramTcPos pos, double* __restrict__ G, double* __restrict__ H) {
  // entries of one output row a (b fastest) are consecutive tile columns
  // for most b, so a warp's reads of one CTA partial coalesce; the loads of
  // 8 CTAs are issued before their (in-order) additions
  const int tot = 2 * m * m;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < tot; o += gridDim.x * blockDim.x) {
    const int a = o / (2 * m), b = o % (2 * m);
    int pr, pc;
    if (b < m) {
      if (b < a) continue;   // upper triangle only, mirrored below
      pr = pos.z[a];
      pc = pos.z[b];
    } else {
      pr = pos.z[a];
      pc = pos.w[b - m];
    }
    double sum = 0.0;
    const size_t stride = (size_t)zrows * R;
    const float* w = work + (size_t)pr * R + pc;
    int c = 0;
    for (; c + 8 <= nblk; c += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldg(w + (size_t)(c + u) * stride);
#pragma unroll
      for (int u = 0; u < 8; ++u) sum += (double)v[u];
    }
    for (; c < nblk; ++c) sum += (double)__ldg(w + (size_t)c * stride);
    if (b < m) {
      G[a + (size_t)b * m] = sum;
      G[b + (size_t)a * m] = sum;
    } else {
      H[a + (size_t)(b - m) * m] = sum;
    }
  }
}

}  // namespace
}  // namespace rb

namespace rb {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      ptr = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }();
  return fn;
}

// Tile rows of a block of `cap` columns.
int r8(int cap) { return (cap + 7) / 8 * 8; }

struct TcLayout {
  int zrows, R, off[6];
};

TcLayout tc_layout(const int cap[6]) {
  TcLayout L;
  L.zrows = r8(cap[0]) + r8(cap[1]) + r8(cap[2]);
  L.off[0] = 0;
  L.off[1] = r8(cap[0]);
  L.off[2] = r8(cap[0]) + r8(cap[1]);
  for (int b = 0; b < 3; ++b) L.off[3 + b] = L.zrows + L.off[b];
  L.R = std::max(128, (2 * L.zrows + 15) / 16 * 16);
  return L;
}

template <int CPT>
cudaError_t launch_tc(const CUtensorMap* maps, const GramTcParams& p, float* work, int* err, int grid,
                      size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc<CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_tc<CPT><<<grid, kTcThreads, smem, s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], p, work, err);
  return cudaGetLastError();
}

}  // namespace

bool gram_tc_eligible(const int cap[6]) {
  for (int b = 0; b < 3; ++b)
    if (cap[b] != cap[3 + b] || cap[b] < 0) return false;
  const TcLayout L = tc_layout(cap);
  return L.zrows > 0 && L.zrows <= 112 && L.R <= 224 && encode_tiled() != nullptr;
}

size_t gram_tc_work_floats(const int cap[6], int grid) {
  const TcLayout L = tc_layout(cap);
  return (size_t)grid * L.zrows * L.R;
}

int gram_tc(const GramTcBlocks& blk, int64_t n, int64_t ld, double* G, double* H, float* work, int* err,
            int grid, cudaStream_t s) {
  if (!gram_tc_eligible(blk.cap) || n <= 0 || ld < n || (ld * 4) % 16 != 0) return RB_EINVAL;
  for (int b = 0; b < 6; ++b)
    if (blk.cols[b] < 0 || blk.cols[b] > blk.cap[b] || (blk.cols[b] > 0 && ((uintptr_t)blk.ptr[b] & 15))) return RB_EINVAL;
  for (int b = 0; b < 3; ++b)
    if (blk.cols[b] != blk.cols[3 + b]) return RB_EINVAL;
  const int m = blk.cols[0] + blk.cols[1] + blk.cols[2];
  if (m <= 0 || m > kMaxGramTc) return RB_EINVAL;
  const TcLayout L = tc_layout(blk.cap);
  GramTcParams p;
  p.n_tiles = (int)((n + 31) / 32);
  p.n_chunks = (p.n_tiles + kChunkTiles - 1) / kChunkTiles;
  p.R = L.R;
  p.zrows = L.zrows;
  const size_t stage_bytes = (size_t)2 * L.R * 128;
  p.nst = (int)std::min<size_t>(4, (227 * 1024 - 2048) / stage_bytes);
  if (p.nst < 2) return RB_EINVAL;
  p.tx_bytes = 0;
  CUtensorMap maps[6];
  auto enc = encode_tiled();
  for (int b = 0; b < 6; ++b) {
    p.off[b] = L.off[b];
    p.active[b] = blk.cols[b] > 0;
    std::memset(&maps[b], 0, sizeof(CUtensorMap));
    if (!p.active[b]) continue;
    p.tx_bytes += (uint32_t)r8(blk.cap[b]) * 128u;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)blk.cols[b]};
    cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    cuuint32_t box[2] = {32u, (cuuint32_t)r8(blk.cap[b])};
    cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = enc(&maps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)blk.ptr[b], dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return RB_ECUDA;
  }
  GramTcPos pos;
  for (int a = 0; a < kMaxGramTc; ++a) pos.z[a] = pos.w[a] = 0;
  {
    int a = 0;
    for (int b = 0; b < 3; ++b)
      for (int j = 0; j < blk.cols[b]; ++j, ++a) {
        pos.z[a] = L.off[b] + j;
        pos.w[a] = L.off[3 + b] + j;
      }
  }
  grid = std::max(1, std::min(grid, p.n_chunks));
  const size_t smem = (size_t)p.nst * stage_bytes + 1024;
  const int half = L.R / 2, cpt = (half + 15) / 16 * 16;
  cudaError_t e;
  count_launches(2);
  switch (cpt) {
    case 64: e = launch_tc<64>(maps, p, work, err, grid, smem, s); break;
    case 80: e = launch_tc<80>(maps, p, work, err, grid, smem, s); break;
    case 96: e = launch_tc<96>(maps, p, work, err, grid, smem, s); break;
    case 112: e = launch_tc<112>(maps, p, work, err, grid, smem, s); break;
    default: return RB_EINVAL;
  }
  if (e != cudaSuccess) return RB_ECUDA;
  const int tot = 2 * m * m;
  k_gram_tc_reduce<<<(tot + 255) / 256, 256, 0, s>>>(work, grid, L.zrows, L.R, m, pos, G, H);
  if (cudaGetLastError() != cudaSuccess) return RB_ECUDA;
  return RB_OK;
}

}  // namespace rb
