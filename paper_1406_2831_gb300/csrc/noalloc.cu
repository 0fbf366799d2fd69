// rbicgstab_residual_noalloc: r = b - A x and ||r||^2 from caller-owned
// device CSR arrays, without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// residual: code running under a framework that owns the device allocator and
// forbids raw cudaMalloc, code about to be captured into a CUDA graph, or a
// service that pre-sizes all device memory at start-up and must not grow it.
// This entry point serves them.  The caller passes every input and output;
// the only scratch this kernel needs (one partial sum per block and per
// group of 16 blocks, and the completion tickets of the grid reduction)
// lives in a fixed file-scope device array of about 9 KB, which every GPU
// that loads the library keeps until the process exits.
#include <mutex>

#include "device.cuh"
#include "kernels.h"

namespace {

constexpr int kNaMaxBlocks = 1024;   // block partials the scratch array holds

struct NaScratch {
  double partials[kNaMaxBlocks + kNaMaxBlocks / 16 + 1];   // block rows + group rows
  rb::GridTicket ticket;
};

// File-scope scratch.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) NaScratch g_na_scratch;

constexpr int kNaMaxDevices = 128;
NaScratch* g_na_addr[kNaMaxDevices] = {};
std::mutex g_na_mutex;

// Device address of the scratch on the current device, looked up once per
// device (this first lookup can load the module, so the first call on a
// device should not be made while a stream is being captured).
int na_scratch(NaScratch** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return RB_ECUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return RB_ECUDA;
    g_na_addr[dev] = (NaScratch*)p;
  }
  *out = g_na_addr[dev];
  return RB_OK;
}

__global__ void __launch_bounds__(rb::kBlock) k_residual_csr_na(
    int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
    const double* __restrict__ val, const double* __restrict__ x, const double* __restrict__ b,
    double* __restrict__ r, double* __restrict__ rnorm2, NaScratch* sc) {
  __shared__ rb::ReduceSmem<1> sm;
  double acc[1] = {0.0};
  for (int64_t i = rb::gtid(); i < n; i += rb::gstride()) {
    double y = 0.0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) y = fma(val[e], x[col[e]], y);
    const double rv = b[i] - y;
    r[i] = rv;
    acc[0] = fma(rv, rv, acc[0]);
  }
  if (rb::block_reduce_last<1>(acc, 1, sm, sc->partials, &sc->ticket) && threadIdx.x == 0)
    *rnorm2 = sm.res[0];
}

}  // namespace

extern "C" int rbicgstab_residual_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col,
                                          const double* val, const double* x, const double* b,
                                          double* r, double* rnorm2, void* cuda_stream) {
  if (n <= 0 || n > 2147483647LL) return RB_EINVAL;
  if (!row_ptr || !col || !val || !x || !b || !r || !rnorm2) return RB_EINVAL;
  NaScratch* sc = nullptr;
  int rc = na_scratch(&sc);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the completion tickets must start at zero; a memset allocates nothing
  RB_CUDA_TRY(cudaMemsetAsync(&sc->ticket, 0, sizeof(rb::GridTicket), s));
  const int64_t want = (n + rb::kBlock - 1) / rb::kBlock;
  const int grid = (int)(want < kNaMaxBlocks ? want : kNaMaxBlocks);
  rb::count_launches(1);
  k_residual_csr_na<<<grid, rb::kBlock, 0, s>>>(n, row_ptr, col, val, x, b, r, rnorm2, sc);
  RB_CUDA_TRY(cudaGetLastError());
  return RB_OK;
}
