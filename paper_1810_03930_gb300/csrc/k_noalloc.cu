// plam_grams_noalloc: the tall-skinny Grams B = X^T X and C = X^T G of
// plam_grams for callers that cannot allocate device memory.
//
// Who needs it: code that runs where a cudaMalloc is not allowed or not
// acceptable -- a host application whose device memory is owned by another
// memory manager with a fixed budget (a framework's caching allocator, an
// embedded runtime that forbids allocations after start-up), or a latency-
// critical loop in which cudaMalloc's implicit device-wide synchronisation
// would stall other streams.  Those callers cannot create a plam handle
// (plam_create allocates its workspace), so this entry point takes no handle
// and allocates nothing: the split-K partial sums go to a fixed array in the
// library's own device memory, which the loader reserves on every device that
// loads the library and which stays reserved until the process exits.
//
// Scratch: kGramScratchBytes (8 MiB).  A call needs nchunks x 2p x p elements
// of the storage type; the row-chunk count is reduced to fit, and a request
// whose single chunk (2 p^2 elements) does not fit is rejected with
// PLAM_ERR_INVALID (p <= 1024 in FP32 mode, p <= 724 in FP64 mode).
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches
// it; that first call should therefore come before any stream capture.
// No entry of the scratch has to start at zero: every partial that the
// reduction reads is written earlier in the same call.  All calls share the
// one array, so calls whose kernels overlap on the GPU (different streams,
// different host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "../../include/plam.h"
#include "plam_common.cuh"

namespace {

constexpr size_t kGramScratchBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_gram_scratch[kGramScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_gram_scratch on the current device (looked up once per device).
plam_status_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    plam::set_last_error("plam_grams_noalloc: cudaGetDevice", cudaGetErrorString(e));
    return PLAM_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    plam::set_last_error("plam_grams_noalloc", "device ordinal beyond the supported 64");
    return PLAM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_gram_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      plam::set_last_error("plam_grams_noalloc: cudaGetSymbolAddress", cudaGetErrorString(e));
      return PLAM_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return PLAM_OK;
}

template <typename T>
plam_status_t grams_noalloc(int64_t n, int p, const T* X, int64_t ldx, const T* G, int64_t ldg,
                            double* B, double* C, cudaStream_t s) {
  const size_t per_chunk = (size_t)2 * p * p * sizeof(T);
  const int64_t max_chunks = (int64_t)(kGramScratchBytes / per_chunk);
  if (max_chunks < 1) {
    plam::set_last_error("plam_grams_noalloc",
                         "p too large: one chunk of 2 p^2 partial sums exceeds the 8 MiB scratch");
    return PLAM_ERR_INVALID;
  }
  // the same chunking rule as a handle (about two CTAs per SM), capped by the scratch
  const int nt = (p + plam::kTile - 1) / plam::kTile;
  const int tiles = nt * (nt + 1) / 2 + (G ? nt * nt : 0);
  int64_t nch = (2 * 152 + tiles - 1) / tiles;
  const int64_t by_rows = (n + plam::kKStep - 1) / plam::kKStep;
  if (nch > by_rows) nch = by_rows;
  if (nch > max_chunks) nch = max_chunks;
  if (nch < 1) nch = 1;
  int64_t rows = (n + nch - 1) / nch;
  rows = (rows + plam::kKStep - 1) / plam::kKStep * plam::kKStep;
  const int nchunks = (int)((n + rows - 1) / rows);
  void* scratch = nullptr;
  plam_status_t st = scratch_address(&scratch);
  if (st != PLAM_OK) return st;
  cudaError_t e = plam::launch_gram_partial<T, T>(n, p, X, ldx, G, ldg, rows, nchunks, (T*)scratch,
                                                  nullptr, s);
  if (e == cudaSuccess) e = plam::launch_gram_reduce<T>(p, nchunks, G != nullptr, (const T*)scratch,
                                                       B, C, s);
  if (e != cudaSuccess) {
    plam::set_last_error("plam_grams_noalloc: launch", cudaGetErrorString(e));
    return PLAM_ERR_CUDA;
  }
  return PLAM_OK;
}

bool aligned_to(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

}  // namespace

extern "C" plam_status_t plam_grams_noalloc(int64_t n, int64_t p, int precision, const void* X,
                                            int64_t ldx, const void* G, int64_t ldg, double* B,
                                            double* C, void* stream) {
  if (n < 1 || p < 1 || p > 65535 || !X || !B || ldx < n || (G && (ldg < n || !C)))
    return PLAM_ERR_INVALID;
  if (precision != PLAM_PREC_FP64 && precision != PLAM_PREC_FP32) return PLAM_ERR_INVALID;
  const size_t esz = precision == PLAM_PREC_FP64 ? 8 : 4;
  if (!aligned_to(X, esz) || (G && !aligned_to(G, esz)) || !aligned_to(B, 8) ||
      (C && !aligned_to(C, 8)))
    return PLAM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == PLAM_PREC_FP64)
    return grams_noalloc<double>(n, (int)p, (const double*)X, ldx, (const double*)G, ldg, B, C, s);
  return grams_noalloc<float>(n, (int)p, (const float*)X, ldx, (const float*)G, ldg, B, C, s);
}
