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
// names a host-side stand-in), so the first call in each CUDA context, with
// that context current, looks the address up with cudaGetSymbolAddress and
// caches it under the context; that first call should therefore come before any
// stream capture.  The cache is keyed on the context's unique id (not the
// device ordinal), so it stays valid across cudaDeviceReset and explicitly
// created contexts, which load the module again at a new address.
// No entry of the scratch has to start at zero: every partial that the
// reduction reads is written earlier in the same call.  All calls share the
// one array, so calls whose kernels overlap on the GPU (different streams,
// different host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "../../include/plam.h"
#include "plam_common.cuh"

namespace {

constexpr size_t kGramScratchBytes = size_t(8) << 20;
constexpr int kCacheSlots = 64;

__device__ __align__(256) unsigned char g_gram_scratch[kGramScratchBytes];

typedef int (*CtxGetCurrentFn)(void**);                    // cuCtxGetCurrent
typedef int (*CtxGetIdFn)(void*, unsigned long long*);       // cuCtxGetId

std::mutex g_scratch_mu;
struct ScratchSlot {
  unsigned long long ctx_id;   // 0: empty
  void* addr;
};
ScratchSlot g_scratch_cache[kCacheSlots] = {};
int g_scratch_next = 0;

void* driver_fn(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return p;
}

// The unique id of the current CUDA context (ids are never reused within a process, unlike
// context handles); 0 when no context is current.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get = (CtxGetCurrentFn)driver_fn("cuCtxGetCurrent");
  static CtxGetIdFn get_id = (CtxGetIdFn)driver_fn("cuCtxGetId");
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get || !get_id || get(&ctx) != 0 || ctx == nullptr || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_gram_scratch in the current context, looked up with
// cudaGetSymbolAddress once per context (the lookup also makes the runtime's
// context current when none is yet).
plam_status_t scratch_address(void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  unsigned long long id = current_context_id();
  if (id != 0)
    for (int i = 0; i < kCacheSlots; ++i)
      if (g_scratch_cache[i].ctx_id == id) {
        *out = g_scratch_cache[i].addr;
        return PLAM_OK;
      }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_gram_scratch);
  if (e != cudaSuccess || ptr == nullptr) {
    plam::set_last_error("plam_grams_noalloc: cudaGetSymbolAddress", cudaGetErrorString(e));
    return PLAM_ERR_CUDA;
  }
  if (id == 0) id = current_context_id();
  if (id != 0) {
    g_scratch_cache[g_scratch_next] = ScratchSlot{id, ptr};
    g_scratch_next = (g_scratch_next + 1) % kCacheSlots;
  }
  *out = ptr;
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
  // the chunking rule of a handle (plam_create), capped by the scratch
  const plam::GramChunkPlan pl = plam::gram_chunk_plan(n, p, G != nullptr, plam::device_sm_count(),
                                                       max_chunks);
  const int64_t rows = pl.rows_per_chunk;
  const int nchunks = pl.nchunks;
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

plam_status_t invalid(const char* why) {
  plam::set_last_error("plam_grams_noalloc", why);
  return PLAM_ERR_INVALID;
}

}  // namespace

extern "C" plam_status_t plam_grams_noalloc(int64_t n, int64_t p, int precision, const void* X,
                                            int64_t ldx, const void* G, int64_t ldg, double* B,
                                            double* C, void* stream) {
  if (n < 1 || p < 1 || p > 65535) return invalid("n and p must be positive (p <= 65535)");
  if (!X || !B || (G && !C)) return invalid("null X, B, or C with G given");
  if (ldx < n || (G && ldg < n)) return invalid("leading dimension below n");
  if (precision != PLAM_PREC_FP64 && precision != PLAM_PREC_FP32) return invalid("bad precision");
  const size_t esz = precision == PLAM_PREC_FP64 ? 8 : 4;
  if (!aligned_to(X, esz) || (G && !aligned_to(G, esz)) || !aligned_to(B, 8) ||
      (C && !aligned_to(C, 8)))
    return invalid("pointer not aligned to its element size");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == PLAM_PREC_FP64)
    return grams_noalloc<double>(n, (int)p, (const double*)X, ldx, (const double*)G, ldg, B, C, s);
  return grams_noalloc<float>(n, (int)p, (const float*)X, ldx, (const float*)G, ldg, B, C, s);
}
