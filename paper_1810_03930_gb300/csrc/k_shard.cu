// Row-sharded iteration (Section 5.4's parallel structure: every O(np) and O(np^2) kernel
// runs on a rank's own rows; the ranks exchange only the reduced Grams [B | C] and the
// per-column dots).  The exchange is an all-gather whose result every rank adds up in rank
// order with the kernel below, so that every rank holds bit-identical sums and takes the
// same step-size and stop decisions without a broadcast.
#include "plam_common.cuh"

namespace plam {

__global__ void rank_sum_kernel(const double* __restrict__ in, int size, int64_t count,
                                double* __restrict__ out, const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    double v = in[i];
    for (int r = 1; r < size; ++r) v += in[(int64_t)r * count + i];
    out[i] = v;
  }
}

cudaError_t launch_rank_sum(const double* in, int size, int64_t count, double* out,
                            const DevState* st, cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  rank_sum_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, size, count, out, st);
  return cudaGetLastError();
}

}  // namespace plam
