// MOptQR, the comparison solver of Sections 5.3-5.4 (Table "cost", rows "MOptQR (cholesky
// LL^T)"): the projected gradient D = G - X (G^T X) comes from the update kernel with
// M = C^T (gram_finalize in MOptQR mode), the step size from the step-size kernel with the
// Barzilai-Borwein sums of this file's kernel, and the retraction X <- V L^{-T}, V = X - D/eta,
// V^T V = L L^T, from the Gram, Cholesky and triangular-product kernels of the final
// orthonormalisation.  The kernel below replaces the update's S/Y sums, which assume the
// PLAM/PCAL update (S from the column scales), by sums of the stored S = X - X_prev.
#include "plam_device.cuh"

namespace plam {

template <typename T>
__global__ void __launch_bounds__(256)
mopt_bb_kernel(int64_t n, int p, const T* __restrict__ X, int64_t ldx, const T* __restrict__ Xp,
               int64_t ldxp, const T* __restrict__ R0, const T* __restrict__ R1, int64_t ldr,
               int tile_rows, int tile_cols, int nct, T* __restrict__ totpart,
               const DevState* __restrict__ st) {
  if (st->stop != kRunning) return;
  const int k = st->k;
  const T* R = (k & 1) ? R1 : R0;
  const T* Rp = (k & 1) ? R0 : R1;
  const int64_t r0 = (int64_t)blockIdx.x * tile_rows;
  const int c0 = blockIdx.y * tile_cols;
  const int64_t r1 = min(n, r0 + (int64_t)tile_rows);
  const int c1 = min(p, c0 + tile_cols);
  double ss = 0.0, sy = 0.0, yy = 0.0;
  if (k > 0) {
    T a = T(0), b = T(0), c = T(0);
    const int64_t rows = r1 - r0;
    for (int64_t e = threadIdx.x; e < rows * (c1 - c0); e += blockDim.x) {
      const int64_t rr = r0 + e % rows;
      const int cc = c0 + (int)(e / rows);
      const T s = X[rr + (int64_t)cc * ldx] - Xp[rr + (int64_t)cc * ldxp];
      const T y = R[rr + (int64_t)cc * ldr] - Rp[rr + (int64_t)cc * ldr];
      a = fma(s, s, a);
      b = fma(s, y, b);
      c = fma(y, y, c);
    }
    ss = (double)a;
    sy = (double)b;
    yy = (double)c;
  }
  __shared__ double scratch[33];
  ss = block_sum(ss, scratch);
  sy = block_sum(sy, scratch);
  yy = block_sum(yy, scratch);
  if (threadIdx.x == 0) {
    T* t = totpart + ((size_t)blockIdx.x * nct + blockIdx.y) * kTotDots;
    t[0] = (T)ss;
    t[1] = (T)sy;
    t[2] = (T)yy;
  }
}

template <typename T>
cudaError_t launch_mopt_bb(int64_t n, int p, const T* X, int64_t ldx, const T* Xprev, int64_t ldxp,
                           const T* R0, const T* R1, int64_t ldr, int tile_rows, int tile_cols,
                           int nrt, int nct, T* totpart, const DevState* st, cudaStream_t s) {
  mopt_bb_kernel<T><<<dim3((unsigned)nrt, (unsigned)nct), 256, 0, s>>>(
      n, p, X, ldx, Xprev, ldxp, R0, R1, ldr, tile_rows, tile_cols, nct, totpart, st);
  return cudaGetLastError();
}

template cudaError_t launch_mopt_bb<float>(int64_t, int, const float*, int64_t, const float*,
                                           int64_t, const float*, const float*, int64_t, int, int,
                                           int, int, float*, const DevState*, cudaStream_t);
template cudaError_t launch_mopt_bb<double>(int64_t, int, const double*, int64_t, const double*,
                                            int64_t, const double*, const double*, int64_t, int,
                                            int, int, int, double*, const DevState*, cudaStream_t);

}  // namespace plam
