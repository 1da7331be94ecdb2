// Final orthonormalisation (Section 5.3, Table "orth step"; the parallel code
// of Section 5.4 uses Eigen's LLT): with B = X^T X (double),
//     B = R^T R  (Cholesky, R upper triangular, diag(R) > 0),
//     Q = X R^{-1}.
//
// cholesky_inverse_kernel (one CTA, double): right-looking Cholesky of the
// upper triangle of B in a p x p work matrix, then the columns of Z = R^{-1}
// by back substitution (one thread per column); for p <= 96 the same steps run
// in shared memory (cholesky_inverse_smem_kernel).  A pivot that is not positive
// and finite stops the factorisation and reports 1 + its index in *info.
// apply_rinv_kernel: Q = X Z over 64 x 64 output tiles, double arithmetic
// (float inputs are converted exactly), Z upper triangular so column c only
// needs rows k <= c.
#include "plam_device.cuh"

namespace plam {

__global__ void __launch_bounds__(1024)
cholesky_inverse_kernel(int p, const double* __restrict__ B, double* __restrict__ W,
                        double* __restrict__ Z, int* __restrict__ info) {
  __shared__ int fail;
  __shared__ double piv;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < p * p; e += nt) W[e] = B[e];
  if (t == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    if (t == 0) {
      const double d = W[j + (size_t)j * p];
      if (!(d > 0.0) || !isfinite(d)) {
        fail = j + 1;
        piv = 1.0;
      } else {
        piv = sqrt(d);
        W[j + (size_t)j * p] = piv;
      }
    }
    __syncthreads();
    if (fail) break;
    const double inv = 1.0 / piv;
    for (int k = j + 1 + t; k < p; k += nt) W[j + (size_t)k * p] *= inv;   // row j of R
    __syncthreads();
    // trailing update of the upper triangle: W[i,k] -= R[j,i] R[j,k], j < i <= k
    const int m = p - j - 1;
    const long long tri = (long long)m * (m + 1) / 2;
    for (long long e = t; e < tri; e += nt) {
      // decode e -> (a, b) with 0 <= a <= b < m, column-major over b
      int b = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
      while ((long long)b * (b + 1) / 2 > e) --b;
      while ((long long)(b + 1) * (b + 2) / 2 <= e) ++b;
      const int a = (int)(e - (long long)b * (b + 1) / 2);
      const int i = j + 1 + a, k = j + 1 + b;
      W[i + (size_t)k * p] -= W[j + (size_t)i * p] * W[j + (size_t)k * p];
    }
    __syncthreads();
  }
  if (t == 0) *info = fail;
  if (fail) return;
  // Z = R^{-1}: column c solves R z = e_c for z_i, i <= c
  for (int c = t; c < p; c += nt) {
    for (int i = p - 1; i > c; --i) Z[i + (size_t)c * p] = 0.0;
    for (int i = c; i >= 0; --i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) s -= W[i + (size_t)k * p] * Z[k + (size_t)c * p];
      Z[i + (size_t)c * p] = s / W[i + (size_t)i * p];
    }
  }
}

// The same factorisation and inverse for p <= kCholSmemMaxP with R and Z in
// shared memory: the trailing update indexes (a, b) of the remaining square
// directly (no square root per element), the pivot reciprocals are formed once,
// and the column-wise back substitution reads shared memory instead of L2.
constexpr int kCholSmemMaxP = 96;   // 2 p^2 doubles <= 144 KB

__global__ void __launch_bounds__(1024)
cholesky_inverse_smem_kernel(int p, const double* __restrict__ B, double* __restrict__ W,
                             double* __restrict__ Z, int* __restrict__ info) {
  extern __shared__ double csm[];
  double* Ws = csm;              // p x p, column-major: the upper triangle becomes R
  double* Zs = csm + p * p;      // p x p, Z = R^{-1}
  __shared__ int fail;
  __shared__ double rpiv[kCholSmemMaxP];
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < p * p; e += nt) Ws[e] = B[e];
  if (t == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    if (t == 0) {
      const double d = Ws[j + j * p];
      if (!(d > 0.0) || !isfinite(d)) {
        fail = j + 1;
        rpiv[j] = 1.0;
      } else {
        const double piv = sqrt(d);
        Ws[j + j * p] = piv;
        rpiv[j] = 1.0 / piv;
      }
    }
    __syncthreads();
    if (fail) break;
    const double inv = rpiv[j];
    for (int k = j + 1 + t; k < p; k += nt) Ws[j + k * p] *= inv;   // row j of R
    __syncthreads();
    // trailing update of the upper triangle: W[i,k] -= R[j,i] R[j,k], j < i <= k
    const int m = p - j - 1;
    for (int e = t; e < m * m; e += nt) {
      const int a = e % m, b = e / m;
      if (a <= b) {
        const int i = j + 1 + a, k = j + 1 + b;
        Ws[i + k * p] -= Ws[j + i * p] * Ws[j + k * p];
      }
    }
    __syncthreads();
  }
  if (t == 0) *info = fail;
  if (fail) return;
  // Z = R^{-1}: column c solves R z = e_c for z_i, i <= c
  for (int c = t; c < p; c += nt) {
    for (int i = p - 1; i > c; --i) Zs[i + c * p] = 0.0;
    for (int i = c; i >= 0; --i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) s -= Ws[i + k * p] * Zs[k + c * p];
      Zs[i + c * p] = s * rpiv[i];
    }
  }
  __syncthreads();
  for (int e = t; e < p * p; e += nt) {
    W[e] = Ws[e];
    Z[e] = Zs[e];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
apply_rinv_kernel(int64_t n, int p, const T* __restrict__ X, int64_t ldx, const double* __restrict__ Z,
                  double* __restrict__ Q, int64_t ldq) {
  constexpr int KS = 16;
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int c0 = blockIdx.y * kTile;
  __shared__ double Xs[KS][kTile];
  __shared__ double Zs[kTile][KS + 1];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  const int kend = min(p, c0 + kTile);
  for (int k0 = 0; k0 < kend; k0 += KS) {
    {
      const int r = t & (kTile - 1);
      const int64_t row = r0 + r;
#pragma unroll
      for (int s = 0; s < KS / 4; ++s) {
        const int q = (t >> 6) + 4 * s;
        const int col = k0 + q;
        Xs[q][r] = (row < n && col < p) ? (double)X[row + (int64_t)col * ldx] : 0.0;
      }
    }
    {
      const int q = t & (KS - 1);
      const int kr = k0 + q;
#pragma unroll
      for (int s = 0; s < kTile * KS / kThreads; ++s) {
        const int c = t / KS + (kThreads / KS) * s;
        const int cc = c0 + c;
        Zs[c][q] = (kr < p && cc < p && kr <= cc) ? Z[kr + (size_t)cc * p] : 0.0;
      }
    }
    __syncthreads();
    // column group v (columns c0 + 16 v .. + 15) gets nothing from rows k0.. of Z
    // when all its columns lie left of k0 (Z is upper triangular): skip it
    // (the same for every thread, and the skipped products are exact zeros)
    bool live[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) live[v] = c0 + 16 * v + 15 >= k0;
#pragma unroll 4
    for (int q = 0; q < KS; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Xs[q][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = live[v] ? Zs[ty + 16 * v][q] : 0.0;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (!live[v]) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][v] = fma(a[u], b[v], acc[u][v]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int c = c0 + ty + 16 * v;
    if (c >= p) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t r = r0 + tx + 16 * u;
      if (r < n) Q[r + (int64_t)c * ldq] = acc[u][v];
    }
  }
}

__global__ void feas_kernel(int p, const double* __restrict__ B, double* __restrict__ out) {
  __shared__ double scratch[33];
  double s = 0.0;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e % p, j = e / p;
    const double d = B[e] - (i == j ? 1.0 : 0.0);
    s += d * d;
  }
  const double tot = block_sum(s, scratch);
  if (threadIdx.x == 0) out[0] = sqrt(tot);
}

cudaError_t launch_cholesky_inverse(int p, const double* B, double* W, double* Z, int* info,
                                    cudaStream_t s) {
  if (p <= kCholSmemMaxP) {
    const size_t smem = (size_t)2 * p * p * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(cholesky_inverse_smem_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cholesky_inverse_smem_kernel<<<1, 1024, smem, s>>>(p, B, W, Z, info);
    return cudaGetLastError();
  }
  cholesky_inverse_kernel<<<1, 1024, 0, s>>>(p, B, W, Z, info);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_rinv(int64_t n, int p, const T* X, int64_t ldx, const double* Z, double* Q,
                              int64_t ldq, cudaStream_t s) {
  dim3 grid((unsigned)((n + kTile - 1) / kTile), (p + kTile - 1) / kTile);
  apply_rinv_kernel<T><<<grid, kThreads, 0, s>>>(n, p, X, ldx, Z, Q, ldq);
  return cudaGetLastError();
}

cudaError_t launch_feas(int p, const double* B, double* out, cudaStream_t s) {
  feas_kernel<<<1, 256, 0, s>>>(p, B, out);
  return cudaGetLastError();
}

template cudaError_t launch_apply_rinv<float>(int64_t, int, const float*, int64_t, const double*,
                                              double*, int64_t, cudaStream_t);
template cudaError_t launch_apply_rinv<double>(int64_t, int, const double*, int64_t, const double*,
                                               double*, int64_t, cudaStream_t);

}  // namespace plam
