// Final orthonormalisation (Section 5.3, Table "orth step"; the parallel code
// of Section 5.4 uses Eigen's LLT): with B = X^T X (double),
//     B = R^T R  (Cholesky, R upper triangular, diag(R) > 0),
//     Q = X R^{-1}.
//
// For p <= 96 (cholesky_inverse_smem_kernel, one CTA, double): right-looking
// Cholesky of the upper triangle of B in shared memory, then the columns of
// Z = R^{-1} by back substitution (one thread per column).  Larger p: the same
// factorisation blocked on 32 x 32 tiles over many CTAs (see below).  A pivot
// that is not positive and finite stops the factorisation and reports 1 + its
// index in *info.
// apply_rinv_kernel: Q = X Z over 64 x 64 output tiles, double arithmetic
// (float inputs are converted exactly), Z upper triangular so column c only
// needs rows k <= c.
#include <type_traits>

#include "exact_sum.cuh"
#include "plam_device.cuh"

namespace plam {

// ---- blocked factorisation and inverse for p > kCholSmemMaxP, on 32 x 32 blocks
// over many CTAs (one launch per step; an earlier failure, recorded in *info,
// turns the later launches into no-ops).  For block column j (rows j0 .. j1-1):
//   chol_diag_kernel    R_jj = chol(W_jj) and its inverse Z_jj = R_jj^{-1} (the
//                       diagonal block of Z), both in shared memory
//   chol_row_kernel     the row panel R[j, k] = R_jj^{-T} W[j, k] = Z_jj^T W[j, k], k >= j1
//   chol_update_kernel  the trailing upper triangle W[i, k] -= R[j, i]^T R[j, k],
//                       j1 <= i <= k, on upper-triangle tiles
// then Z = R^{-1} from the inverted 32 x 32 diagonal blocks by recursive doubling
// (rinv_pair_t_kernel, rinv_pair_z_kernel, below).  Only the upper triangle of W is read; Z is
// zero below its diagonal on return.

constexpr int kCB = 32;

__global__ void __launch_bounds__(1024)
chol_diag_kernel(int p, int j0, double* __restrict__ W, double* __restrict__ Z,
                 int* __restrict__ info) {
  __shared__ double A[kCB][kCB + 1];    // W_jj, updated in place (upper triangle)
  __shared__ double Rs[kCB][kCB + 1];   // R_jj, row by row
  __shared__ double Zi[kCB][kCB + 1];   // R_jj^{-1}
  __shared__ double rpiv[kCB];          // reciprocals of the pivots
  __shared__ int fail;
  if (*(volatile int*)info != 0) return;
  const int t = threadIdx.x;
  const int r = t & 31, c = t >> 5;
  const int nb = min(kCB, p - j0);
  A[r][c] = (r < nb && c < nb) ? W[(j0 + r) + (size_t)(j0 + c) * p] : 0.0;
  Rs[r][c] = 0.0;
  if (t == 0) fail = 0;
  __syncthreads();
  // right-looking: pivot j, then row j of R and the trailing update from the unscaled row j
  // (R_jk = A_jk / R_jj, A_rc -= R_jr R_jc), two block barriers per step
  for (int j = 0; j < nb; ++j) {
    if (t == 0) {
      const double d = A[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        fail = j0 + j + 1;
      } else {
        const double q = rsqrt(d);
        rpiv[j] = q;
        Rs[j][j] = d * q;
      }
    }
    __syncthreads();
    if (fail) break;
    const double q = rpiv[j];
    if (r == j && c > j && c < nb) Rs[j][c] = A[j][c] * q;
    if (r > j && c >= r && c < nb) A[r][c] -= (A[j][r] * q) * (A[j][c] * q);
    __syncthreads();
  }
  if (fail) {
    if (t == 0) *info = fail;
    return;
  }
  // Z = R_jj^{-1} (R Z = I), right-looking over k = nb-1 .. 0: row k of the running sums A'
  // (the identity minus the rows below, kept in A, whose factorisation is no longer needed)
  // is final at step k, Z_kc = A'_kc / R_kk, and rows r < k subtract R_rk Z_kc.  One block
  // barrier per step; the 32 steps replace a 32-deep serial chain per column.
  A[r][c] = (r == c) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = nb - 1; k >= 0; --k) {
    if (c >= k && c < nb) {
      const double zkc = A[k][c] * rpiv[k];
      if (r < k) A[r][c] -= Rs[r][k] * zkc;
      if (r == k) Zi[k][c] = zkc;
    }
    __syncthreads();
  }
  if (r < nb && c < nb) {
    W[(j0 + r) + (size_t)(j0 + c) * p] = (r <= c) ? Rs[r][c] : 0.0;
    Z[(j0 + r) + (size_t)(j0 + c) * p] = (r <= c) ? Zi[r][c] : 0.0;
  }
}

__global__ void __launch_bounds__(256)
chol_row_kernel(int p, int j0, double* __restrict__ W, const double* __restrict__ Z,
                const int* __restrict__ info) {
  __shared__ double Zs[kCB][kCB + 1];
  __shared__ double Ws[kCB][kCB + 1];
  if (*(volatile const int*)info != 0) return;
  const int nb = min(kCB, p - j0), j1 = j0 + nb;
  const int k0 = j1 + (int)blockIdx.x * kCB;
  const int nk = min(kCB, p - k0);
  const int t = threadIdx.x;
  for (int e = t; e < kCB * kCB; e += 256) {
    const int m = e & 31, l = e >> 5;
    Zs[m][l] = (m < nb && l < nb) ? Z[(j0 + m) + (size_t)(j0 + l) * p] : 0.0;
    Ws[m][l] = (m < nb && l < nk) ? W[(j0 + m) + (size_t)(k0 + l) * p] : 0.0;
  }
  __syncthreads();
  for (int e = t; e < kCB * kCB; e += 256) {
    const int l = e & 31, kk = e >> 5;
    if (l < nb && kk < nk) {
      double v = 0.0;
      for (int m = 0; m <= l; ++m) v += Zs[m][l] * Ws[m][kk];
      W[(j0 + l) + (size_t)(k0 + kk) * p] = v;
    }
  }
}

__global__ void __launch_bounds__(256)
chol_update_kernel(int p, int j0, double* __restrict__ W, const int* __restrict__ info) {
  __shared__ double Ri[kCB][kCB + 1];
  __shared__ double Rk[kCB][kCB + 1];
  const int ti = blockIdx.x, tk = blockIdx.y;
  if (ti > tk || *(volatile const int*)info != 0) return;
  const int nb = min(kCB, p - j0), j1 = j0 + nb;
  const int i0 = j1 + ti * kCB, k0 = j1 + tk * kCB;
  const int ni = min(kCB, p - i0), nk = min(kCB, p - k0);
  const int t = threadIdx.x;
  for (int e = t; e < kCB * kCB; e += 256) {
    const int l = e & 31, a = e >> 5;
    Ri[l][a] = (l < nb && a < ni) ? W[(j0 + l) + (size_t)(i0 + a) * p] : 0.0;
    Rk[l][a] = (l < nb && a < nk) ? W[(j0 + l) + (size_t)(k0 + a) * p] : 0.0;
  }
  __syncthreads();
  const int a = t & 31;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int b = (t >> 5) + 8 * v;
    if (a < ni && b < nk && (ti < tk || a <= b)) {
      double acc = 0.0;
      for (int l = 0; l < nb; ++l) acc += Ri[l][a] * Rk[l][b];
      W[(i0 + a) + (size_t)(k0 + b) * p] -= acc;
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

// ---- Z = R^{-1} by recursive doubling (the blocked path, p > kCholSmemMaxP):
// once the diagonal super-blocks of size s are inverted (the 32 x 32 ones by chol_diag_kernel),
// each pair of adjacent super-blocks A = [2qs, (2q+1)s), C = [(2q+1)s, (2q+2)s) gets its
// off-diagonal block from
//     T = R_AC Z_CC,      Z_AC = -Z_AA T,
// and the pairs of one level are independent: log2(p / 32) levels of two batched launches
// instead of p / 32 dependent block rows.  T is kept transposed in the (otherwise unused)
// lower triangle of Z, which a last pass sets back to zero.  32 x 32 output tiles of 256
// threads (4 entries each), FP64, the triangular factors' zero parts skipped.
__device__ __forceinline__ bool rinv_pair(int p, int s, int q, int& a0, int& na, int& c0, int& nc) {
  a0 = 2 * q * s;
  c0 = a0 + s;
  if (c0 >= p) return false;
  na = s;
  nc = min(s, p - c0);
  return true;
}

// T^T (rows C, columns A of Z) = (R_AC Z_CC)^T; grid (tiles of A, tiles of C, pairs).
__global__ void __launch_bounds__(256)
rinv_pair_t_kernel(int p, int s, const double* __restrict__ W, double* __restrict__ Z,
                   const int* __restrict__ info) {
  __shared__ double Rs[kCB][kCB + 1];
  __shared__ double Zs[kCB][kCB + 1];
  if (*(volatile const int*)info != 0) return;
  int a0, na, c0, nc;
  if (!rinv_pair(p, s, (int)blockIdx.z, a0, na, c0, nc)) return;
  const int ti = (int)blockIdx.x * kCB, tj = (int)blockIdx.y * kCB;
  if (ti >= na || tj >= nc) return;
  const int t = threadIdx.x, a = t & 31;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  // k runs over C up to the tile's last column (Z_CC is upper triangular)
  const int kend = min(nc, tj + kCB);
  for (int k0 = 0; k0 < kend; k0 += kCB) {
    __syncthreads();
    for (int e = t; e < kCB * kCB; e += 256) {
      const int x = e & 31, y = e >> 5;
      const int gi = a0 + ti + x, gk = c0 + k0 + y;
      Rs[x][y] = (ti + x < na && k0 + y < nc) ? W[gi + (size_t)gk * p] : 0.0;
      const int lk = k0 + x, lj = tj + y;                       // Z_CC (lk, lj)
      Zs[x][y] = (lk < nc && lj < nc && lk <= lj) ? Z[(c0 + lk) + (size_t)(c0 + lj) * p] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int b = (t >> 5) + 8 * v;
      double sum = acc[v];
#pragma unroll 8
      for (int k = 0; k < kCB; ++k) sum = fma(Rs[a][k], Zs[k][b], sum);
      acc[v] = sum;
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int b = (t >> 5) + 8 * v;
    if (ti + a < na && tj + b < nc)
      Z[(c0 + tj + b) + (size_t)(a0 + ti + a) * p] = acc[v];   // T(i, j) at Z[j, i]
  }
}

// Z_AC = -Z_AA T with T(k, j) read from Z[j, k]; grid (tiles of A, tiles of C, pairs).
__global__ void __launch_bounds__(256)
rinv_pair_z_kernel(int p, int s, double* __restrict__ Z, const int* __restrict__ info) {
  __shared__ double As[kCB][kCB + 1];
  __shared__ double Ts[kCB][kCB + 1];
  if (*(volatile const int*)info != 0) return;
  int a0, na, c0, nc;
  if (!rinv_pair(p, s, (int)blockIdx.z, a0, na, c0, nc)) return;
  const int ti = (int)blockIdx.x * kCB, tj = (int)blockIdx.y * kCB;
  if (ti >= na || tj >= nc) return;
  const int t = threadIdx.x, a = t & 31;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  // k runs over A from the tile's first row (Z_AA is upper triangular)
  for (int k0 = ti; k0 < na; k0 += kCB) {
    __syncthreads();
    for (int e = t; e < kCB * kCB; e += 256) {
      const int x = e & 31, y = e >> 5;
      const int li = ti + x, lk = k0 + y;                       // Z_AA (li, lk)
      As[x][y] = (li < na && lk < na && li <= lk) ? Z[(a0 + li) + (size_t)(a0 + lk) * p] : 0.0;
      const int kk = k0 + x, lj = tj + y;                       // T(kk, lj) = Z[c0 + lj, a0 + kk]
      Ts[x][y] = (kk < na && lj < nc) ? Z[(c0 + lj) + (size_t)(a0 + kk) * p] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int b = (t >> 5) + 8 * v;
      double sum = acc[v];
#pragma unroll 8
      for (int k = 0; k < kCB; ++k) sum = fma(As[a][k], Ts[k][b], sum);
      acc[v] = sum;
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int b = (t >> 5) + 8 * v;
    if (ti + a < na && tj + b < nc) Z[(a0 + ti + a) + (size_t)(c0 + tj + b) * p] = -acc[v];
  }
}

// The strictly lower triangle of Z back to zero (it held the transposed T blocks).
__global__ void zero_lower_kernel(int p, double* __restrict__ Z) {
  const size_t total = (size_t)p * p;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % p), c = (int)(e / p);
    if (r > c) Z[e] = 0.0;
  }
}

template <typename T, typename To>
__global__ void __launch_bounds__(kThreads)
apply_rinv_kernel(int64_t n, int p, const T* __restrict__ X, int64_t ldx, const double* __restrict__ Z,
                  To* __restrict__ Q, int64_t ldq, const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
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
      if (r < n) Q[r + (int64_t)c * ldq] = (To)acc[u][v];
    }
  }
}

// Z = R^{-1} as two float planes z = z_hi + z_lo (z_lo = fl(z - z_hi): the pair carries z to
// about 2^-48), written once into scratch for the FP64-free Q = X Z below.
__global__ void split_z_kernel(int p, const double* __restrict__ Z, float* __restrict__ Zh,
                               float* __restrict__ Zl) {
  const size_t total = (size_t)p * p;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double z = Z[e];
    const float zh = (float)z;
    Zh[e] = zh;
    Zl[e] = (float)(z - (double)zh);
  }
}

// Q = X Z for a float X without FP64 multiplies (GB300 executes FP64 at 1/64 of the FP32 rate):
// x z_hi is formed exactly (TwoProduct: h + r), x z_lo in FP32 (a term 2^-24 smaller), and the
// terms are summed in the three levels of exact_sum.cuh.  Same tiles and triangular skipping as
// apply_rinv_kernel; Z arrives split into float planes (split_z_kernel).
template <typename To>
__global__ void __launch_bounds__(kThreads, 1)
apply_rinv_exact_kernel(int64_t n, int p, const float* __restrict__ X, int64_t ldx,
                        const float* __restrict__ Zhp, const float* __restrict__ Zlp,
                        To* __restrict__ Q, int64_t ldq, const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  constexpr int KS = 16;
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int c0 = blockIdx.y * kTile;
  __shared__ float Xs[KS][kTile];
  __shared__ float Zh[kTile][KS + 1];
  __shared__ float Zl[kTile][KS + 1];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  ExactAcc acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) exact_zero(acc[u][v]);
  const int kend = min(p, c0 + kTile);
  int since = 0, segs = 0;
  for (int k0 = 0; k0 < kend; k0 += KS) {
    {
      const int r = t & (kTile - 1);
      const int64_t row = r0 + r;
#pragma unroll
      for (int s = 0; s < KS / 4; ++s) {
        const int q = (t >> 6) + 4 * s;
        const int col = k0 + q;
        Xs[q][r] = (row < n && col < p) ? X[row + (int64_t)col * ldx] : 0.f;
      }
    }
    {
      const int q = t & (KS - 1);
      const int kr = k0 + q;
#pragma unroll
      for (int s = 0; s < kTile * KS / kThreads; ++s) {
        const int c = t / KS + (kThreads / KS) * s;
        const int cc = c0 + c;
        const bool ok = kr < p && cc < p && kr <= cc;
        Zh[c][q] = ok ? Zhp[kr + (size_t)cc * p] : 0.f;
        Zl[c][q] = ok ? Zlp[kr + (size_t)cc * p] : 0.f;
      }
    }
    __syncthreads();
    bool live[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) live[v] = c0 + 16 * v + 15 >= k0;
#pragma unroll 2
    for (int q = 0; q < KS; ++q) {
      float a[4], bh[4], bl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Xs[q][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        bh[v] = live[v] ? Zh[ty + 16 * v][q] : 0.f;
        bl[v] = live[v] ? Zl[ty + 16 * v][q] : 0.f;
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (!live[v]) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float h = __fmul_rn(a[u], bh[v]);
          const float r = __fmaf_rn(a[u], bh[v], -h);          // x z_hi - h, exact
          exact_add(acc[u][v], h, __fmaf_rn(a[u], bl[v], r));  // + x z_lo
        }
      }
    }
    __syncthreads();
    since += KS;
    if (since >= kExactSeg) {
      since = 0;
      const bool block = ++segs == kExactSeg2;
      if (block) segs = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          exact_seg(acc[u][v]);
          if (block) exact_block(acc[u][v]);
        }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int c = c0 + ty + 16 * v;
    if (c >= p) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t r = r0 + tx + 16 * u;
      if (r < n) Q[r + (int64_t)c * ldq] = (To)exact_value(acc[u][v]);
    }
  }
}

// ||B - I||_F: one CTA per column (coalesced), then the column sums in order.
__global__ void feas_col_kernel(int p, const double* __restrict__ B, double* __restrict__ col) {
  __shared__ double scratch[33];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const double d = B[i + (size_t)j * p] - (i == j ? 1.0 : 0.0);
    s += d * d;
  }
  const double tot = block_sum(s, scratch);
  if (threadIdx.x == 0) col[j] = tot;
}

__global__ void feas_sum_kernel(int p, const double* __restrict__ col, double* __restrict__ out) {
  __shared__ double scratch[33];
  double s = 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) s += col[j];
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
  cudaError_t e = cudaMemcpyAsync(W, B, (size_t)p * p * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Z, 0, (size_t)p * p * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int nbt = (p + kCB - 1) / kCB;
  for (int jb = 0; jb < nbt; ++jb) {
    const int j0 = jb * kCB;
    chol_diag_kernel<<<1, 1024, 0, s>>>(p, j0, W, Z, info);
    const int rest = nbt - 1 - jb;   // block columns to the right
    if (rest > 0) {
      chol_row_kernel<<<rest, 256, 0, s>>>(p, j0, W, Z, info);
      chol_update_kernel<<<dim3(rest, rest), 256, 0, s>>>(p, j0, W, info);
    }
  }
  for (int sz = kCB; sz < p; sz *= 2) {
    const int pairs = (p + 2 * sz - 1) / (2 * sz);
    const dim3 grid((unsigned)((sz + kCB - 1) / kCB), (unsigned)((sz + kCB - 1) / kCB),
                    (unsigned)pairs);
    rinv_pair_t_kernel<<<grid, 256, 0, s>>>(p, sz, W, Z, info);
    rinv_pair_z_kernel<<<grid, 256, 0, s>>>(p, sz, Z, info);
  }
  {
    int blocks = (int)(((size_t)p * p + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    zero_lower_kernel<<<blocks, 256, 0, s>>>(p, Z);
  }
  return cudaGetLastError();
}

int cholesky_inverse_launches(int p) {
  if (p <= kCholSmemMaxP) return 1;
  const int nbt = (p + kCB - 1) / kCB;
  int levels = 0;
  for (int sz = kCB; sz < p; sz *= 2) ++levels;
  return nbt + 2 * (nbt - 1) + 2 * levels + 1;
}

// scratch: p^2 doubles (the float planes of Z for a float X; unused for a double X).
static cudaError_t launch_split_z(int p, const double* Z, double* scratch, cudaStream_t s) {
  int blocks = (int)(((size_t)p * p + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  float* zh = reinterpret_cast<float*>(scratch);
  split_z_kernel<<<blocks, 256, 0, s>>>(p, Z, zh, zh + (size_t)p * p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_rinv(int64_t n, int p, const T* X, int64_t ldx, const double* Z, double* Q,
                              int64_t ldq, double* scratch, cudaStream_t s) {
  dim3 grid((unsigned)((n + kTile - 1) / kTile), (p + kTile - 1) / kTile);
  if constexpr (std::is_same<T, float>::value) {
    cudaError_t e = launch_split_z(p, Z, scratch, s);
    if (e != cudaSuccess) return e;
    const float* zh = reinterpret_cast<const float*>(scratch);
    apply_rinv_exact_kernel<double><<<grid, kThreads, 0, s>>>(n, p, X, ldx, zh, zh + (size_t)p * p,
                                                              Q, ldq, nullptr);
  } else {
    apply_rinv_kernel<T, double><<<grid, kThreads, 0, s>>>(n, p, X, ldx, Z, Q, ldq, nullptr);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_rinv_same(int64_t n, int p, const T* X, int64_t ldx, const double* Z, T* Q,
                                   int64_t ldq, double* scratch, const DevState* st,
                                   cudaStream_t s) {
  dim3 grid((unsigned)((n + kTile - 1) / kTile), (p + kTile - 1) / kTile);
  if constexpr (std::is_same<T, float>::value) {
    cudaError_t e = launch_split_z(p, Z, scratch, s);
    if (e != cudaSuccess) return e;
    const float* zh = reinterpret_cast<const float*>(scratch);
    apply_rinv_exact_kernel<float><<<grid, kThreads, 0, s>>>(n, p, X, ldx, zh, zh + (size_t)p * p,
                                                             Q, ldq, st);
  } else {
    apply_rinv_kernel<T, T><<<grid, kThreads, 0, s>>>(n, p, X, ldx, Z, Q, ldq, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_feas(int p, const double* B, double* col, double* out, cudaStream_t s) {
  feas_col_kernel<<<p, 128, 0, s>>>(p, B, col);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  feas_sum_kernel<<<1, 256, 0, s>>>(p, col, out);
  return cudaGetLastError();
}

template cudaError_t launch_apply_rinv<float>(int64_t, int, const float*, int64_t, const double*,
                                              double*, int64_t, double*, cudaStream_t);
template cudaError_t launch_apply_rinv<double>(int64_t, int, const double*, int64_t, const double*,
                                               double*, int64_t, double*, cudaStream_t);
template cudaError_t launch_apply_rinv_same<float>(int64_t, int, const float*, int64_t,
                                                   const double*, float*, int64_t, double*,
                                                   const DevState*, cudaStream_t);
template cudaError_t launch_apply_rinv_same<double>(int64_t, int, const double*, int64_t,
                                                    const double*, double*, int64_t, double*,
                                                    const DevState*, cudaStream_t);

}  // namespace plam
