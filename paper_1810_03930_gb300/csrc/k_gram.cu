// Tall-skinny Grams B = X^T X and C = X^T G (Table "cost" rows X^T X and
// grad f^T X), split over row chunks, then reduced in a fixed order.
//
// gram_partial_kernel: one CTA per (64 x 64 output tile, row chunk).  Tiles of
// B are computed only on and above the diagonal (B is symmetric); all tiles of
// C are computed.  Rows are staged 32 at a time in shared memory exactly as
// they lie in memory (contiguous along the row index), so global loads are
// coalesced and the Gram inner product runs over shared memory.  In FP32 mode
// the products and running sums are float; every kFlushRows rows the running
// sums are added into an outer float sum with Kahan compensation, so the
// rounding error grows with sqrt(kFlushRows) rather than with the chunk
// length.  (GB300 executes FP64 at 1/64 of the FP32 rate, so FP32 mode keeps
// double arithmetic out of every O(n p^2) and O(chunks p^2) loop.)  FP64 mode
// is double throughout.  The chunk's partial tile is written in the storage
// type to part[chunk][col][row] with col in [0, p) for B and [p, 2p) for C.
//
// gram_reduce_kernel: B and C (double) from the partials, summed over chunks
// in chunk order (bitwise reproducible; FP32 partials with Kahan compensation).
//
// gram_chunk_reduce_kernel + gram_finalize_kernel: the same reduction
// (coalesced, fixed order) followed by the p x p part of one iteration (one
// CTA per row i of the symmetric matrices):
//   Lambda0 = Psi(C)                                  eq. (Lambda1)
//   d_i = diag(X^T grad_X L_beta(X, Lambda0))_i        eq. (lambda2)
//       = C_ii - sum_k B_ik Lambda0_ik + beta (sum_k B_ik^2 - B_ii)
//     (since X^T (G - X Lambda0 + beta X (B - I)) = C - B Lambda0 + beta B (B - I)
//      and B, Lambda0 are symmetric)
//   M = Lambda0 + Diag(d) - beta (B - I)               eq. (S1): grad_X L_beta = G - X M
//   or, for PLAM-DA / PCAL-DA (Section 5.3), the dual ascent step of Algorithm 1
//   Lambda^k = Lambda^{k-1} - beta (B^k - I), Lambda^0 = Psi(C^0), M = Lambda^k - beta (B - I)
//   feas_row_i = sum_j (B_ij - delta_ij)^2
// M is symmetric, so column i of M is row i.
#include <type_traits>

#include "exact_sum.cuh"
#include "plam_device.cuh"

namespace plam {

__device__ inline void decode_tile(int bx, int nt, int& ti, int& tj, int& isg) {
  const int upper = nt * (nt + 1) / 2;
  if (bx < upper) {
    int r = 0, rem = bx;
    while (rem >= nt - r) { rem -= nt - r; ++r; }
    ti = r; tj = r + rem; isg = 0;
  } else {
    const int idx = bx - upper;
    ti = idx % nt; tj = idx / nt; isg = 1;
  }
}

// Fixed-order sum of the partials of one entry over the chunks.
template <typename T>
__device__ inline double sum_chunks(const T* __restrict__ src, int nchunks, size_t cstride) {
  if (sizeof(T) == 8) {
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += (double)src[(size_t)c * cstride];
    return s;
  } else {
    float s = 0.0f, comp = 0.0f;
    for (int c = 0; c < nchunks; ++c) {
      const float y = (float)src[(size_t)c * cstride] - comp;
      const float t = s + y;
      comp = (t - s) - y;
      s = t;
    }
    return (double)s - (double)comp;
  }
}

// Tin: element type of X and G.  T: arithmetic / partial type (float, or
// double; double with float inputs forms exact products, used by the final
// orthonormalisation).
template <typename Tin, typename T>
__global__ void __launch_bounds__(kThreads)
gram_partial_kernel(int64_t n, int p, const Tin* __restrict__ X, int64_t ldx, const Tin* __restrict__ G,
                    int64_t ldg, int64_t rows_per_chunk, T* __restrict__ part,
                    const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  const int nt = (p + kTile - 1) / kTile;
  int ti, tj, isg;
  decode_tile(blockIdx.x, nt, ti, tj, isg);
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  const Tin* __restrict__ Y = isg ? G : X;
  const int64_t ldy = isg ? ldg : ldx;
  const int i0 = ti * kTile, j0 = tj * kTile;

  __shared__ T As[kTile][kKStep + 1];
  __shared__ T Bs[kTile][kKStep + 1];

  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int kk = t & (kKStep - 1);
  const int cb = t / kKStep;
  T acc[4][4], oacc[4][4], ocmp[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) { acc[u][v] = T(0); oacc[u][v] = T(0); ocmp[u][v] = T(0); }
  int since = 0;

  for (int64_t k0 = r0; k0 < r1; k0 += kKStep) {
    const int64_t row = k0 + kk;
    const bool rok = row < r1;
#pragma unroll
    for (int s = 0; s < kTile / 8; ++s) {
      const int c = cb + 8 * s;
      const int ci = i0 + c, cj = j0 + c;
      As[c][kk] = (rok && ci < p) ? (T)X[row + (int64_t)ci * ldx] : T(0);
      Bs[c][kk] = (rok && cj < p) ? (T)Y[row + (int64_t)cj * ldy] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < kKStep; ++q) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[tx + 16 * u][q]; b[u] = Bs[ty + 16 * u][q]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
    if (sizeof(T) == 4) {
      since += kKStep;
      if (since >= kFlushRows) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const T y = acc[u][v] - ocmp[u][v];
            const T tt = oacc[u][v] + y;
            ocmp[u][v] = (tt - oacc[u][v]) - y;
            oacc[u][v] = tt;
            acc[u][v] = T(0);
          }
        since = 0;
      }
    }
  }
  const size_t cstride = (size_t)2 * p * p;
  T* out = part + (size_t)blockIdx.y * cstride;
  const int cofs = isg ? p : 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tx + 16 * u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + ty + 16 * v;
      if (i < p && j < p) out[(size_t)(cofs + j) * p + i] = (oacc[u][v] - ocmp[u][v]) + acc[u][v];
    }
  }
}

// The FP64 Gram X^T X of a float X (the final orthonormalisation's, and MOptQR's retraction's)
// without FP64 multiplies: each product is formed exactly in FP32 arithmetic and summed in the
// three levels of exact_sum.cuh (a double addition every 1024 rows).  Same tiles, stages and
// partial layout as gram_partial_kernel (B only: G is not used).
// Tin = double (the feasibility report of a double Q): each entry is split into float parts
// q = q_hi + q_lo (about 48 bits), q_hi q_hi' is formed exactly and the cross terms
// q_hi q_lo' + q_lo q_hi' in FP32 (q_lo q_lo' is below 2^-48 of the product and dropped).
template <typename Tin>
__global__ void __launch_bounds__(kThreads, 1)
gram_partial_exact_kernel(int64_t n, int p, const Tin* __restrict__ X, int64_t ldx,
                          int64_t rows_per_chunk, double* __restrict__ part,
                          const DevState* __restrict__ st) {
  constexpr bool kSplit = std::is_same<Tin, double>::value;
  if (st != nullptr && st->stop != kRunning) return;
  const int nt = (p + kTile - 1) / kTile;
  int ti, tj, isg;
  decode_tile(blockIdx.x, nt, ti, tj, isg);
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  const int i0 = ti * kTile, j0 = tj * kTile;

  __shared__ float As[kTile][kKStep + 1];
  __shared__ float Bs[kTile][kKStep + 1];
  __shared__ float Al[kSplit ? kTile : 1][kKStep + 1];
  __shared__ float Bl[kSplit ? kTile : 1][kKStep + 1];

  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int kk = t & (kKStep - 1);
  const int cb = t / kKStep;
  ExactAcc acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) exact_zero(acc[u][v]);
  int since = 0, segs = 0;

  for (int64_t k0 = r0; k0 < r1; k0 += kKStep) {
    const int64_t row = k0 + kk;
    const bool rok = row < r1;
#pragma unroll
    for (int s = 0; s < kTile / 8; ++s) {
      const int c = cb + 8 * s;
      const int ci = i0 + c, cj = j0 + c;
      if constexpr (kSplit) {
        const double xa = (rok && ci < p) ? X[row + (int64_t)ci * ldx] : 0.0;
        const double xb = (rok && cj < p) ? X[row + (int64_t)cj * ldx] : 0.0;
        const float ha = (float)xa, hb = (float)xb;
        As[c][kk] = ha;
        Bs[c][kk] = hb;
        Al[c][kk] = (float)(xa - (double)ha);
        Bl[c][kk] = (float)(xb - (double)hb);
      } else {
        As[c][kk] = (rok && ci < p) ? X[row + (int64_t)ci * ldx] : 0.f;
        Bs[c][kk] = (rok && cj < p) ? X[row + (int64_t)cj * ldx] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 2
    for (int q = 0; q < kKStep; ++q) {
      float a[4], b[4], al[4], bl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[tx + 16 * u][q];
        b[u] = Bs[ty + 16 * u][q];
        if constexpr (kSplit) {
          al[u] = Al[tx + 16 * u][q];
          bl[u] = Bl[ty + 16 * u][q];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float h = __fmul_rn(a[u], b[v]);
          float r = __fmaf_rn(a[u], b[v], -h);                // x y - h, exact
          if constexpr (kSplit) r = __fadd_rn(r, __fmaf_rn(al[u], b[v], __fmul_rn(a[u], bl[v])));
          exact_add(acc[u][v], h, r);
        }
    }
    __syncthreads();
    since += kKStep;
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
  const size_t cstride = (size_t)2 * p * p;
  double* out = part + (size_t)blockIdx.y * cstride;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tx + 16 * u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + ty + 16 * v;
      if (i < p && j < p) out[(size_t)j * p + i] = exact_value(acc[u][v]);
    }
  }
}

template <typename T>
__global__ void gram_reduce_kernel(int p, int nchunks, int with_g, const T* __restrict__ part,
                                   double* __restrict__ B, double* __restrict__ C) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int col = blockIdx.y * 8 + threadIdx.y;
  const int ncols = with_g ? 2 * p : p;
  if (i >= p || col >= ncols) return;
  if (col < p && i > col) return;
  const size_t cstride = (size_t)2 * p * p;
  const double s = sum_chunks<T>(part + (size_t)col * p + i, nchunks, cstride);
  if (col < p) {
    B[i + (size_t)col * p] = s;
    B[col + (size_t)i * p] = s;
  } else {
    C[i + (size_t)(col - p) * p] = s;
  }
}

// Cross-chunk reduction of the partial Grams, coalesced: each CTA owns 32
// consecutive entries of the 2p x p partial layout (lane = entry), its 8 warps
// sum the chunks c = w, w + 8, ... in increasing order, and the 8 warp sums
// are added in warp order (bitwise reproducible).  Entries of the lower
// triangle of B are never formed and are skipped.  red: 2p x p, double.
constexpr int kRedWarps = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kRedWarps)
gram_chunk_reduce_kernel(int p, int nchunks, const T* __restrict__ part, double* __restrict__ red,
                         const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  __shared__ T ws[kRedWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t E = (size_t)2 * p * p;
  const size_t e = (size_t)blockIdx.x * 32 + lane;
  const bool live = e < E && !((int)(e / p) < p && (int)(e % p) > (int)(e / p));
  T v = T(0);
  if (live) {
#pragma unroll 4
    for (int c = w; c < nchunks; c += kRedWarps) v += part[(size_t)c * E + e];
  }
  ws[w][lane] = v;
  __syncthreads();
  if (w == 0 && live) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kRedWarps; ++i) s += ws[i][lane];
    red[e] = (double)s;
  }
}

// p x p part of one iteration from the reduced Grams (one CTA per row i; B is
// read through its upper triangle, B_ij = red[max(i,j) p + min(i,j)]).
template <typename T>
__global__ void __launch_bounds__(128)
gram_finalize_kernel(int p, const double* __restrict__ red, double* __restrict__ Bout,
                     double* __restrict__ L0out, T* __restrict__ Mt, T* __restrict__ L0t,
                     double* __restrict__ feas_row, const DevState* __restrict__ st, IterParams prm) {
  if (st != nullptr && st->stop != kRunning) return;
  extern __shared__ double sh[];
  double* Brow = sh;          // B_ij
  double* Lrow = sh + p;      // Psi(C)_ij
  __shared__ double scratch[33];
  __shared__ double cii;
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double b = red[(size_t)max(i, j) * p + min(i, j)];
    const double cij = red[(size_t)(p + j) * p + i];
    const double cji = red[(size_t)(p + i) * p + j];
    Brow[j] = b;
    Lrow[j] = 0.5 * (cij + cji);
    if (j == i) cii = cij;
  }
  __syncthreads();
  double t1 = 0.0, t2 = 0.0, tf = 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double bij = Brow[j];
    t1 += bij * Lrow[j];
    t2 += bij * bij;
    const double e = bij - (j == i ? 1.0 : 0.0);
    tf += e * e;
  }
  const double s1 = block_sum(t1, scratch);
  const double s2 = block_sum(t2, scratch);
  const double sf = block_sum(tf, scratch);
  const double beta = prm.beta;
  const double d = prm.lambda2 ? (cii - s1 + beta * (s2 - Brow[i])) : 0.0;
  const bool da = prm.lambda_da && prm.lam != nullptr;
  const bool da_first = da && (st == nullptr || st->k == 0);
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double delta = (j == i) ? 1.0 : 0.0;
    double lam = Lrow[j] + delta * d;
    if (da) {   // dual ascent (Algorithm 1's multiplier step) from Lambda^0 = Psi(C^0)
      double* lp = prm.lam + j + (size_t)i * p;
      lam = da_first ? Lrow[j] : *lp - beta * (Brow[j] - delta);
      *lp = lam;
    }
    // MOptQR (Table "cost"): R = G - X (G^T X), i.e. the product with C^T = G^T X
    const double m = prm.moptqr ? red[(size_t)(p + j) * p + i] : lam - beta * (Brow[j] - delta);
    Mt[j + (size_t)i * p] = (T)m;
    L0t[j + (size_t)i * p] = (T)Lrow[j];
    if (Bout) Bout[j + (size_t)i * p] = Brow[j];
    if (L0out) L0out[j + (size_t)i * p] = Lrow[j];
  }
  if (threadIdx.x == 0) feas_row[i] = sf;
}

// ---------------------------------------------------------------- launchers

template <typename Tin, typename T>
cudaError_t launch_gram_partial(int64_t n, int p, const Tin* X, int64_t ldx, const Tin* G,
                                int64_t ldg, int64_t rows_per_chunk, int nchunks, T* part,
                                const DevState* st, cudaStream_t s) {
  const int nt = (p + kTile - 1) / kTile;
  const int tiles = nt * (nt + 1) / 2 + (G ? nt * nt : 0);
  dim3 grid(tiles, nchunks);
  if constexpr (std::is_same<Tin, float>::value && std::is_same<T, double>::value) {
    if (G == nullptr) {   // the FP64 Gram of a float X: exact products, compensated FP32 sums
      gram_partial_exact_kernel<float><<<grid, kThreads, 0, s>>>(n, p, X, ldx, rows_per_chunk, part,
                                                                 st);
      return cudaGetLastError();
    }
  }
  gram_partial_kernel<Tin, T><<<grid, kThreads, 0, s>>>(n, p, X, ldx, G, ldg, rows_per_chunk, part,
                                                          st);
  return cudaGetLastError();
}

cudaError_t launch_gram_report(int64_t n, int p, const double* Q, int64_t ldq,
                               int64_t rows_per_chunk, int nchunks, double* part, cudaStream_t s) {
  const int nt = (p + kTile - 1) / kTile;
  dim3 grid(nt * (nt + 1) / 2, nchunks);
  gram_partial_exact_kernel<double><<<grid, kThreads, 0, s>>>(n, p, Q, ldq, rows_per_chunk, part,
                                                              nullptr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram_reduce(int p, int nchunks, int with_g, const T* part, double* B,
                               double* C, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((p + 31) / 32, ((with_g ? 2 * p : p) + 7) / 8);
  gram_reduce_kernel<T><<<grid, block, 0, s>>>(p, nchunks, with_g, part, B, C);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram_finalize(int p, int nchunks, const T* part, double* red, double* B,
                                 double* L0, T* Mt, T* L0t, double* feas_row, const DevState* st,
                                 IterParams prm, cudaStream_t s, int stage) {
  cudaError_t e = cudaSuccess;
  if (stage != 2) {
    const size_t E = (size_t)2 * p * p;
    gram_chunk_reduce_kernel<T><<<(unsigned)((E + 31) / 32), 32 * kRedWarps, 0, s>>>(p, nchunks,
                                                                                   part, red, st);
    e = cudaGetLastError();
    if (e != cudaSuccess || stage == 1) return e;
  }
  const size_t smem = (size_t)2 * p * sizeof(double);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(gram_finalize_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
  }
  gram_finalize_kernel<T><<<p, 128, smem, s>>>(p, red, B, L0, Mt, L0t, feas_row, st, prm);
  return cudaGetLastError();
}

cudaError_t preload_gram_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_partial_kernel<float, float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_partial_kernel<float, double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_partial_kernel<double, double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_partial_exact_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_partial_exact_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_reduce_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_reduce_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_finalize_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_finalize_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_chunk_reduce_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_chunk_reduce_kernel<double>);
  return e;
}

template cudaError_t launch_gram_partial<float, float>(int64_t, int, const float*, int64_t,
                                                       const float*, int64_t, int64_t, int, float*,
                                                       const DevState*, cudaStream_t);
template cudaError_t launch_gram_partial<float, double>(int64_t, int, const float*, int64_t,
                                                        const float*, int64_t, int64_t, int, double*,
                                                        const DevState*, cudaStream_t);
template cudaError_t launch_gram_partial<double, double>(int64_t, int, const double*, int64_t,
                                                         const double*, int64_t, int64_t, int,
                                                         double*, const DevState*, cudaStream_t);
template cudaError_t launch_gram_reduce<float>(int, int, int, const float*, double*, double*,
                                               cudaStream_t);
template cudaError_t launch_gram_reduce<double>(int, int, int, const double*, double*, double*,
                                                cudaStream_t);
template cudaError_t launch_gram_finalize<float>(int, int, const float*, double*, double*, double*,
                                                 float*, float*, double*, const DevState*,
                                                 IterParams, cudaStream_t, int);
template cudaError_t launch_gram_finalize<double>(int, int, const double*, double*, double*,
                                                  double*, double*, double*, double*,
                                                  const DevState*, IterParams, cudaStream_t, int);

}  // namespace plam
