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
// gram_chunk_reduce_kernel, gram_tile_finalize_kernel, gram_row_finalize_kernel:
// the same reduction (coalesced, fixed order; at large p inside the tile kernel)
// followed by the p x p part of one iteration, on 32 x 32 tile pairs of the
// symmetric matrices, then per row i:
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

// Cross-chunk reduction of the partial Grams, coalesced: each CTA owns 32 * kPer
// entries of the 2p x p partial layout (lane + 32 q, q < kPer), its 8 warps sum the
// chunks c = w, w + 8, ... in increasing order, and the 8 warp sums are added in
// warp order (bitwise reproducible).  Entries of the lower triangle of B are never
// formed and are skipped.  red: 2p x p, double.  kPer > 1 when the entries alone
// give every SM several CTAs (a CTA per 32 entries is launch-bound at large p).
constexpr int kRedWarps = 8;

template <typename T, int kPer>
__global__ void __launch_bounds__(32 * kRedWarps)
gram_chunk_reduce_kernel(int p, int nchunks, const T* __restrict__ part, double* __restrict__ red,
                         const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  __shared__ T ws[kRedWarps][32 * kPer];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t E = (size_t)2 * p * p;
  const size_t e0 = (size_t)blockIdx.x * (32 * kPer) + lane;
  // loads of dead entries read entry 0 of the chunk (always in bounds) and are not added:
  // no branch around a load, so all of a thread's loads of one chunk are in flight together
  unsigned live = 0;
  T v[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const size_t e = e0 + 32 * q;
    if (e < E && !((int)(e / p) < p && (int)(e % p) > (int)(e / p))) live |= 1u << q;
    v[q] = T(0);
  }
#pragma unroll 2
  for (int c = w; c < nchunks; c += kRedWarps) {
    const T* src = part + (size_t)c * E;
    T x[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) x[q] = src[(live >> q & 1u) ? e0 + 32 * q : 0];
#pragma unroll
    for (int q = 0; q < kPer; ++q) v[q] += (live >> q & 1u) ? x[q] : T(0);
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) ws[w][lane + 32 * q] = v[q];
  __syncthreads();
  for (int t = threadIdx.x; t < 32 * kPer; t += blockDim.x) {
    const size_t e = (size_t)blockIdx.x * (32 * kPer) + t;
    if (e >= E || ((int)(e / p) < p && (int)(e % p) > (int)(e / p))) continue;
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kRedWarps; ++i) s += ws[i][t];
    red[e] = (double)s;
  }
}

// The p x p part of one iteration, on 32 x 32 tile pairs.  The CTA of tile pair (a, b),
// a <= b, holds for rows i of tile a and columns j of tile b
//   B_ij (B's upper triangle, as formed), C_ij and C_ji,
// each summed over the chunks in chunk order (or read from the reduced Grams, nchunks = 1),
// with every load coalesced along the partial layout's row index.  It writes
//   Psi(C)_ij = (C_ij + C_ji) / 2 to L0t, and M_ij = Lambda_ij - beta (B_ij - delta_ij) to Mt
//   (Lambda = Psi(C), or the dual ascent step; MOptQR: M_ij = C_ij, M = C^T in Mt's layout),
// for row i and, mirrored, for row j (B, Psi(C), M and Lambda are symmetric), and the row
// sums of B_ij Psi(C)_ij, B_ij^2 and (B_ij - delta_ij)^2 over its 32 columns, one slot per
// (row, column tile): rowpart[(q nt + t) p + row].  A diagonal tile also records B_ii and C_ii
// in dg = rowpart + 3 nt p.  gram_row_finalize_kernel then sums a row's slots in tile order:
//   d_i = C_ii - sum_j B_ij Psi_ij + beta (sum_j B_ij^2 - B_ii)      eq. (lambda2)
//   M_ii = (Psi_ii + d_i) - beta (B_ii - 1),  feas_row_i = sum_j (B_ij - delta_ij)^2.
constexpr int kFinTile = 32;
constexpr int kFinThreads = 256;

// (a + b) / 2 = h + l exactly (TwoSum; halving is exact above the subnormal range).
__device__ __forceinline__ float half_sum(float a, float b, float& l) {
  float e;
  const float s = two_sum(a, b, e);
  l = 0.5f * e;
  return 0.5f * s;
}

__device__ inline void decode_upper(int bx, int nt, int& a, int& b) {
  int r = 0, rem = bx;
  while (rem >= nt - r) { rem -= nt - r; ++r; }
  a = r;
  b = r + rem;
}

template <typename Tp, typename T>
__global__ void __launch_bounds__(kFinThreads)
gram_tile_finalize_kernel(int p, int nchunks, const Tp* __restrict__ part,
                          double* __restrict__ rowpart, T* __restrict__ Mt, T* __restrict__ L0t,
                          const DevState* __restrict__ st, IterParams prm) {
  if (st != nullptr && st->stop != kRunning) return;
  __shared__ T sB[kFinTile][kFinTile + 1];    // B_ij   [i - i0][j - j0]
  __shared__ T sC[kFinTile][kFinTile + 1];    // C_ij
  __shared__ T sCt[kFinTile][kFinTile + 1];   // C_ji
  const int nt = (p + kFinTile - 1) / kFinTile;
  int a, b;
  decode_upper(blockIdx.x, nt, a, b);
  const bool diag = a == b;
  const int i0 = a * kFinTile, j0 = b * kFinTile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t E = (size_t)2 * p * p;
  constexpr int kQ = kFinTile / (kFinThreads / 32);
  // thread (lane, w): B_ij and C_ij at i = i0 + lane, j = j0 + w + 8 q; C_ji at j = j0 + lane,
  // i = i0 + w + 8 q (lane along the partial layout's row index in all three)
  // entry q of a thread lies 8 q columns (8 q p elements) past its entry 0; a dead entry
  // (ragged edge, or B's lower triangle in a diagonal tile) loads element 0 of the chunk and
  // is not added: no branch around a load, so the 3 kQ loads of a chunk are in flight together
  const size_t ob0 = (size_t)(j0 + w) * p + i0 + lane;        // B_ij,  j = j0 + w + 8 q
  const size_t oc0 = (size_t)(p + j0 + w) * p + i0 + lane;    // C_ij
  const size_t ot0 = (size_t)(p + i0 + w) * p + j0 + lane;    // C_ji,  i = i0 + w + 8 q
  const size_t s8 = (size_t)8 * p;
  unsigned mb = 0, mc = 0, mt = 0;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int r = w + 8 * q;
    if (i0 + lane < p && j0 + r < p && (!diag || lane <= r)) mb |= 1u << q;
    if (i0 + lane < p && j0 + r < p) mc |= 1u << q;
    if (!diag && i0 + r < p && j0 + lane < p) mt |= 1u << q;
  }
  Tp vb[kQ], vc[kQ], vt[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) vb[q] = vc[q] = vt[q] = Tp(0);
  for (int c = 0; c < nchunks; ++c) {
    const Tp* src = part + (size_t)c * E;
    Tp xb[kQ], xc[kQ], xt[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      xb[q] = src[(mb >> q & 1u) ? ob0 + q * s8 : 0];
      xc[q] = src[(mc >> q & 1u) ? oc0 + q * s8 : 0];
      xt[q] = src[(mt >> q & 1u) ? ot0 + q * s8 : 0];
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      vb[q] += (mb >> q & 1u) ? xb[q] : Tp(0);
      vc[q] += (mc >> q & 1u) ? xc[q] : Tp(0);
      vt[q] += (mt >> q & 1u) ? xt[q] : Tp(0);
    }
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int r = w + 8 * q;
    sB[lane][r] = (T)vb[q];
    sC[lane][r] = (T)vc[q];
    sCt[r][lane] = (T)vt[q];
  }
  __syncthreads();
  if (diag) {   // B's lower triangle and C_ji from the tile's own C
    for (int t = threadIdx.x; t < kFinTile * kFinTile; t += kFinThreads) {
      const int il = t / kFinTile, jl = t % kFinTile;
      if (il > jl) sB[il][jl] = sB[jl][il];
      sCt[il][jl] = sC[jl][il];
    }
    __syncthreads();
  }
  const double beta = prm.beta;
  const bool da = prm.lambda_da && prm.lam != nullptr;
  const bool da_first = da && (st == nullptr || st->k == 0);
  // FP32 storage: beta = bh + bl to 2^-48, and the entries of Mt and L0t in FP32 arithmetic
  // (GB300 runs FP64 at 1/64 of the FP32 rate), each within about one rounding of its value
  const float bh = (float)beta, bl = (float)(beta - (double)(float)beta);
  // pass 0: row i = i0 + il, column j = j0 + jl; pass 1 (off-diagonal tiles): row j, column i
  for (int pass = 0; pass < (diag ? 1 : 2); ++pass) {
    for (int t = threadIdx.x; t < kFinTile * kFinTile; t += kFinThreads) {
      const int il = pass == 0 ? t / kFinTile : t % kFinTile;
      const int jl = pass == 0 ? t % kFinTile : t / kFinTile;
      const int i = i0 + il, j = j0 + jl;
      if (i >= p || j >= p) continue;
      const int row = pass == 0 ? i : j, col = pass == 0 ? j : i;
      const T bij = sB[il][jl];
      const T crc = pass == 0 ? sC[il][jl] : sCt[il][jl];   // C_row,col
      const T ccr = pass == 0 ? sCt[il][jl] : sC[il][jl];   // C_col,row
      T m, psi_out;
      if constexpr (std::is_same<T, float>::value) {
        float pl;
        const float ph = half_sum(crc, ccr, pl);   // Psi(C)_ij = ph + pl exactly
        psi_out = ph;
        const float e = __fsub_rn(bij, row == col ? 1.f : 0.f);   // exact
        if (prm.moptqr) {   // MOptQR (Table "cost"): R = G - X (G^T X), the product with C^T
          m = crc;
        } else if (da) {    // dual ascent (Algorithm 1's multiplier step), FP64 multiplier
          double* lp = prm.lam + col + (size_t)row * p;
          const double lam = da_first ? (double)ph + (double)pl : *lp - beta * (double)e;
          *lp = lam;
          m = (float)(lam - beta * (double)e);
        } else {            // Lambda - beta (B - I) = (ph + pl) - (th + tl)
          const float th = __fmul_rn(bh, e);
          const float tl = fmaf(bh, e, -th) + bl * e;
          m = __fadd_rn(__fsub_rn(ph, th), __fsub_rn(pl, tl));
        }
      } else {
        const double psi = 0.5 * (crc + ccr);
        const double delta = row == col ? 1.0 : 0.0;
        double lam = psi;
        if (da) {   // dual ascent (Algorithm 1's multiplier step) from Lambda^0 = Psi(C^0)
          double* lp = prm.lam + col + (size_t)row * p;
          lam = da_first ? psi : *lp - beta * (bij - delta);
          *lp = lam;
        }
        // MOptQR (Table "cost"): R = G - X (G^T X), i.e. the product with C^T = G^T X
        m = prm.moptqr ? crc : lam - beta * (bij - delta);
        psi_out = psi;
      }
      Mt[col + (size_t)row * p] = m;
      L0t[col + (size_t)row * p] = psi_out;
    }
  }
  // row sums over the tile's 32 columns: threads 0..95 for rows i (three sums), 96..191 for
  // rows j of an off-diagonal tile (its columns are the rows i of tile a).  FP32 storage: each
  // product split exactly (TwoProduct) and summed as Dot2 (exact_add), so the sum is as
  // accurate as an FP64 one with FP32 arithmetic only
  const int t = threadIdx.x;
  const int side = t / (3 * kFinTile), q = (t / kFinTile) % 3, r = t % kFinTile;
  if (side < (diag ? 1 : 2)) {
    const int row = (side == 0 ? i0 : j0) + r;
    if (row < p) {
      double acc = 0.0;
      if constexpr (std::is_same<T, float>::value) {
        ExactAcc ea;
        exact_zero(ea);
        for (int k = 0; k < kFinTile; ++k) {
          const int il = side == 0 ? r : k, jl = side == 0 ? k : r;
          const float bij = sB[il][jl];
          float x = bij, y = bij, lo = 0.f;
          if (q == 0) {          // B_ij Psi(C)_ij, symmetric in i, j
            float pl;
            y = half_sum(sC[il][jl], sCt[il][jl], pl);
            lo = bij * pl;
          } else if (q == 2) {   // (B_ij - delta_ij)^2
            x = y = __fsub_rn(bij, (i0 + il) == (j0 + jl) ? 1.f : 0.f);
          }
          const float h = __fmul_rn(x, y);
          exact_add(ea, h, fmaf(x, y, -h) + lo);
        }
        acc = exact_value(ea);
      } else {
        for (int k = 0; k < kFinTile; ++k) {
          const int il = side == 0 ? r : k, jl = side == 0 ? k : r;
          const double bij = sB[il][jl];
          double v;
          if (q == 0) {
            v = bij * (0.5 * (sC[il][jl] + sCt[il][jl]));   // B_ij Psi(C)_ij
          } else if (q == 1) {
            v = bij * bij;
          } else {
            const double e = bij - ((i0 + il) == (j0 + jl) ? 1.0 : 0.0);
            v = e * e;
          }
          acc += v;
        }
      }
      rowpart[((size_t)q * nt + (side == 0 ? b : a)) * p + row] = acc;
    }
  }
  if (diag && t < kFinTile && i0 + t < p) {
    double* dg = rowpart + (size_t)3 * nt * p;
    dg[i0 + t] = (double)sB[t][t];
    dg[p + i0 + t] = (double)sC[t][t];
  }
}

// One warp per row: lane l sums the row's slots t = l, l + 32, ... in order, then a fixed
// butterfly adds the 32 lane sums (bitwise reproducible).
constexpr int kRowWarps = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kRowWarps)
gram_row_finalize_kernel(int p, const double* __restrict__ rowpart, T* __restrict__ Mt,
                         double* __restrict__ feas_row, const DevState* __restrict__ st,
                         IterParams prm) {
  if (st != nullptr && st->stop != kRunning) return;
  const int i = blockIdx.x * kRowWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= p) return;
  const int nt = (p + kFinTile - 1) / kFinTile;
  double s1 = 0.0, s2 = 0.0, sf = 0.0;
  for (int t = lane; t < nt; t += 32) {
    s1 += rowpart[(size_t)t * p + i];
    s2 += rowpart[((size_t)nt + t) * p + i];
    sf += rowpart[((size_t)2 * nt + t) * p + i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    sf += __shfl_xor_sync(0xffffffffu, sf, o);
  }
  if (lane != 0) return;
  feas_row[i] = sf;
  const bool da = prm.lambda_da && prm.lam != nullptr;
  if (prm.lambda2 && !da && !prm.moptqr) {
    const double* dg = rowpart + (size_t)3 * nt * p;
    const double bii = dg[i], cii = dg[p + i];   // Psi(C)_ii = C_ii
    const double beta = prm.beta;
    const double d = cii - s1 + beta * (s2 - bii);
    Mt[i + (size_t)i * p] = (T)((cii + d) - beta * (bii - 1.0));
  }
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

size_t gram_rowpart_doubles(int p) {
  const int nt = (p + kFinTile - 1) / kFinTile;
  return ((size_t)3 * nt + 2) * (size_t)p;
}

template <typename T>
static cudaError_t launch_chunk_reduce(int p, int nchunks, const T* part, double* red,
                                       const DevState* st, cudaStream_t s) {
  const size_t E = (size_t)2 * p * p;
  const size_t want = (size_t)8 * device_sm_count();   // CTAs enough to fill the SMs
  if ((E + 255) / 256 >= want) {
    gram_chunk_reduce_kernel<T, 8><<<(unsigned)((E + 255) / 256), 32 * kRedWarps, 0, s>>>(
        p, nchunks, part, red, st);
  } else if ((E + 127) / 128 >= want) {
    gram_chunk_reduce_kernel<T, 4><<<(unsigned)((E + 127) / 128), 32 * kRedWarps, 0, s>>>(
        p, nchunks, part, red, st);
  } else {
    gram_chunk_reduce_kernel<T, 1><<<(unsigned)((E + 31) / 32), 32 * kRedWarps, 0, s>>>(
        p, nchunks, part, red, st);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram_finalize(int p, int nchunks, const T* part, double* red, double* rowpart,
                                 T* Mt, T* L0t, double* feas_row, const DevState* st,
                                 IterParams prm, cudaStream_t s, int stage) {
  cudaError_t e = cudaSuccess;
  const int nt = (p + kFinTile - 1) / kFinTile;
  const unsigned tiles = (unsigned)(nt * (nt + 1) / 2);
  // enough tile pairs to give every SM two CTAs: sum the chunks inside the tile kernel;
  // otherwise reduce over the chunks first (all entries in parallel)
  const bool fused = stage == 0 && tiles >= 2u * (unsigned)device_sm_count();
  if (stage == 1 || (stage == 0 && !fused)) {
    e = launch_chunk_reduce<T>(p, nchunks, part, red, st, s);
    if (e != cudaSuccess || stage == 1) return e;
  }
  if (fused)
    gram_tile_finalize_kernel<T, T><<<tiles, kFinThreads, 0, s>>>(p, nchunks, part, rowpart, Mt,
                                                                  L0t, st, prm);
  else
    gram_tile_finalize_kernel<double, T><<<tiles, kFinThreads, 0, s>>>(p, 1, red, rowpart, Mt,
                                                                       L0t, st, prm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_row_finalize_kernel<T><<<(unsigned)((p + kRowWarps - 1) / kRowWarps), 32 * kRowWarps, 0,
                                 s>>>(p, rowpart, Mt, feas_row, st, prm);
  return cudaGetLastError();
}

int gram_finalize_launches(int p, int stage) {
  const int nt = (p + kFinTile - 1) / kFinTile;
  const bool fused = stage == 0 && nt * (nt + 1) / 2 >= 2 * device_sm_count();
  if (stage == 1) return 1;
  return (stage == 0 && !fused) ? 3 : 2;
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
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_tile_finalize_kernel<float, float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_tile_finalize_kernel<double, float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_tile_finalize_kernel<double, double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_row_finalize_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_row_finalize_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_chunk_reduce_kernel<float, 1>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_chunk_reduce_kernel<float, 4>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_chunk_reduce_kernel<float, 8>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_chunk_reduce_kernel<double, 1>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_chunk_reduce_kernel<double, 4>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gram_chunk_reduce_kernel<double, 8>);
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
template cudaError_t launch_gram_finalize<float>(int, int, const float*, double*, double*, float*,
                                                 float*, double*, const DevState*, IterParams,
                                                 cudaStream_t, int);
template cudaError_t launch_gram_finalize<double>(int, int, const double*, double*, double*,
                                                  double*, double*, double*, const DevState*,
                                                  IterParams, cudaStream_t, int);

}  // namespace plam
