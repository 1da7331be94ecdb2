// Gradients of the built-in objectives (Section 5.2; Table "cost", rows
// "evaluate function").
//
// dense_grad_kernel     G = A X for f = 1/2 tr(X^T A X) (Problem 3), a tiled
//                       64 x 64 GEMM over shared-memory stages of A and X.
// right_multiply_kernel Y = X B (n x p times p x p): with the dense kernel, Problem 4's
//                       gradient A X B of f = 1/2 tr(A^T X B X^T) (eq. QAP).
// hartree kernels       f = q tr(X^T L X) + (alpha/4) rho^T L^{-1} rho - (3 xc / 4) sum rho^{4/3}
//                       (the last term: Problem 6's exchange, 0 unless xc is set)
//                       (eq. KS-energy, Problem 1 with L = tridiag(-1,2,-1)),
//                       G = 2 q L X + alpha Diag(y) X with y = L^{-1} rho.
//   The Dirichlet Laplacian has the closed-form inverse (1-based indices)
//       (L^{-1})_ij = min(i,j) (n+1-max(i,j)) / (n+1),
//   so y_i = [ (n+1-i) P_i + i Q_i ] / (n+1) with the prefix / suffix sums
//       P_i = sum_{j<=i} j rho_j,   Q_i = sum_{j>i} (n+1-j) rho_j,
//   all terms non-negative (no cancellation).  Kernel 1 forms rho and the
//   per-block sums of j rho_j and (n+1-j) rho_j; kernel 2 adds the sums of the
//   preceding / following blocks in a fixed order, scans inside its block,
//   forms y and writes G and the block's share of rho^T y (for f).  rho, y and
//   the scans are double (O(n) work); G is computed in the storage type.
// chain kernels         the same 1D objective with a block-diagonal L and Problem 2's linear
//                       term (Section 5.4), over row tiles x column groups (see below).
// stencil_grad_kernel   G = (L3 + Diag(V)) X, L3 the 7-point Dirichlet
//                       Laplacian (6 on the diagonal, -1 per neighbour inside
//                       the grid), index i = x + nx (y + ny z).
#include "plam_device.cuh"

namespace plam {

// ---------------------------------------------------------------- dense

template <typename T>
__global__ void __launch_bounds__(kThreads)
dense_grad_kernel(int64_t n, int p, const T* __restrict__ A, int64_t lda, const T* __restrict__ X,
                  int64_t ldx, T* __restrict__ G, int64_t ldg, const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  constexpr int KS = sizeof(T) == 8 ? 16 : kKStep;
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int c0 = blockIdx.y * kTile;
  __shared__ T As[KS][kTile];
  __shared__ T Bs[kTile][KS + 1];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  for (int64_t k0 = 0; k0 < n; k0 += KS) {
    {
      const int r = t & (kTile - 1);
      const int64_t row = r0 + r;
#pragma unroll
      for (int s = 0; s < KS / 4; ++s) {
        const int q = (t >> 6) + 4 * s;
        const int64_t col = k0 + q;
        As[q][r] = (row < n && col < n) ? A[row + col * lda] : T(0);
      }
    }
    {
      const int q = t & (KS - 1);
      const int64_t kr = k0 + q;
#pragma unroll
      for (int s = 0; s < kTile * KS / kThreads; ++s) {
        const int c = t / KS + (kThreads / KS) * s;
        const int cc = c0 + c;
        Bs[c][q] = (kr < n && cc < p) ? X[kr + (int64_t)cc * ldx] : T(0);
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < KS; ++q) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[q][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[ty + 16 * v][q];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
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
      if (r < n) G[r + (int64_t)c * ldg] = acc[u][v];
    }
  }
}

// ---------------------------------------------------------------- Hartree (1D)

constexpr int kHB = 256;   // rows per Hartree block

int hartree_blocks(int64_t n) { return (int)((n + kHB - 1) / kHB); }

template <typename T>
__global__ void __launch_bounds__(kHB)
hartree_density_kernel(int64_t n, int p, const T* __restrict__ X, int64_t ldx,
                       double* __restrict__ rho, double* __restrict__ blk,
                       const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  __shared__ double scratch[33];
  const int64_t r = (int64_t)blockIdx.x * kHB + threadIdx.x;
  double rv = 0.0;
  if (r < n) {
    T s = T(0);
    for (int c = 0; c < p; ++c) {
      const T x = X[r + (int64_t)c * ldx];
      s = fma(x, x, s);
    }
    rv = (double)s;
    rho[r] = rv;
  }
  const double i1 = (double)(r + 1);                 // 1-based index
  const double w2 = (double)(n - r);                 // n + 1 - i
  const double s1 = block_sum(r < n ? i1 * rv : 0.0, scratch);
  const double s2 = block_sum(r < n ? w2 * rv : 0.0, scratch);
  if (threadIdx.x == 0) {
    blk[2 * blockIdx.x] = s1;
    blk[2 * blockIdx.x + 1] = s2;
  }
}

template <typename T>
__global__ void __launch_bounds__(kHB)
hartree_grad_kernel(int64_t n, int p, double alpha, double q, double xc, double inv_np1,
                    const T* __restrict__ X, int64_t ldx,
                    T* __restrict__ G, int64_t ldg, const double* __restrict__ rho,
                    const double* __restrict__ blk, double* __restrict__ yout,
                    double* __restrict__ fpart, const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  __shared__ double scratch[33];
  __shared__ double wscan[2][kHB / 32];
  const int b = blockIdx.x;
  const int nb = gridDim.x;
  // sums over the preceding blocks (P) and the following blocks (Q), fixed order
  double pa = 0.0, qa = 0.0;
  for (int j = threadIdx.x; j < nb; j += kHB) {
    if (j < b) pa += blk[2 * j];
    if (j > b) qa += blk[2 * j + 1];
  }
  const double Pbefore = block_sum(pa, scratch);
  const double Qafter = block_sum(qa, scratch);
  const int64_t r = (int64_t)b * kHB + threadIdx.x;
  const double rv = (r < n) ? rho[r] : 0.0;
  const double i1 = (double)(r + 1);
  const double w2 = (double)(n - r);
  // inclusive scan of i rho_i and of (n+1-i) rho_i inside the block
  double a = (r < n) ? i1 * rv : 0.0;
  double c = (r < n) ? w2 * rv : 0.0;
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double ta = __shfl_up_sync(0xffffffffu, a, o);
    const double tc = __shfl_up_sync(0xffffffffu, c, o);
    if (l >= o) { a += ta; c += tc; }
  }
  if (l == 31) { wscan[0][w] = a; wscan[1][w] = c; }
  __syncthreads();
  double wa = 0.0, wc = 0.0, ctot = 0.0;
  for (int j = 0; j < kHB / 32; ++j) {
    if (j < w) { wa += wscan[0][j]; wc += wscan[1][j]; }
    ctot += wscan[1][j];
  }
  const double incl_a = a + wa;          // sum_{j <= i, j in block} j rho_j
  const double incl_c = c + wc;          // sum_{j <= i, j in block} (n+1-j) rho_j
  const double P = Pbefore + incl_a;
  const double Q = Qafter + (ctot - incl_c);   // strictly after i
  const double y = ((double)(n - r) * P + i1 * Q) * inv_np1;   // 1/(n+1) from the host
  // f partial of this block: f = 1/2 <X, G> - (alpha/4) rho^T y + (xc/4) sum rho^{4/3}
  const double c3 = (xc != 0.0 && r < n) ? cbrt(rv) : 0.0;
  const double fy = block_sum((r < n) ? -0.25 * alpha * rv * y + 0.25 * xc * rv * c3 : 0.0, scratch);
  if (threadIdx.x == 0 && fpart) fpart[b] = fy;
  if (r >= n) return;
  if (yout) yout[r] = y;
  // row scale: alpha L^{-1} rho (Hartree) - 2 xc rho^{1/3} (exchange, Problem 6)
  const T ty = (T)(alpha * y - 2.0 * xc * c3);
  const T q2 = (T)(2.0 * q);
  for (int cc = 0; cc < p; ++cc) {
    const T* xc = X + (int64_t)cc * ldx;
    const T x = xc[r];
    const T xm = (r > 0) ? xc[r - 1] : T(0);
    const T xp = (r + 1 < n) ? xc[r + 1] : T(0);
    const T lx = (x + x) - xm - xp;
    G[r + (int64_t)cc * ldg] = fma(q2, lx, ty * x);
  }
}

// ---------------------------------------------------------------- 1D, block-diagonal L, linear term
//
// The parallel forms of Problems 1 and 2 in Section 5.4:
//   f = q tr(X^T L X) + (alpha/4) rho^T L^{-1} rho - (3 xc/4) sum rho^{4/3} + tr(G_lin^T X),
//   L = Diag(L_1, ..., L_s), every L_j = tridiag(-1, 2, -1) on `block` rows (the last one on the
//   rows left; block = 0: one block of n rows), G = 2q L X + Diag(alpha y - 2 xc rho^{1/3}) X + G_lin.
// Inside a block of m rows the Dirichlet inverse is (L_j^{-1})_uv = min(u,v)(m+1-max(u,v))/(m+1)
// (1-based positions), so for blocks of at most kChainMaxBlock rows y = L^{-1} rho is a direct sum
// over the block in shared memory.  The grid is row tiles x column groups, sized to about eight
// CTAs per SM; when y is needed a tile holds whole blocks (kChainTile rows rounded down to a
// multiple of the block), so no CTA reads rho of rows outside its tile.
//   chain_density_kernel  the column group's share of rho_r = sum_c X_rc^2 (storage type, stored
//                         as double), for every row
//   chain_grad_kernel     rho (the groups' shares added in group order), y and the row scale of
//                         its tile; G of its tile and column group; its f partial
//                         -(alpha/4) rho^T y + (xc/4) sum rho^{4/3} (column group 0) + 1/2 <G_lin, X>,
//                         so that f = 1/2 <X, G> + (sum of the partials).

constexpr int kChainTile = 256;
constexpr int kChainCtasPerSm = 8;   // the row tiles x column groups aim at this many CTAs per SM

ChainPlan chain_plan(int64_t n, int p, int64_t block, bool need_y) {
  ChainPlan c;
  c.tile = (need_y && block > 0) ? (int)((kChainTile / block) * block) : kChainTile;
  c.ntiles = (int)((n + c.tile - 1) / c.tile);
  const int64_t target = (int64_t)kChainCtasPerSm * device_sm_count();
  const int64_t want = (target + (int64_t)c.ntiles - 1) / c.ntiles;
  const int ncg = (int)std::max<int64_t>(1, std::min<int64_t>(p, want));
  c.cw = (p + ncg - 1) / ncg;
  c.ncg = (p + c.cw - 1) / c.cw;
  return c;
}

template <typename T>
__global__ void __launch_bounds__(kChainTile)
chain_density_kernel(int64_t n, int p, int tile, int cw, const T* __restrict__ X, int64_t ldx,
                     double* __restrict__ rho_part, const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  const int t = threadIdx.x;
  const int64_t r = (int64_t)blockIdx.x * tile + t;
  if (t >= tile || r >= n) return;
  const int g = blockIdx.y;
  const int c0 = g * cw, c1 = min(p, c0 + cw);
  T s = T(0);
  for (int c = c0; c < c1; ++c) {
    const T x = X[r + (int64_t)c * ldx];
    s = fma(x, x, s);
  }
  rho_part[(int64_t)g * n + r] = (double)s;
}

template <typename T>
__global__ void __launch_bounds__(kChainTile)
chain_grad_kernel(int64_t n, int p, int64_t block, int tile, int cw, int ncg, double alpha,
                  double q, double xc, const T* __restrict__ X, int64_t ldx,
                  const T* __restrict__ lin, int64_t ldl, T* __restrict__ G, int64_t ldg,
                  const double* __restrict__ rho_part, double* __restrict__ fpart,
                  const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  __shared__ double rho_s[kChainTile];
  __shared__ double scratch[33];
  const int t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * tile;
  const int64_t r = r0 + t;
  const bool row = t < tile && r < n;
  const int g = blockIdx.y;
  double scale = 0.0, fr = 0.0;
  if (alpha != 0.0 || xc != 0.0) {          // the same for every thread of the launch
    double rv = 0.0;
    if (row)
      for (int gg = 0; gg < ncg; ++gg) rv += rho_part[(int64_t)gg * n + r];
    rho_s[t] = rv;
    __syncthreads();
    if (row) {
      double y = 0.0;
      if (alpha != 0.0) {
        // the block of row r lies inside this tile (the tile is a multiple of the block)
        const int64_t bs = (r / block) * block;
        const int m = (int)(min(n, bs + block) - bs);
        const int u = (int)(r - bs) + 1;
        const double* rb = rho_s + (bs - r0);
        double acc = 0.0;
        for (int v = 1; v <= m; ++v) {
          const int lo = min(u, v), hi = max(u, v);
          acc += (double)(lo * (m + 1 - hi)) * rb[v - 1];
        }
        y = acc / (double)(m + 1);
      }
      const double c3 = (xc != 0.0) ? cbrt(rv) : 0.0;
      scale = alpha * y - 2.0 * xc * c3;
      if (g == 0) fr = -0.25 * alpha * rv * y + 0.25 * xc * rv * c3;
    }
  }
  if (row) {
    const bool has_m = (block > 0) ? (r % block != 0) : (r > 0);
    const bool has_p = (r + 1 < n) && ((block > 0) ? ((r + 1) % block != 0) : true);
    const T ts = (T)scale;
    const T q2 = (T)(2.0 * q);
    const int c0 = g * cw, c1 = min(p, c0 + cw);
    T fl = T(0);
    for (int c = c0; c < c1; ++c) {
      const T* xcol = X + (int64_t)c * ldx;
      const T x = xcol[r];
      const T xm = has_m ? xcol[r - 1] : T(0);
      const T xp = has_p ? xcol[r + 1] : T(0);
      T gv = fma(q2, (x + x) - xm - xp, ts * x);
      if (lin != nullptr) {
        const T l = lin[r + (int64_t)c * ldl];
        gv += l;
        fl = fma(l, x, fl);
      }
      G[r + (int64_t)c * ldg] = gv;
    }
    fr += 0.5 * (double)fl;
  }
  const double fs = block_sum(fr, scratch);
  if (t == 0 && fpart != nullptr) fpart[(int64_t)blockIdx.x * ncg + g] = fs;
}

template <typename T>
cudaError_t launch_chain_grad(int64_t n, int p, int64_t block, double alpha, double q, double xc,
                              const T* X, int64_t ldx, const T* lin, int64_t ldl, T* G,
                              int64_t ldg, double* rho_part, double* fpart, const DevState* st,
                              cudaStream_t s, int* launches) {
  const ChainPlan c = chain_plan(n, p, block, alpha != 0.0);
  const dim3 grid((unsigned)c.ntiles, (unsigned)c.ncg);
  *launches = 0;
  if (alpha != 0.0 || xc != 0.0) {
    chain_density_kernel<T><<<grid, kChainTile, 0, s>>>(n, p, c.tile, c.cw, X, ldx, rho_part, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 1;
  }
  chain_grad_kernel<T><<<grid, kChainTile, 0, s>>>(n, p, block, c.tile, c.cw, c.ncg, alpha, q, xc,
                                                    X, ldx, lin, ldl, G, ldg, rho_part, fpart, st);
  *launches += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- 3D stencil

// One CTA of 32 x 8 threads owns a 32 (x) x 8 (y) tile of one column of X
// and marches through kStencilZ planes of z, keeping the planes z - 1, z and
// z + 1 of its point in registers; x neighbours come from the adjacent lanes
// of the warp (a warp is one x row), y neighbours through the L1 cache.  Each
// element of X is read once from DRAM and G is written once.
constexpr int kStencilZ = 16;

template <typename T>
__global__ void __launch_bounds__(256)
stencil_grad_kernel(int nx, int ny, int nz, int p, const T* __restrict__ V,
                    const T* __restrict__ X, int64_t ldx, T* __restrict__ G, int64_t ldg,
                    const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  const int nzb = (nz + kStencilZ - 1) / kStencilZ;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const bool in = x < nx && y < ny;
  const int sxy = nx * ny;
  for (int zc = blockIdx.z; zc < nzb * p; zc += gridDim.z) {
    const int c = zc / nzb;
    const int z0 = (zc - c * nzb) * kStencilZ;
    const int z1 = min(nz, z0 + kStencilZ);
    const T* xc = X + (int64_t)c * ldx;
    T* gc = G + (int64_t)c * ldg;
    int i = x + nx * (y + ny * z0);
    T prev = T(0), cur = T(0);
    if (in) {
      prev = z0 > 0 ? __ldg(xc + i - sxy) : T(0);
      cur = __ldg(xc + i);
    }
#pragma unroll 4
    for (int z = z0; z < z1; ++z, i += sxy) {
      T next = T(0), ym = T(0), yp = T(0), v = T(0);
      if (in) {
        if (z + 1 < nz) next = __ldg(xc + i + sxy);
        if (y > 0) ym = __ldg(xc + i - nx);
        if (y + 1 < ny) yp = __ldg(xc + i + nx);
        if (V) v = __ldg(V + i);
      }
      T xm = __shfl_up_sync(0xffffffffu, cur, 1);
      T xp = __shfl_down_sync(0xffffffffu, cur, 1);
      if (threadIdx.x == 0) xm = (in && x > 0) ? __ldg(xc + i - 1) : T(0);
      if (threadIdx.x == 31) xp = (in && x + 1 < nx) ? __ldg(xc + i + 1) : T(0);
      if (x + 1 >= nx) xp = T(0);
      if (in) {
        const T nb = ((((xm + xp) + ym) + yp) + prev) + next;
        gc[i] = fma(T(6) + v, cur, -nb);
      }
      prev = cur;
      cur = next;
    }
  }
}

// The same operator on 16-byte vectors (four floats or two doubles of
// consecutive x), for grids whose x extent is a multiple of the vector width
// and 16-byte-aligned columns.  A CTA of 256 threads owns 256 consecutive
// vectors of a plane (whole x rows when a row is at most 256 vectors) and
// marches through kStencilZ planes with z - 1, z, z + 1 in registers; the x
// neighbour of a vector's first and last element comes from the adjacent lane
// (or, at a warp edge inside a row, from memory), the y neighbours are vector
// loads that mostly hit L1.  One load instruction now serves four (two)
// points, which removes the instruction-issue limit of the scalar kernel.
template <typename T> struct StencilVec;
template <> struct StencilVec<float> {
  typedef float4 V;
  static constexpr int W = 4;
  __device__ static float first(const V& v) { return v.x; }
  __device__ static float last(const V& v) { return v.w; }
  __device__ static V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  // g = (6 + v) c - (xm + xp + ym + yp + zm + zp), neighbours summed in a fixed order
  __device__ static V apply(const V& c, const V& ym, const V& yp, const V& zm, const V& zp,
                            const V& v, float left, float right) {
    V g;
    g.x = fmaf(6.f + v.x, c.x, -(((((left + c.y) + ym.x) + yp.x) + zm.x) + zp.x));
    g.y = fmaf(6.f + v.y, c.y, -(((((c.x + c.z) + ym.y) + yp.y) + zm.y) + zp.y));
    g.z = fmaf(6.f + v.z, c.z, -(((((c.y + c.w) + ym.z) + yp.z) + zm.z) + zp.z));
    g.w = fmaf(6.f + v.w, c.w, -(((((c.z + right) + ym.w) + yp.w) + zm.w) + zp.w));
    return g;
  }
};
template <> struct StencilVec<double> {
  typedef double2 V;
  static constexpr int W = 2;
  __device__ static double first(const V& v) { return v.x; }
  __device__ static double last(const V& v) { return v.y; }
  __device__ static V zero() { return make_double2(0.0, 0.0); }
  __device__ static V apply(const V& c, const V& ym, const V& yp, const V& zm, const V& zp,
                            const V& v, double left, double right) {
    V g;
    g.x = fma(6.0 + v.x, c.x, -(((((left + c.y) + ym.x) + yp.x) + zm.x) + zp.x));
    g.y = fma(6.0 + v.y, c.y, -(((((c.x + right) + ym.y) + yp.y) + zm.y) + zp.y));
    return g;
  }
};

constexpr int kStencilVThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kStencilVThreads)
stencil_grad_vec_kernel(int nx, int ny, int nz, int p, const T* __restrict__ V,
                        const T* __restrict__ X, int64_t ldx, T* __restrict__ G, int64_t ldg,
                        const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  typedef StencilVec<T> SV;
  typedef typename SV::V Vt;
  constexpr int W = SV::W;
  const int nxv = nx / W;                       // vectors per x row
  const int64_t nvp = (int64_t)nxv * ny;        // vectors per plane
  const int nzb = (nz + kStencilZ - 1) / kStencilZ;
  const int64_t v = (int64_t)blockIdx.x * kStencilVThreads + threadIdx.x;
  const bool in = v < nvp;
  const int lane = threadIdx.x & 31;
  const int xv = in ? (int)(v % nxv) : 0;
  const int y = in ? (int)(v / nxv) : 0;
  const int64_t sxy = (int64_t)nx * ny;         // elements per plane
  for (int zc = blockIdx.y; zc < nzb * p; zc += gridDim.y) {
    const int c = zc / nzb;
    const int z0 = (zc - c * nzb) * kStencilZ;
    const int z1 = min(nz, z0 + kStencilZ);
    const T* xc = X + (int64_t)c * ldx;
    T* gc = G + (int64_t)c * ldg;
    int64_t i = (int64_t)xv * W + (int64_t)nx * y + sxy * z0;   // first element of the vector
    Vt prev = SV::zero(), cur = SV::zero();
    if (in) {
      if (z0 > 0) prev = __ldg(reinterpret_cast<const Vt*>(xc + i - sxy));
      cur = __ldg(reinterpret_cast<const Vt*>(xc + i));
    }
    for (int z = z0; z < z1; ++z, i += sxy) {
      Vt next = SV::zero(), ym = SV::zero(), yp = SV::zero(), vv = SV::zero();
      if (in) {
        if (z + 1 < nz) next = __ldg(reinterpret_cast<const Vt*>(xc + i + sxy));
        if (y > 0) ym = __ldg(reinterpret_cast<const Vt*>(xc + i - nx));
        if (y + 1 < ny) yp = __ldg(reinterpret_cast<const Vt*>(xc + i + nx));
        if (V) vv = __ldg(reinterpret_cast<const Vt*>(V + i));
      }
      T left = __shfl_up_sync(0xffffffffu, SV::last(cur), 1);
      T right = __shfl_down_sync(0xffffffffu, SV::first(cur), 1);
      if (in) {
        if (xv == 0) left = T(0);
        else if (lane == 0) left = __ldg(xc + i - 1);
        if (xv == nxv - 1) right = T(0);
        else if (lane == 31) right = __ldg(xc + i + W);
        *reinterpret_cast<Vt*>(gc + i) = SV::apply(cur, ym, yp, prev, next, vv, left, right);
      }
      prev = cur;
      cur = next;
    }
  }
}

// ---------------------------------------------------------------- launchers

// Y = X Bm: an n x p times p x p product (Bm column-major, leading dimension ldb), 64 x 64
// output tiles over shared-memory stages of X and Bm.  Problem 4's gradient A X B is the
// dense kernel's A X followed by this.
template <typename T>
__global__ void __launch_bounds__(kThreads)
right_multiply_kernel(int64_t n, int p, const T* __restrict__ X, int64_t ldx,
                      const T* __restrict__ Bm, int64_t ldb, T* __restrict__ Y, int64_t ldy,
                      const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  constexpr int KS = sizeof(T) == 8 ? 16 : kKStep;
  __shared__ T Xs[KS][kTile];        // X(r0 + r, k0 + q) at Xs[q][r]
  __shared__ T Bs[kTile][KS + 1];    // Bm(k0 + q, c0 + c) at Bs[c][q]
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int c0 = blockIdx.y * kTile;
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  for (int k0 = 0; k0 < p; k0 += KS) {
    {
      const int r = t & (kTile - 1);
      const int64_t row = r0 + r;
#pragma unroll
      for (int s = 0; s < KS / 4; ++s) {
        const int q = (t >> 6) + 4 * s;
        const int col = k0 + q;
        Xs[q][r] = (row < n && col < p) ? X[row + (int64_t)col * ldx] : T(0);
      }
    }
    {
      const int q = t & (KS - 1);
      const int kr = k0 + q;
#pragma unroll
      for (int s = 0; s < kTile * KS / kThreads; ++s) {
        const int c = t / KS + (kThreads / KS) * s;
        const int cc = c0 + c;
        Bs[c][q] = (kr < p && cc < p) ? Bm[kr + (int64_t)cc * ldb] : T(0);
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < KS; ++q) {
      T xa[4], bb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xa[u] = Xs[q][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) bb[v] = Bs[ty + 16 * v][q];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(xa[u], bb[v], acc[u][v]);
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
      if (r < n) Y[r + (int64_t)c * ldy] = acc[u][v];
    }
  }
}

template <typename T>
cudaError_t launch_right_multiply(int64_t n, int p, const T* X, int64_t ldx, const T* Bm,
                                  int64_t ldb, T* Y, int64_t ldy, const DevState* st,
                                  cudaStream_t s) {
  dim3 grid((unsigned)((n + kTile - 1) / kTile), (p + kTile - 1) / kTile);
  right_multiply_kernel<T><<<grid, kThreads, 0, s>>>(n, p, X, ldx, Bm, ldb, Y, ldy, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dense_grad(int64_t n, int p, const T* A, int64_t lda, const T* X, int64_t ldx,
                              T* G, int64_t ldg, const DevState* st, cudaStream_t s) {
  dim3 grid((unsigned)((n + kTile - 1) / kTile), (p + kTile - 1) / kTile);
  dense_grad_kernel<T><<<grid, kThreads, 0, s>>>(n, p, A, lda, X, ldx, G, ldg, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hartree_grad(int64_t n, int p, double alpha, double q, double xc, const T* X,
                                int64_t ldx, T* G, int64_t ldg, double* rho, double* blk, double* y,
                                double* fpart, const DevState* st, cudaStream_t s) {
  const int nb = hartree_blocks(n);
  hartree_density_kernel<T><<<nb, kHB, 0, s>>>(n, p, X, ldx, rho, blk, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hartree_grad_kernel<T><<<nb, kHB, 0, s>>>(n, p, alpha, q, xc, 1.0 / (double)(n + 1), X, ldx, G,
                                             ldg, rho, blk, y, fpart, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stencil_grad(int nx, int ny, int nz, int p, const T* V, const T* X, int64_t ldx,
                                T* G, int64_t ldg, const DevState* st, cudaStream_t s) {
  const int nzb = (nz + kStencilZ - 1) / kStencilZ;
  int64_t gz = (int64_t)nzb * p;
  if (gz > 65535) gz = 65535;
  constexpr int W = StencilVec<T>::W;
  const bool vec = nx % W == 0 && ldx % W == 0 && ldg % W == 0 && ((uintptr_t)X % 16) == 0 &&
                   ((uintptr_t)G % 16) == 0 && (V == nullptr || ((uintptr_t)V % 16) == 0);
  if (vec) {
    const int64_t nvp = (int64_t)(nx / W) * ny;
    dim3 grid((unsigned)((nvp + kStencilVThreads - 1) / kStencilVThreads), (unsigned)gz);
    stencil_grad_vec_kernel<T><<<grid, kStencilVThreads, 0, s>>>(nx, ny, nz, p, V, X, ldx, G, ldg,
                                                                 st);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8), (unsigned)gz);
  stencil_grad_kernel<T><<<grid, dim3(32, 8), 0, s>>>(nx, ny, nz, p, V, X, ldx, G, ldg, st);
  return cudaGetLastError();
}

cudaError_t preload_objective_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dense_grad_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dense_grad_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, right_multiply_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, right_multiply_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, hartree_density_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, hartree_density_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, hartree_grad_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, hartree_grad_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, chain_density_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, chain_density_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, chain_grad_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, chain_grad_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stencil_grad_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stencil_grad_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stencil_grad_vec_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stencil_grad_vec_kernel<double>);
  return e;
}

#define PLAM_INST(T)                                                                              \
  template cudaError_t launch_dense_grad<T>(int64_t, int, const T*, int64_t, const T*, int64_t,   \
                                            T*, int64_t, const DevState*, cudaStream_t);          \
  template cudaError_t launch_right_multiply<T>(int64_t, int, const T*, int64_t, const T*,       \
                                                int64_t, T*, int64_t, const DevState*,            \
                                                cudaStream_t);                                    \
  template cudaError_t launch_hartree_grad<T>(int64_t, int, double, double, double, const T*, int64_t, \
                                              T*, int64_t, double*, double*, double*, double*,    \
                                              const DevState*, cudaStream_t);                     \
  template cudaError_t launch_chain_grad<T>(int64_t, int, int64_t, double, double, double, const T*, \
                                            int64_t, const T*, int64_t, T*, int64_t, double*,     \
                                            double*, const DevState*, cudaStream_t, int*);       \
  template cudaError_t launch_stencil_grad<T>(int, int, int, int, const T*, const T*, int64_t, T*, \
                                              int64_t, const DevState*, cudaStream_t);
PLAM_INST(float)
PLAM_INST(double)
#undef PLAM_INST

}  // namespace plam
