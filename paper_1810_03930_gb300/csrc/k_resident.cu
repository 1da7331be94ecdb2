// Resident PCAL / PLAM solve for problems whose iterate fits in the shared
// memory of the GPU's SMs (FP32 storage, p <= 64, the 1D Hartree and dense
// trace objectives).
//
// One cooperative launch runs the whole loop of Algorithm 2 / 3.  CTA b (one
// per SM) owns rows [b*rows, b*rows + nr) and keeps X, G (overwritten by R)
// and the previous R of those rows in shared memory for the entire solve.
// Per iteration only small data crosses CTAs, through L2:
//   P1  rho_r = ||X_r||^2 and the block sums of i rho_i, (n+1-i) rho_i
//       (Hartree), the halo rows, or the rows of X (dense)      -> barrier 1
//   P2  gradient G of the own rows (Hartree: Green's-function prefix sums over
//       the preceding / following CTAs and a block scan; dense: A[rows,:] X),
//       then the partial Grams X^T [X | G] of the own rows   -> barrier 2
//   P3  CTA b sums its share of the 2p^2 entries over all CTAs, in CTA order
//                                                             -> barrier 3
//   P4  every CTA reads the reduced Grams and forms Psi(C), d (eq. lambda2)
//       and M = Lambda - beta (B - I) (eq. S1); R = G - X M and
//       K = G - X Psi(C) for its rows, with the column dots  -> barrier 4
//   P5  CTA b sums its share of the dot slots over all CTAs  -> barrier 5;
//       every CTA reads the sums and takes the same decisions (KKT test,
//       eta by Section 5.1, PCAL column norms), then updates its rows of X.
// All cross-CTA sums are in a fixed order, and every CTA computes the
// scalars from the same sums with the same code, so the run is bitwise
// reproducible and needs no broadcast.  Data written by other CTAs is read
// with ld.global.cg (L2), never through the non-coherent L1.
//
// The grid barrier is an arrival counter plus a generation word.  Its wait is
// bounded (kBarrierSpins polls with __nanosleep): on expiry the CTA raises a
// global error flag and every CTA leaves the loop at its next check, so the
// kernel always terminates; the host reports PLAM_ERR_TIMEOUT.
#include "plam_device.cuh"

namespace plam {

constexpr int kResThreads = 512;
constexpr int kObjHartree = 1;   // the C ABI's PLAM_OBJ_HARTREE1D
constexpr int kResMaxP = 64;
constexpr long long kBarrierSpins = 1ll << 24;   // ~1 s: 4096 busy polls, then ~64 ns per poll

struct ResidentArgs {
  int64_t n;
  int p, nblk, rows, rp;
  int kind;                   // PLAM_OBJ_DENSE (0) or PLAM_OBJ_HARTREE1D (1)
  const float* A;
  int64_t lda;
  double alpha, q, inv_np1;
  float* X;
  int64_t ldx;
  float* R0;
  float* R1;
  int64_t ldr;
  float* halo;                // nblk x 2 x p
  double* blk;                // nblk x 2
  float* part;                // nblk x 2p^2
  float* red;                 // 2p^2
  float* dots;                // nblk x (3p + 7)
  double* dred;               // 3p + 7
  unsigned int* bar;          // [arrivals, generation]
  unsigned int bar_expect;    // arrivals that release a barrier (nblk)
  int* err;
  DevState* st;
  double* nubuf;
  float* coef;
  double* hist;
  IterParams prm;
};

__device__ inline float ldcg_f(const float* p) { return __ldcg(p); }
__device__ inline double ldcg_d(const double* p) { return __ldcg(p); }

__device__ __forceinline__ void red_add_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier with a bounded wait.  bar[0] counts arrivals over the
// whole launch (zeroed before it); barrier number g releases when the count
// reaches (g + 1) * expect, and every CTA polls the count directly.  The CTA's
// writes are ordered before thread 0's arrival by the block barrier and
// published by the arrival's release semantics; the polling load acquires
// the other CTAs' writes, and the closing block barrier passes them on to the
// CTA's threads (no full fences).  Returns false when the wait expired here
// or the error flag is already raised.
__device__ bool grid_barrier(unsigned int* bar, unsigned int expect, unsigned int& gen, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int target = (gen + 1u) * expect;
    red_add_release_gpu(&bar[0], 1u);
    long long spins = 0;
    while (ld_acquire_gpu(bar) < target) {
      if (++spins > kBarrierSpins) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
      if (spins > 4096) __nanosleep(64);   // busy-poll first, then back off
    }
    gen = gen + 1u;
    if (ok && *(volatile int*)err != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// Six float sums over the block at once (fixed butterfly, warps in order);
// the results are left in out[0..5] for every thread.
__device__ inline void block_sum6_f(float v[6], float* scratch /* >= 16*6 */, float* out) {
#pragma unroll
  for (int d = 0; d < 6; ++d)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[d] += __shfl_xor_sync(0xffffffffu, v[d], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int d = 0; d < 6; ++d) scratch[d * 16 + w] = v[d];
  __syncthreads();
  if (threadIdx.x < 6) {
    float s = 0.f;
    for (int i = 0; i < 16; ++i) s += scratch[threadIdx.x * 16 + i];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Deterministic block-wide float sum (fixed butterfly, warps in order).  The
// resident kernel keeps double arithmetic to a few scalars per iteration:
// GB300 runs FP64 at 1/64 of the FP32 rate, so a double block sum over 512
// threads alone costs ~1 us.
__device__ inline float block_sum_f(float v, float* scratch /* >= 17 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < kResThreads / 32; ++i) s += scratch[i];
    scratch[16] = s;
  }
  __syncthreads();
  return scratch[16];
}

// Two block_sum_f at once: each value is summed in exactly the order block_sum_f
// uses (butterfly in the warp, then the 16 warp sums in order by one thread),
// with one set of block barriers for both.
__device__ inline void block_sum2_f(float& v0, float& v1, float* scratch /* >= 34 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    scratch[w] = v0;
    scratch[17 + w] = v1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const float* src = scratch + 17 * threadIdx.x;
    float s = 0.f;
    for (int i = 0; i < kResThreads / 32; ++i) s += src[i];
    scratch[16 + 17 * threadIdx.x] = s;
  }
  __syncthreads();
  v0 = scratch[16];
  v1 = scratch[33];
}

// Deterministic block-wide inclusive scan of two floats (blockDim = kResThreads).
__device__ inline void block_scan2(float& a, float& c, float* sh /* 2 x 16 */, float& tot_a,
                                   float& tot_c) {
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float ta = __shfl_up_sync(0xffffffffu, a, o);
    const float tc = __shfl_up_sync(0xffffffffu, c, o);
    if (l >= o) { a += ta; c += tc; }
  }
  __syncthreads();
  if (l == 31) { sh[w] = a; sh[16 + w] = c; }
  __syncthreads();
  float wa = 0.f, wc = 0.f, ta = 0.f, tc = 0.f;
  for (int j = 0; j < kResThreads / 32; ++j) {
    if (j < w) { wa += sh[j]; wc += sh[16 + j]; }
    ta += sh[j];
    tc += sh[16 + j];
  }
  a += wa;
  c += wc;
  tot_a = ta;
  tot_c = tc;
}

__global__ void __launch_bounds__(kResThreads, 1) resident_solve_kernel(ResidentArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = a.p, rp = a.rp, b = blockIdx.x, t = threadIdx.x;
  const int64_t n = a.n;
  const int64_t r0 = (int64_t)b * a.rows;
  const int nr = (int)min((int64_t)a.rows, n - r0);
  const int E = 2 * p * p;
  const int S = 3 * p + 7;
  const IterParams& prm = a.prm;

  float* Xs = reinterpret_cast<float*>(smem_raw);   // p x rp, column c at Xs + c*rp
  float* GR = Xs + p * rp;                           // G, then R of this iteration
  float* RP = GR + p * rp;                           // R of the previous iteration
  const int pp = (p + 3) & ~3;                       // padded row stride of M and Psi(C)
  float* Ms = RP + p * rp;                           // M, Ms[k*pp + c]
  float* Ls = Ms + p * pp;                           // Psi(C), Ls[k*pp + c]
  float* Ws = Ls + p * pp;                           // reduced Grams [B | C], 2p^2
  float* zrow = Ws + ((E + 3) & ~3);                 // rp zeros (padding operand), 16-byte aligned
  float* inu = zrow + rp;                            // 1/nu_c of the latest update
  float* omn = inu + kResMaxP;                       // 1 - nu_c of the latest update
  float* colsum = omn + kResMaxP;                    // 3 x chunks x p column-dot partials (<= 3 x 512)
  float* grp = colsum + 3 * kResThreads;             // kResThreads reduction scratch
  double* dsh = reinterpret_cast<double*>(grp + kResThreads);   // 64 scratch doubles
  double* rho = dsh + 64;                            // rp
  double* dsum = rho + rp;                           // S reduced dot sums

  __shared__ double scratch[33];
  __shared__ float fscr[40];
  __shared__ float scr6[96];
  __shared__ float tot6[6];
  __shared__ float halo_s[2 * kResMaxP];
  __shared__ double sc[8];
  __shared__ int bad;

  // ---- load the own rows of X; zero the padding rows of every buffer
  for (int e = t; e < p * rp; e += kResThreads) {
    const int c = e / rp, r = e % rp;
    Xs[e] = (r < nr) ? a.X[r0 + r + (int64_t)c * a.ldx] : 0.f;
    GR[e] = 0.f;
    RP[e] = 0.f;
  }
  for (int r = t; r < rp; r += kResThreads) zrow[r] = 0.f;
  __syncthreads();

  unsigned int gen = 0;
  int k = 0;
  double K0 = 0.0, eta0 = 0.0, eta = 0.0, eta_prev = 0.0;
  float inv_etap = 0.f;
  int nrec = 0;
  int stop = kRunning;
  double last_kkt = 0.0, last_feas = 0.0, last_f = 0.0, last_ss = 0.0, last_sy = 0.0, last_yy = 0.0;
  const float beta = (float)prm.beta;
  float* gr = GR;
  float* rpv = RP;

  for (;;) {
    // ================= P1: density, block sums, halos / rows of X
    float s1 = 0.f, s2 = 0.f;
    if (t < nr) {
      float s = 0.f;
      for (int c = 0; c < p; ++c) {
        const float x = Xs[c * rp + t];
        s = fmaf(x, x, s);
      }
      rho[t] = (double)s;
      const int64_t gi = r0 + t;
      s1 = (float)(gi + 1) * s;
      s2 = (float)(n - gi) * s;
    }
    if (a.kind == kObjHartree) {
      block_sum2_f(s1, s2, fscr);
      const double S1 = (double)s1;
      const double S2 = (double)s2;
      if (t == 0) {
        a.blk[2 * b] = S1;
        a.blk[2 * b + 1] = S2;
      }
      if (t < p) {
        a.halo[(size_t)b * 2 * p + t] = Xs[t * rp];
        a.halo[(size_t)b * 2 * p + p + t] = Xs[t * rp + nr - 1];
      }
    } else {
      for (int e = t; e < p * nr; e += kResThreads) {
        const int c = e / nr, r = e % nr;
        a.X[r0 + r + (int64_t)c * a.ldx] = Xs[c * rp + r];
      }
    }
    if (!grid_barrier(a.bar, a.bar_expect, gen, a.err)) break;

    // ================= P2: gradient of the own rows, partial Grams
    float fy = 0.f;
    if (a.kind == kObjHartree) {
      // the neighbours' boundary rows do not depend on the block sums: load them first,
      // so that their L2 round trip overlaps the one of the block sums
      float hv = 0.f;
      if (t < p) hv = (b > 0) ? ldcg_f(a.halo + (size_t)(b - 1) * 2 * p + p + t) : 0.f;
      else if (t < 2 * p) hv = (r0 + nr < n) ? ldcg_f(a.halo + (size_t)(b + 1) * 2 * p + t - p) : 0.f;
      float pa = 0.f, qa = 0.f;
      for (int j = t; j < a.nblk; j += kResThreads) {
        if (j < b) pa += (float)ldcg_d(a.blk + 2 * j);
        if (j > b) qa += (float)ldcg_d(a.blk + 2 * j + 1);
      }
      block_sum2_f(pa, qa, fscr);
      const float Pbefore = pa;
      const float Qafter = qa;
      const int64_t gi = r0 + t;
      const float rv = (t < nr) ? (float)rho[t] : 0.f;
      float ia = (t < nr) ? (float)(gi + 1) * rv : 0.f;
      float ic = (t < nr) ? (float)(n - gi) * rv : 0.f;
      float tot_a, tot_c;
      block_scan2(ia, ic, reinterpret_cast<float*>(dsh), tot_a, tot_c);
      const float P = Pbefore + ia;
      const float Q = Qafter + (tot_c - ic);
      const float y = ((float)(n - gi) * P + (float)(gi + 1) * Q) * (float)a.inv_np1;
      fy = block_sum_f((t < nr) ? rv * y : 0.f, fscr);
      // neighbours' boundary rows; alpha y of each row for all threads
      if (t < 2 * p) halo_s[t] = hv;
      if (t < nr) grp[t] = (float)a.alpha * y;
      __syncthreads();
      {
        // row r = t mod nr, columns g, g + ng, ... for the ng = 512 / nr groups of rows
        const int ng = kResThreads / nr;
        const int g = t / nr, r = t - g * nr;
        if (g < ng) {
          const float ty = grp[r];
          const float q2 = (float)(2.0 * a.q);
          const bool first = (r == 0), last = (r == nr - 1);
          for (int c = g; c < p; c += ng) {
            const float x = Xs[c * rp + r];
            const float xm = first ? halo_s[c] : Xs[c * rp + r - 1];
            const float xp = last ? halo_s[p + c] : Xs[c * rp + r + 1];
            gr[c * rp + r] = fmaf(q2, (x + x) - xm - xp, ty * x);
          }
        }
      }
    } else {
      // G = A X for the own rows (A symmetric: row r of A is column r)
      for (int e = t; e < p * nr; e += kResThreads) {
        const int c = e / nr, r = e % nr;
        const float* arow = a.A + (r0 + r) * a.lda;
        const float* xc = a.X + (int64_t)c * a.ldx;
        float acc = 0.f;
        for (int64_t j = 0; j < n; ++j) acc = fmaf(arow[j], ldcg_f(xc + j), acc);
        gr[c * rp + r] = acc;
      }
    }
    __syncthreads();
    {
      // X^T [X | G] over the own rows.  Tiles of 4 i x 4 j outputs, 4 rows per
      // step.  The four i of a tile are strided (ib, ib + nib, ...), so the
      // lanes of a warp (consecutive ib) read consecutive columns of X and hit
      // distinct shared-memory banks; the j of a tile are consecutive and
      // shared by neighbouring lanes (broadcast).
      const int nib = (p + 3) / 4, njb = (2 * p + 3) / 4;
      const int rows4 = (nr + 3) & ~3;
      for (int tile = t; tile < nib * njb; tile += kResThreads) {
        const int ib = tile % nib, jb = tile / nib;
        const float* ap[4];
        const float* bp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = ib + u * nib;
          ap[u] = (i < p) ? Xs + i * rp : zrow;
          const int j = 4 * jb + u;
          bp[u] = (j < p) ? Xs + j * rp : (j < 2 * p) ? gr + (j - p) * rp : zrow;
        }
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        for (int r = 0; r < rows4; r += 4) {
          float4 av[4], bv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            av[u] = *reinterpret_cast<const float4*>(ap[u] + r);
            bv[u] = *reinterpret_cast<const float4*>(bp[u] + r);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              acc[u][v] = fmaf(av[u].x, bv[v].x, acc[u][v]);
              acc[u][v] = fmaf(av[u].y, bv[v].y, acc[u][v]);
              acc[u][v] = fmaf(av[u].z, bv[v].z, acc[u][v]);
              acc[u][v] = fmaf(av[u].w, bv[v].w, acc[u][v]);
            }
        }
        float* out = a.part + (size_t)b * E;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = ib + u * nib;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int j = 4 * jb + v;
            if (i < p && j < 2 * p) out[(size_t)j * p + i] = acc[u][v];
          }
        }
      }
    }
    if (!grid_barrier(a.bar, a.bar_expect, gen, a.err)) break;

    // ================= P3: reduce this CTA's share of the Gram entries over all CTAs
    {
      const int epb = (E + a.nblk - 1) / a.nblk;
      const int e0 = b * epb;
      const int ne = max(0, min(epb, E - e0));
      if (ne > 0) {
        const int ng = kResThreads / ne;
        const int le = t % ne, g = t / ne;
        float v = 0.f;
        if (g < ng) {
          constexpr int kBatch = 8;
          for (int c0 = g; c0 < a.nblk; c0 += kBatch * ng) {
            float buf[kBatch];
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
              const int c = c0 + q * ng;
              buf[q] = (c < a.nblk) ? ldcg_f(a.part + (size_t)c * E + e0 + le) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < kBatch; ++q) v += buf[q];
          }
        }
        grp[t] = v;
        __syncthreads();
        if (t < ne) {
          float s = 0.f;
          for (int gg = 0; gg < ng; ++gg) s += grp[gg * ne + t];
          a.red[e0 + t] = s;
        }
      }
    }
    if (!grid_barrier(a.bar, a.bar_expect, gen, a.err)) break;

    // ================= P4: multiplier, update matrix, R and K of the own rows, dots
    for (int e = 4 * t; e < E; e += 4 * kResThreads) {
      if (e + 3 < E) {
        const float4 v4 = __ldcg(reinterpret_cast<const float4*>(a.red + e));
        Ws[e] = v4.x; Ws[e + 1] = v4.y; Ws[e + 2] = v4.z; Ws[e + 3] = v4.w;
      } else {
        for (int q = e; q < E; ++q) Ws[q] = ldcg_f(a.red + q);
      }
    }
    __syncthreads();
    // Ws[j*p + i]: B_ij for j < p, C_i(j-p) for j >= p
    for (int e = t; e < p * pp; e += kResThreads) {
      const int i = e / pp, j = e % pp;
      Ls[e] = (j < p) ? 0.5f * (Ws[(p + j) * p + i] + Ws[(p + i) * p + j]) : 0.f;
    }
    // (the block barriers inside block_sum_f below also order these writes of Ls
    // before the reads of the d loop)
#define BU(i, j) Ws[(size_t)(j) * p + (i)]
    double feas2 = 0.0;
    {
      float fr = 0.f;
      for (int e = t; e < p * p; e += kResThreads) {
        const int i = e % p, j = e / p;
        const float d = BU(i, j) - (i == j ? 1.f : 0.f);
        fr = fmaf(d, d, fr);
      }
      feas2 = (double)block_sum_f(fr, fscr);
    }
    if (t < p) {
      // d_i = C_ii - sum_k B_ik Psi_ki + beta (sum_k B_ik^2 - B_ii) (eq. lambda2)
      const int i = t;
      float s1f = 0.f, s2f = 0.f;
      for (int kk2 = 0; kk2 < p; ++kk2) {
        const float bik = BU(i, kk2);
        s1f = fmaf(bik, Ls[kk2 * pp + i], s1f);   // Psi(C) is symmetric: read along the lanes
        s2f = fmaf(bik, bik, s2f);
      }
      const float d = prm.lambda2 ? (Ws[(p + i) * p + i] - s1f + beta * (s2f - BU(i, i))) : 0.f;
      grp[i] = d;
    }
    __syncthreads();
    for (int e = t; e < p * pp; e += kResThreads) {
      const int kk2 = e / pp, c = e % pp;
      const float delta = (kk2 == c) ? 1.f : 0.f;
      Ms[e] = (c < p) ? Ls[e] + delta * grp[kk2] - beta * (BU(kk2, c) - delta) : 0.f;
    }
#undef BU
    __syncthreads();
    float ss = 0.f, sy = 0.f, yy = 0.f, kk = 0.f, gg = 0.f, xg = 0.f;
    {
      // one 4-row x 4-column micro-tile of R = G - X M and K = G - X Psi(C) per thread
      const int nrb = (nr + 3) / 4, ncb = (p + 3) / 4;
      for (int tile = t; tile < nrb * ncb; tile += kResThreads) {
        const int rb = tile % nrb, cb = tile / nrb;
        float a1[4][4], a2[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) { a1[u][v] = 0.f; a2[u][v] = 0.f; }
        for (int kk2 = 0; kk2 < p; ++kk2) {
          const float4 xv = *reinterpret_cast<const float4*>(Xs + kk2 * rp + 4 * rb);
          const float4 mv = *reinterpret_cast<const float4*>(Ms + kk2 * pp + 4 * cb);
          const float4 lv = *reinterpret_cast<const float4*>(Ls + kk2 * pp + 4 * cb);
          const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
          const float ma[4] = {mv.x, mv.y, mv.z, mv.w};
          const float la[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
          for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              a1[u][v] = fmaf(xa[u], ma[v], a1[u][v]);
              a2[u][v] = fmaf(xa[u], la[v], a2[u][v]);
            }
        }
        // the tile's four rows of a column are one 16-byte vector (rp is a multiple
        // of 4), so consecutive lanes touch consecutive vectors: no bank conflicts
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = 4 * cb + v;
          if (c >= p) continue;
          const int o = c * rp + 4 * rb;
          const float4 g4 = *reinterpret_cast<const float4*>(gr + o);
          const float4 x4 = *reinterpret_cast<const float4*>(Xs + o);
          const float4 p4 = (k > 0) ? *reinterpret_cast<const float4*>(rpv + o)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
          const float ga[4] = {g4.x, g4.y, g4.z, g4.w};
          const float xa2[4] = {x4.x, x4.y, x4.z, x4.w};
          const float pa[4] = {p4.x, p4.y, p4.z, p4.w};
          float rva[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = 4 * rb + u;
            rva[u] = ga[u];
            if (r >= nr) continue;
            const float g = ga[u];
            const float x = xa2[u];
            const float rv = g - a1[u][v];
            const float kv = g - a2[u][v];
            rva[u] = rv;
            kk = fmaf(kv, kv, kk);
            gg = fmaf(g, g, gg);
            xg = fmaf(x, g, xg);
            if (k > 0) {
              const float rpe = pa[u];
              const float sv = omn[c] * x - rpe * inv_etap;
              const float yv = rv - rpe;
              ss = fmaf(sv, sv, ss);
              sy = fmaf(sv, yv, sy);
              yy = fmaf(yv, yv, yy);
            }
          }
          *reinterpret_cast<float4*>(gr + o) = make_float4(rva[0], rva[1], rva[2], rva[3]);
        }
      }
      __syncthreads();
      // per-column ||X_c||^2, <X_c,R_c>, ||R_c||^2: each column split into row
      // chunks (coalesced shared-memory walks), chunks added in order
      const int chunks = kResThreads / p;
      const int rpc = (nr + chunks - 1) / chunks;
      if (t < chunks * p) {
        // chunk index fastest across the lanes: their rows are rpc apart, which
        // spreads a warp's loads over the banks better than columns rp apart
        const int c = t / chunks, ch = t % chunks;
        const int ra = ch * rpc, rb2 = min(nr, ra + rpc);
        float sx = 0.f, sxr = 0.f, sr = 0.f;
        for (int r = ra; r < rb2; ++r) {
          const float x = Xs[c * rp + r], rv = gr[c * rp + r];
          sx = fmaf(x, x, sx);
          sxr = fmaf(x, rv, sxr);
          sr = fmaf(rv, rv, sr);
        }
        colsum[(0 * chunks + ch) * p + c] = sx;
        colsum[(1 * chunks + ch) * p + c] = sxr;
        colsum[(2 * chunks + ch) * p + c] = sr;
      }
      __syncthreads();
      float* dp = a.dots + (size_t)b * S;
      if (t < 3 * p) {
        const int d = t / p, c = t % p;
        float s = 0.f;
        for (int ch = 0; ch < chunks; ++ch) s += colsum[(d * chunks + ch) * p + c];
        dp[d * p + c] = s;
      }
      float v6[6] = {ss, sy, yy, kk, gg, xg};
      block_sum6_f(v6, scr6, tot6);
      if (t < 6) dp[3 * p + t] = tot6[t];
      if (t == 0) dp[3 * p + 6] = fy;
    }
    if (!grid_barrier(a.bar, a.bar_expect, gen, a.err)) break;

    // ================= P5: reduce this CTA's dot slots over all CTAs (one warp per slot)
    {
      const int w = t >> 5, l = t & 31;
      for (int sidx = b + w * a.nblk; sidx < S; sidx += a.nblk * (kResThreads / 32)) {
        double v = 0.0;
        for (int c = l; c < a.nblk; c += 32) v += (double)ldcg_f(a.dots + (size_t)c * S + sidx);
        v = warp_sum_d(v);
        if (l == 0) a.dred[sidx] = v;
      }
    }
    if (!grid_barrier(a.bar, a.bar_expect, gen, a.err)) break;

    for (int e = t; e < S; e += kResThreads) dsum[e] = ldcg_d(a.dred + e);
    if (t == 0) bad = 0;
    __syncthreads();
    {
      // every CTA takes the same decisions from the same sums
      if (t == 0) {
        const double* tot = dsum + 3 * p;
        const double ssd = tot[0], syd = tot[1], yyd = tot[2], kkd = tot[3], ggd = tot[4], xgd = tot[5];
        if (k == 0) {
          double xx_all = 0.0;
          for (int c = 0; c < p; ++c) xx_all += dsum[c];
          K0 = sqrt(kkd);
          eta0 = (prm.eta0_user > 0.0) ? prm.eta0_user
                                        : ((xx_all > 0.0 ? sqrt(ggd / xx_all) : 1.0) + prm.beta);
          eta = eta0;
        }
        const double kkt = (K0 > 0.0) ? sqrt(kkd) / K0 : 0.0;
        const double f = prm.f_xg * xgd + prm.f_part * tot[6];
        const double feas = sqrt(feas2);
        last_kkt = kkt; last_feas = feas; last_f = f; last_ss = ssd; last_sy = syd; last_yy = yyd;
        if (b == 0 && nrec < prm.hist_cap) {
          double* h = a.hist + (size_t)nrec * 5;
          h[0] = (double)k; h[1] = f; h[2] = kkt; h[3] = feas; h[4] = nan("");
        }
        nrec = min(nrec + 1, prm.hist_cap);
        int s = kRunning;
        double e2 = eta;
        if (!isfinite(kkt) || !isfinite(feas) || (prm.feas_max > 0.0 && feas > prm.feas_max))
          s = kDiverged;
        else if (K0 == 0.0 || kkt < prm.tol) s = kConverged;
        else if (k >= prm.maxit) s = kMaxit;
        else {
          if (prm.eta_rule == 3) e2 = (prm.gamma > 0.0) ? prm.gamma : eta0;
          else if (k == 0) e2 = eta0;
          else if (prm.eta_rule == 4) e2 = (ssd > 0.0 && yyd > 0.0) ? sqrt(yyd / ssd) : eta;
          else if (ssd == 0.0 || syd == 0.0) e2 = eta;
          else {
            const double bb1 = fabs(syd) / ssd, bb2 = yyd / fabs(syd);
            e2 = (prm.eta_rule == 1) ? bb1 : (prm.eta_rule == 2) ? bb2 : ((k & 1) ? bb1 : bb2);
          }
          if (!isfinite(e2)) s = kDiverged;
          else e2 = eta_clamp(e2, eta0, prm.eta_min, prm.eta_max);
        }
        sc[0] = e2;
        sc[1] = (double)s;
        sc[2] = 1.0 / e2;
      }
      __syncthreads();
      const double e2 = sc[0];
      stop = (int)sc[1];
      const double ie = sc[2];
      if (stop == kRunning && t < p) {
        // ||X_c - R_c/eta||^2 formed in double from the double sums, then the
        // column scale in float (FP32 mode: the iterate is float)
        const float q = (float)(dsum[t] - 2.0 * dsum[p + t] * ie + dsum[2 * p + t] * ie * ie);
        float v = 1.f;
        if (prm.variant == 1) {
          v = sqrtf(q);
          if (!(v > 0.f) || !isfinite(v)) bad = 1;
        } else if (!isfinite(q)) {
          bad = 1;
        }
        inu[t] = 1.f / v;
        omn[t] = 1.f - v;
        if (b == 0) {
          a.nubuf[(size_t)(k & 1) * p + t] = v;
          a.coef[(size_t)(k & 1) * (2 * p + 1) + 1 + t] = 1.f / v;
          a.coef[(size_t)(k & 1) * (2 * p + 1) + 1 + p + t] = (float)(1.0 - v);
        }
      }
      __syncthreads();
      if (stop == kRunning && bad) stop = kDiverged;
      if (stop != kRunning) break;
      if (b == 0 && t == 0) {
        a.coef[(size_t)(k & 1) * (2 * p + 1)] = (float)ie;
        if (nrec - 1 < prm.hist_cap) a.hist[(size_t)(nrec - 1) * 5 + 4] = e2;
      }
      // X <- (X - R/eta) / nu  (PLAM: nu = 1), four rows of one column per
      // thread and step over all threads (rp is a multiple of 4; the padding
      // rows of X and R are zero and stay zero)
      const float fie = (float)ie;
      float4* X4 = reinterpret_cast<float4*>(Xs);
      const float4* R4 = reinterpret_cast<const float4*>(gr);
      for (int e4 = t; e4 < p * rp / 4; e4 += kResThreads) {
        const float sc = prm.variant == 1 ? inu[(4 * e4) / rp] : 1.f;
        float4 x = X4[e4];
        const float4 g = R4[e4];
        x.x = (x.x - g.x * fie) * sc;
        x.y = (x.y - g.y * fie) * sc;
        x.z = (x.z - g.z * fie) * sc;
        x.w = (x.w - g.w * fie) * sc;
        X4[e4] = x;
      }
      eta_prev = eta;
      eta = e2;
      inv_etap = fie;
      float* tmp = gr;
      gr = rpv;
      rpv = tmp;
      ++k;
      __syncthreads();
    }
  }

  // ---- write back the own rows of X and the last residual, then the state
  const bool timed_out = atomicAdd(a.err, 0) != 0;
  for (int e = t; e < p * nr; e += kResThreads) {
    const int c = e / nr, r = e % nr;
    a.X[r0 + r + (int64_t)c * a.ldx] = Xs[c * rp + r];
    // R^k in buffer k mod 2, R^{k-1} in the other (as the multi-kernel path leaves them)
    float* Rk = (k & 1) ? a.R1 : a.R0;
    float* Rk1 = (k & 1) ? a.R0 : a.R1;
    Rk[r0 + r + (int64_t)c * a.ldr] = gr[c * rp + r];
    Rk1[r0 + r + (int64_t)c * a.ldr] = rpv[c * rp + r];
  }
  if (b == 0 && t == 0) {
    DevState* st = a.st;
    st->k = k;
    st->stop = timed_out ? kTimeout : stop;
    st->nrec = nrec;
    st->K0 = K0;
    st->eta = eta;
    st->eta_prev = eta_prev;
    st->eta0 = eta0;
    st->kkt = last_kkt;
    st->feas = last_feas;
    st->f = last_f;
    st->ss = last_ss;
    st->sy = last_sy;
    st->yy = last_yy;
  }
}

// Shared memory bytes of one CTA for rows-per-CTA padding rp and width p.
size_t resident_smem_bytes(int p, int rp) {
  const int pp = (p + 3) & ~3;
  const size_t floats = (size_t)3 * p * rp + (size_t)2 * p * pp + (((size_t)2 * p * p + 3) & ~(size_t)3) + rp +
                        2 * kResMaxP + 3 * kResThreads + kResThreads;
  const size_t doubles = 64 + (size_t)rp + (size_t)(3 * p + 7);
  return floats * sizeof(float) + doubles * sizeof(double) + 16;
}

// Rows per CTA and CTA count for n rows on `sms` SMs; 0 CTAs when the problem
// does not fit the resident kernel.
void resident_plan(int64_t n, int p, int sms, size_t smem_limit, int* nblk, int* rows, int* rp,
                   size_t* smem) {
  *nblk = 0;
  if (p < 1 || p > kResMaxP || sms < 1) return;
  const int64_t rws = (n + sms - 1) / sms;
  if (rws > kResThreads || rws < 1) return;       // one row per thread in the row phases
  const int r = (int)rws;
  const int pad = (r + 3) & ~3;
  const size_t need = resident_smem_bytes(p, pad);
  if (need > smem_limit) return;
  *rows = r;
  *rp = pad;
  *nblk = (int)((n + r - 1) / r);
  *smem = need;
}

cudaError_t launch_resident_solve(const ResidentLaunch& L, cudaStream_t s) {
  ResidentArgs a;
  a.n = L.n; a.p = L.p; a.nblk = L.nblk; a.rows = L.rows; a.rp = L.rp;
  a.kind = L.kind; a.A = L.A; a.lda = L.lda; a.alpha = L.alpha; a.q = L.q;
  a.inv_np1 = 1.0 / (double)(L.n + 1);
  a.X = L.X; a.ldx = L.ldx; a.R0 = L.R0; a.R1 = L.R1; a.ldr = L.ldr;
  a.halo = L.halo; a.blk = L.blk; a.part = L.part; a.red = L.red; a.dots = L.dots; a.dred = L.dred;
  a.bar = L.bar; a.bar_expect = (unsigned int)(L.nblk + L.bar_extra); a.err = L.err; a.st = L.st; a.nubuf = L.nubuf; a.coef = L.coef; a.hist = L.hist;
  a.prm = L.prm;
  cudaError_t e = cudaFuncSetAttribute(resident_solve_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)resident_solve_kernel, dim3(L.nblk),
                                     dim3(kResThreads), args, L.smem, s);
}

cudaError_t preload_resident_kernels() {
  cudaFuncAttributes at;
  return cudaFuncGetAttributes(&at, resident_solve_kernel);
}

}  // namespace plam
