// Update GEMM, step size and primal update of one PLAM / PCAL iteration.
//
// update_kernel (eq. S1 and the Section 3.3 KKT shortcut): one CTA per
// 64 x 64 tile of the n x p output,
//     R = G - X M        (= grad_X L_beta(X, Lambda), M = Lambda - beta (B - I))
//     K = G - X Psi(C)   (KKT residual; only its squared norm is kept)
// with two accumulators over the same staged X tile, and an epilogue that
// forms, per column c, ||X_c||^2, <X_c,R_c>, ||R_c||^2, and, over the tile,
// <S,S>, <S,Y>, <Y,Y>, ||K||^2, ||G||^2 and <X,G>, where the Barzilai-Borwein
// pair (Section 5.1) S = X^k - X^{k-1}, Y = R^k - R^{k-1} is formed without
// storing X^{k-1}: the previous update was X^k_c = (X^{k-1}_c - R^{k-1}_c /
// eta^{k-1}) / nu^{k-1}_c (nu = 1 for PLAM), hence
//     S_c = (1 - nu^{k-1}_c) X^k_c - R^{k-1}_c / eta^{k-1}.
// The iteration counter k lives in device memory: R^k goes to buffer k mod 2
// and R^{k-1} is read from the other one, so the same launch sequence serves
// every iteration (and can be captured once in a CUDA graph).
//
// step_size_kernel: reduces the per-tile sums in a fixed order (CTAs over
// groups of 32 dot slots x ranges of row tiles, coalesced loads, then the
// ranges in order), and the last CTA to finish (atomic ticket, no waiting)
// computes the KKT value, the stopping decision,
// eta (rules of Section 5.1 with the safeguards of the design notes) and, for
// PCAL, the column norms nu_c = ||X_c - R_c/eta|| from
//     nu_c^2 = ||X_c||^2 - 2 <X_c,R_c> / eta + ||R_c||^2 / eta^2.
//
// primal_update_kernel: PLAM X <- X - R/eta (eq. PLAM-main); PCAL
// X_c <- (X_c - R_c/eta) / nu_c (Algorithm 3's closed form).
//
// GB300 runs double precision at 1/64 of the float rate (a double division
// costs about ten double FMAs), so the step-size kernel converts the scales
// 1/eta, 1/nu_c and 1 - nu_c once into the storage type (`coef`, two parity
// buffers of 2p + 1 entries) and the O(n p) kernels do no double arithmetic.
#include "plam_device.cuh"

namespace plam {

template <typename T>
__global__ void __launch_bounds__(kThreads)
update_kernel(int64_t n, int p, const T* __restrict__ X, int64_t ldx, const T* __restrict__ G,
              int64_t ldg, const T* __restrict__ R0, T* __restrict__ R1buf, int64_t ldr,
              const T* __restrict__ Mt, const T* __restrict__ L0t, const T* __restrict__ coef,
              const DevState* __restrict__ st, T* __restrict__ colpart, T* __restrict__ totpart) {
  if (st->stop != kRunning) return;
  const int k = st->k;
  T* R = (k & 1) ? R1buf : const_cast<T*>(R0);
  const T* Rprev = (k & 1) ? R0 : R1buf;
  // scales of the previous update (written by that iteration's step-size kernel)
  const T* cprev = coef + (size_t)((k + 1) & 1) * (2 * p + 1);
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int c0 = blockIdx.y * kTile;
  // inner-index step: 32 (float) or 16 (double, to stay within 48 KB of static shared memory)
  constexpr int KS = sizeof(T) == 8 ? 16 : kKStep;

  __shared__ T Xs[KS][kTile];
  __shared__ T Ms[kTile][KS + 1];
  __shared__ T Ls[kTile][KS + 1];

  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  T a1[4][4], a2[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) { a1[u][v] = T(0); a2[u][v] = T(0); }

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
        const bool ok = kr < p && cc < p;
        Ms[c][q] = ok ? Mt[kr + (size_t)cc * p] : T(0);
        Ls[c][q] = ok ? L0t[kr + (size_t)cc * p] : T(0);
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < KS; ++q) {
      T xa[4], mb[4], lb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xa[u] = Xs[q][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) { mb[v] = Ms[ty + 16 * v][q]; lb[v] = Ls[ty + 16 * v][q]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          a1[u][v] = fma(xa[u], mb[v], a1[u][v]);
          a2[u][v] = fma(xa[u], lb[v], a2[u][v]);
        }
    }
    __syncthreads();
  }

  // epilogue
  const T inv_etap = (k > 0) ? cprev[0] : T(0);
  T cxx[4], cxr[4], crr[4];
  T ss = 0, sy = 0, yy = 0, kk = 0, gg = 0, xg = 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    cxx[v] = 0; cxr[v] = 0; crr[v] = 0;
    const int c = c0 + ty + 16 * v;
    if (c >= p) continue;
    const T one_m_nu = (k > 0) ? cprev[1 + p + c] : T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t r = r0 + tx + 16 * u;
      if (r >= n) continue;
      const T x = X[r + (int64_t)c * ldx];
      const T g = G[r + (int64_t)c * ldg];
      const T rv = g - a1[u][v];
      const T kv = g - a2[u][v];
      R[r + (int64_t)c * ldr] = rv;
      cxx[v] = fma(x, x, cxx[v]);
      cxr[v] = fma(x, rv, cxr[v]);
      crr[v] = fma(rv, rv, crr[v]);
      kk = fma(kv, kv, kk);
      gg = fma(g, g, gg);
      xg = fma(x, g, xg);
      if (k > 0) {
        const T rp = Rprev[r + (int64_t)c * ldr];
        const T sv = one_m_nu * x - rp * inv_etap;
        const T yv = rv - rp;
        ss = fma(sv, sv, ss);
        sy = fma(sv, yv, sy);
        yy = fma(yv, yv, yy);
      }
    }
  }
  // column sums over the 16 threads (tx) that share a column: a half-warp butterfly
#pragma unroll
  for (int v = 0; v < 4; ++v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      cxx[v] += __shfl_xor_sync(0xffffffffu, cxx[v], o);
      cxr[v] += __shfl_xor_sync(0xffffffffu, cxr[v], o);
      crr[v] += __shfl_xor_sync(0xffffffffu, crr[v], o);
    }
  }
  if (tx == 0) {
    T* cp = colpart + (size_t)blockIdx.x * kColDots * p;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = c0 + ty + 16 * v;
      if (c < p) {
        cp[c] = cxx[v];
        cp[p + c] = cxr[v];
        cp[2 * p + c] = crr[v];
      }
    }
  }
  // tile totals: warp butterfly then warps in order
  T tot[kTotDots] = {ss, sy, yy, kk, gg, xg};
  __shared__ T wsum[kThreads / 32][kTotDots];
#pragma unroll
  for (int d = 0; d < kTotDots; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot[d] += __shfl_xor_sync(0xffffffffu, tot[d], o);
  }
  if ((t & 31) == 0) {
#pragma unroll
    for (int d = 0; d < kTotDots; ++d) wsum[t >> 5][d] = tot[d];
  }
  __syncthreads();
  if (t < kTotDots) {
    T s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += wsum[w][t];
    totpart[((size_t)blockIdx.x * gridDim.y + blockIdx.y) * kTotDots + t] = s;
  }
}

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;

// Phase 1 of the step-size kernel: CTA (g, t) sums, for the 32 dot slots of
// group g (lane = slot, so every load of a warp is one coalesced 128-byte
// line), the partials of the t-th range of row tiles.  Warp w takes the rows
// w, w + 8, ... of the range, eight independent loads in flight per lane,
// added in row order; the eight warps are then added in warp order.  The
// last group holds the six whole-tile sums.
template <typename T>
__device__ inline void step_partial_sums(int nrt, int nct, int p, const T* __restrict__ colpart,
                                         const T* __restrict__ totpart, T* __restrict__ dsum) {
  const int ncg = (kColDots * p + 31) / 32;
  const bool tot = (int)blockIdx.x == ncg;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int rows = tot ? nrt * nct : nrt;
  const int width = tot ? kTotDots : kColDots * p;
  const T* src = tot ? totpart : colpart;
  const int col = tot ? lane : (int)blockIdx.x * 32 + lane;
  const int per = (rows + (int)gridDim.y - 1) / (int)gridDim.y;
  const int i0 = (int)blockIdx.y * per;
  const int i1 = min(rows, i0 + per);
  T s = T(0);
  if (col < width) {
    int i = i0 + w;
    for (; i + 7 * kStepWarps < i1; i += 8 * kStepWarps) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(src + (size_t)(i + u * kStepWarps) * width + col);
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; i < i1; i += kStepWarps) s += __ldcg(src + (size_t)i * width + col);
  }
  __shared__ T red[kStepWarps][32];
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && col < width) {
    T t = red[0][lane];
#pragma unroll
    for (int u = 1; u < kStepWarps; ++u) t += red[u][lane];
    dsum[(size_t)blockIdx.y * (kColDots * p + kTotDots) + (tot ? kColDots * p : 0) + col] = t;
  }
}

template <typename T>
__global__ void __launch_bounds__(kStepThreads)
step_size_kernel(int nrt, int nct, const T* __restrict__ colpart, const T* __restrict__ totpart,
                 T* __restrict__ dsum, const double* __restrict__ feas_row,
                 const double* __restrict__ fpart, int nfpart, double* __restrict__ sums,
                 unsigned int* __restrict__ ticket, DevState* st, double* __restrict__ nubuf,
                 T* __restrict__ coef, double* __restrict__ hist, IterParams prm, int phase) {
  // phase 0: the whole step.  A row-sharded solve splits it around an all-reduce of `sums`:
  // phase 1 (every CTA) reduces this rank's partials into sums[0 .. nslots) and the objective's
  // f partials into sums[nslots]; phase 2 (one CTA) takes the sums of all ranks from there.
  if (st->stop != kRunning) return;
  const int p = prm.p;
  const int nslots = kColDots * p + kTotDots;
  __shared__ double scratch[33];
  __shared__ double sc[8];
  if (phase != 2) {
    step_partial_sums<T>(nrt, nct, p, colpart, totpart, dsum);
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the row ranges in order (all loads of a slot issued before the adds), in
    // the storage type: this CTA runs alone, and GB300 adds doubles at 1/64 of
    // the float rate, so ~25k double adds here would cost ~10 us
    const int nranges = (int)gridDim.y;
    for (int slot = threadIdx.x; slot < nslots; slot += blockDim.x) {
      T buf[kStepRanges];
#pragma unroll
      for (int u = 0; u < kStepRanges; ++u)
        buf[u] = (u < nranges) ? __ldcg(dsum + (size_t)u * nslots + slot) : T(0);
      T v = buf[0];
#pragma unroll
      for (int u = 1; u < kStepRanges; ++u)
        if (u < nranges) v += buf[u];
      sums[slot] = (double)v;
    }
    __syncthreads();
    if (phase == 1) {
      double hs = 0.0;
      for (int i = threadIdx.x; i < nfpart; i += blockDim.x) hs += __ldcg(fpart + i);
      const double hpart = block_sum(hs, scratch);
      if (threadIdx.x == 0) {
        sums[nslots] = hpart;
        *ticket = 0u;
      }
      return;
    }
  }
  const double* xx = sums;
  const double* xr = sums + p;
  const double* rr = sums + 2 * p;
  const double* tot = sums + kColDots * p;
  // sums of p and nfpart doubles (fixed order)
  double fsum = 0.0, xsum = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    fsum += __ldcg(feas_row + i);
    xsum += __ldcg(xx + i);
  }
  const double feas2 = block_sum(fsum, scratch);
  const double xx_all = block_sum(xsum, scratch);
  double hsum = 0.0;
  if (phase == 0)
    for (int i = threadIdx.x; i < nfpart; i += blockDim.x) hsum += __ldcg(fpart + i);
  const double hartree = phase == 0 ? block_sum(hsum, scratch) : __ldcg(sums + nslots);
  const int k = st->k;
  if (threadIdx.x == 0) {
    const double ss = __ldcg(tot + 0), sy = __ldcg(tot + 1), yy = __ldcg(tot + 2);
    const double kk = __ldcg(tot + 3), gg = __ldcg(tot + 4), xg = __ldcg(tot + 5);
    if (k == 0) {
      st->K0 = sqrt(kk);
      st->eta0 = (prm.eta0_user > 0.0) ? prm.eta0_user
                                        : ((xx_all > 0.0 ? sqrt(gg / xx_all) : 1.0) + prm.beta);
    }
    const double K0 = st->K0;
    const double kkt = (K0 > 0.0) ? sqrt(kk) / K0 : 0.0;
    const double feas = sqrt(feas2);
    const double f = prm.f_xg * xg + prm.f_part * hartree;
    st->kkt = kkt;
    st->feas = feas;
    st->f = f;
    st->ss = ss; st->sy = sy; st->yy = yy;
    if (!st->refine && prm.refine_switch > 0.0 && isfinite(kkt)) {
      if (k == 0 || kkt < 0.5 * st->kkt_best) {
        st->kkt_best = kkt;
        st->k_best = k;
      }
      if (kkt < prm.refine_switch || k - st->k_best >= kStallIters) st->refine = 1;
    }
    const int rec = st->nrec;
    if (rec < prm.hist_cap) {
      double* h = hist + (size_t)rec * 5;
      h[0] = (double)k; h[1] = f; h[2] = kkt; h[3] = feas; h[4] = nan("");
      st->nrec = rec + 1;
    }
    int stop = kRunning;
    double eta = st->eta;
    if (!isfinite(kkt) || !isfinite(feas) || (prm.feas_max > 0.0 && feas > prm.feas_max))
      stop = kDiverged;
    else if (K0 == 0.0 || kkt < prm.tol) stop = kConverged;
    else if (k >= prm.maxit) stop = kMaxit;
    else {
      const double eta0 = st->eta0;
      const double eprev = st->eta;
      if (prm.eta_rule == 3) {                      // constant
        eta = (prm.gamma > 0.0) ? prm.gamma : eta0;
      } else if (k == 0) {
        eta = eta0;
      } else if (prm.eta_rule == 4) {               // differential ||Y|| / ||S||
        eta = (ss > 0.0 && yy > 0.0) ? sqrt(yy / ss) : eprev;
      } else if (ss == 0.0 || sy == 0.0) {
        eta = eprev;
      } else {
        const double bb1 = fabs(sy) / ss, bb2 = yy / fabs(sy);
        if (prm.eta_rule == 1) eta = bb1;
        else if (prm.eta_rule == 2) eta = bb2;
        else eta = (k & 1) ? bb1 : bb2;              // alternating BB
      }
      if (!isfinite(eta)) stop = kDiverged;
      else eta = eta_clamp(eta, eta0, prm.eta_min, prm.eta_max);
    }
    sc[0] = eta;
    sc[1] = (double)stop;
  }
  __syncthreads();
  const double eta = sc[0];
  int stop = (int)sc[1];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  double* nu = nubuf + (size_t)(k & 1) * p;
  // per-update scales in the storage type: [1/eta, 1/nu_c (p), 1 - nu_c (p)]
  T* cf = coef + (size_t)(k & 1) * (2 * p + 1);
  if (stop == kRunning) {
    const double ie = 1.0 / eta;
    if (threadIdx.x == 0) cf[0] = (T)ie;
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
      // ||X_c - R_c/eta||^2; for PLAM only checked (an overflowing step stops the run
      // before X is overwritten), for PCAL also the column scale of Algorithm 3
      const double q = __ldcg(xx + c) - 2.0 * __ldcg(xr + c) * ie + __ldcg(rr + c) * ie * ie;
      double v = 1.0;
      if (prm.variant == 1) {
        v = sqrt(q);
        if (!(v > 0.0) || !isfinite(v)) bad = 1;
      } else if (!isfinite(q)) {
        bad = 1;
      }
      nu[c] = v;
      cf[1 + c] = (T)(1.0 / v);
      cf[1 + p + c] = (T)(1.0 - v);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (stop == kRunning && bad) stop = kDiverged;
    if (stop == kRunning) {
      st->eta_prev = st->eta;
      st->eta = eta;
      const int rec = st->nrec - 1;
      if (rec >= 0 && rec < prm.hist_cap) hist[(size_t)rec * 5 + 4] = eta;
      st->k = k + 1;
    }
    st->stop = stop;
    *ticket = 0u;
  }
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; static constexpr int n = 4; };
template <> struct Vec16<double> { typedef double2 type; static constexpr int n = 2; };

__device__ __forceinline__ float4 axpy_scale(float4 x, float4 r, float ie, float inu) {
  return make_float4((x.x - r.x * ie) * inu, (x.y - r.y * ie) * inu, (x.z - r.z * ie) * inu,
                     (x.w - r.w * ie) * inu);
}
__device__ __forceinline__ double2 axpy_scale(double2 x, double2 r, double ie, double inu) {
  return make_double2((x.x - r.x * ie) * inu, (x.y - r.y * ie) * inu);
}

// vec = 1: columns start on 16-byte boundaries, so each thread moves whole
// 16-byte vectors (four floats or two doubles) and the tail of a column, if
// any, is done element by element.
template <typename T>
__global__ void __launch_bounds__(256)
primal_update_kernel(int64_t n, int p, T* __restrict__ X, int64_t ldx,
                     const T* __restrict__ R0, const T* __restrict__ R1, int64_t ldr,
                     const T* __restrict__ coef, const DevState* __restrict__ st, int variant,
                     int vec) {
  if (st->stop != kRunning) return;
  const int km1 = st->k - 1;                 // the step kernel already counted this update
  const T* R = (km1 & 1) ? R1 : R0;
  const T* cf = coef + (size_t)(km1 & 1) * (2 * p + 1);
  const T ie = cf[0];
  const int c = blockIdx.y;
  const T inu = (variant == 1) ? cf[1 + c] : T(1);
  T* xc = X + (int64_t)c * ldx;
  const T* rc = R + (int64_t)c * ldr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    typedef typename Vec16<T>::type V;
    constexpr int W = Vec16<T>::n;
    const int64_t nv = n / W;
    V* xv = reinterpret_cast<V*>(xc);
    const V* rv = reinterpret_cast<const V*>(rc);
    for (int64_t i = r; i < nv; i += stride) xv[i] = axpy_scale(xv[i], __ldg(rv + i), ie, inu);
    r += nv * W;
  }
  for (; r < n; r += stride) xc[r] = (xc[r] - rc[r] * ie) * inu;
}

// ---------------------------------------------------------------- launchers

template <typename T>
cudaError_t launch_update(int64_t n, int p, const T* X, int64_t ldx, const T* G, int64_t ldg,
                          T* R0, T* R1, int64_t ldr, const T* Mt, const T* L0t, const T* coef,
                          const DevState* st, T* colpart, T* totpart, cudaStream_t s) {
  dim3 grid((unsigned)((n + kTile - 1) / kTile), (p + kTile - 1) / kTile);
  update_kernel<T><<<grid, kThreads, 0, s>>>(n, p, X, ldx, G, ldg, R0, R1, ldr, Mt, L0t, coef, st,
                                              colpart, totpart);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_size(int nrt, int nct, const T* colpart, const T* totpart, T* dsum,
                             const double* feas_row, const double* fpart, int nfpart, double* sums,
                             unsigned int* ticket, DevState* st, double* nubuf, T* coef,
                             double* hist, IterParams prm, cudaStream_t s, int phase) {
  // 32 dot slots per CTA column, about 64 row tiles (8 per warp) per CTA row
  const int groups = (kColDots * prm.p + 31) / 32 + 1;
  int ranges = (nrt + 8 * kStepWarps - 1) / (8 * kStepWarps);
  ranges = ranges < 1 ? 1 : (ranges > kStepRanges ? kStepRanges : ranges);
  const dim3 grid = phase == 2 ? dim3(1, 1) : dim3(groups, ranges);
  step_size_kernel<T><<<grid, kStepThreads, 0, s>>>(nrt, nct, colpart, totpart, dsum, feas_row,
                                                     fpart, nfpart, sums, ticket, st, nubuf, coef,
                                                     hist, prm, phase);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_primal_update(int64_t n, int p, T* X, int64_t ldx, const T* R0, const T* R1,
                                 int64_t ldr, const T* coef, const DevState* st, int variant,
                                 cudaStream_t s) {
  // one wave of CTAs (8 per SM), grid-stride over rows: the state and scale
  // loads at the top of each CTA are paid once, not once per 256 elements
  const int threads = 256;
  int64_t bx = (n + threads - 1) / threads;
  const int64_t cap = ((int64_t)device_sm_count() * 8 + p - 1) / p;
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  dim3 grid((unsigned)bx, p);
  const int vec = (ldx * (int64_t)sizeof(T)) % 16 == 0 && (ldr * (int64_t)sizeof(T)) % 16 == 0 &&
                  (uintptr_t)X % 16 == 0 && (uintptr_t)R0 % 16 == 0 && (uintptr_t)R1 % 16 == 0;
  primal_update_kernel<T><<<grid, threads, 0, s>>>(n, p, X, ldx, R0, R1, ldr, coef, st, variant,
                                                   vec);
  return cudaGetLastError();
}

cudaError_t preload_update_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, update_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, update_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, step_size_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, step_size_kernel<double>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, primal_update_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, primal_update_kernel<double>);
  return e;
}

#define PLAM_INST(T)                                                                              \
  template cudaError_t launch_update<T>(int64_t, int, const T*, int64_t, const T*, int64_t, T*,    \
                                        T*, int64_t, const T*, const T*, const T*,                 \
                                        const DevState*, T*, T*, cudaStream_t);                    \
  template cudaError_t launch_step_size<T>(int, int, const T*, const T*, T*, const double*,       \
                                           const double*, int, double*, unsigned int*, DevState*,  \
                                           double*, T*, double*, IterParams, cudaStream_t, int);   \
  template cudaError_t launch_primal_update<T>(int64_t, int, T*, int64_t, const T*, const T*,      \
                                               int64_t, const T*, const DevState*, int,            \
                                               cudaStream_t);
PLAM_INST(float)
PLAM_INST(double)
#undef PLAM_INST

}  // namespace plam
