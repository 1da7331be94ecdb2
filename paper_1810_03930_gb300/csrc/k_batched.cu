// Batched PCAL / PLAM: many independent dense trace problems
// f_b = 1/2 tr(X_b^T A_b X_b) (Problem 3 of Section 5.2) of uneven n_b, p_b
// (p_b <= 64) in ONE persistent launch.  Each CTA takes problems from a
// device work queue (largest first, as ordered by the host) and runs the
// whole iteration of Algorithm 2 / 3 for one problem with block-level
// synchronisation only; the p x p algebra (Grams in FP64, eq. Lambda1 /
// lambda2, M = Lambda - beta (B - I), eq. S1) stays in shared memory.
//
// Per iteration of problem b (FP32 storage and products, FP64 p x p algebra
// and scalars, as the single-problem FP32 mode):
//   1. G = A X                      RB x 64 output tiles, 32-deep stages of A and X
//   2. B = X^T X, C = X^T G          FP32 sums over 32-row stages, added up in FP64
//   3. Psi(C), d (eq. lambda2), M, ||B - I||, f = 1/2 tr(C)
//   4. R = G - X M, K = G - X Psi(C) with the column dots and the BB sums
//   5. eta (Section 5.1 rules), stop test, PCAL column norms nu
//   6. X <- (X - R / eta) / nu
// and, at the end, the FP64 Cholesky-QR of the final iterate (Section 5.3).
//
// The row-block height RB (64, 128 or 256) is the tile shape the host
// autotuner chooses; a warp owns 16 output columns and 32 rows per row slice,
// so the column dots are warp sums with no cross-warp reduction.
#include "../../include/plam.h"
#include "plam_device.cuh"

namespace plam {

constexpr int kBThreads = 512;
constexpr int kBMaxP = 64;
constexpr int kBK = 32;              // inner-index depth of one shared-memory stage
// Row strides of the staged tiles, padded against bank conflicts: the X tile of
// A X is written with 32 consecutive lanes on 32 consecutive rows and read as
// 16-byte vectors (stride 68: a multiple of 4, 4 banks apart per row), the Gram
// tiles are written the same way and read element-wise (stride 65).
constexpr int kBXS = kBMaxP + 4;
constexpr int kBGS = kBMaxP + 1;

// Shared memory of one CTA (dynamic, 16-byte aligned).
struct BatchSmem {
  double B[kBMaxP][kBMaxP];
  double C[kBMaxP][kBMaxP];
  float M[kBMaxP][kBMaxP];      // M[j][c]
  float L[kBMaxP][kBMaxP];      // Psi(C)[j][c]
  double col[3][kBMaxP];        // ||X_c||^2, <X_c, R_c>, ||R_c||^2
  double d[kBMaxP];
  float inv_nu[kBMaxP], omn[kBMaxP], omn_prev[kBMaxP];
  double scratch[40];
  double sc[16];
  int flags[4];
  int problem;
};

// one stage buffer: a 32 x RB tile of A and a 32 x 64 tile of X (two buffers per CTA)
__host__ __device__ inline size_t batch_stage_floats(int rb) { return (size_t)kBK * rb + (size_t)kBK * kBXS; }

// ---------------------------------------------------------------- step 1: G = A X
// The sum over n runs in float within each 32-deep stage and is carried across
// stages in a compensated (Kahan) pair, so that the FP32 rounding of G grows
// with the stage depth, not with n.  Lane tx owns RB/32 rows in groups of four
// consecutive ones (conflict-free float4 loads from shared memory; pairs for
// RB = 64), warp ty the columns 4ty .. 4ty + 3 (a broadcast float4); the next
// stage is fetched into registers while the current one is multiplied (two
// shared-memory buffers, one barrier a stage).
template <int RB>
__device__ void batch_ax(const BatchDesc& q, float* st0, float* st1) {
  constexpr int R4 = RB / 32;
  constexpr int NA = kBK * RB / kBThreads;
  constexpr int NX = kBK * kBMaxP / kBThreads;
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  const int64_t n = q.n;
  const int p = q.p;
  const bool active = 4 * ty < p;            // warp-uniform: this warp has columns
  float pa[NA], px[NX];
  for (int64_t r0 = 0; r0 < n; r0 += RB) {
    float sum[R4][4], comp[R4][4];
#pragma unroll
    for (int i = 0; i < R4; ++i)
#pragma unroll
      for (int v = 0; v < 4; ++v) sum[i][v] = comp[i][v] = 0.f;
    auto fetch = [&](int64_t k0) {
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int e = t + j * kBThreads, i = e % RB, kk = e / RB;
        const int64_t r = r0 + i, kc = k0 + kk;
        pa[j] = (r < n && kc < n) ? q.A[r + kc * q.lda] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        const int e = t + j * kBThreads, kk = e % kBK, c = e / kBK;
        const int64_t kr = k0 + kk;
        px[j] = (kr < n && c < p) ? q.X[kr + (int64_t)c * q.ldx] : 0.f;
      }
    };
    auto stash = [&](float* st) {
#pragma unroll
      for (int j = 0; j < NA; ++j) st[t + j * kBThreads] = pa[j];
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        const int e = t + j * kBThreads;
        st[kBK * RB + (e % kBK) * kBXS + e / kBK] = px[j];
      }
    };
    fetch(0);
    stash(st0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = 0; k0 < n; k0 += kBK) {
      const bool more = k0 + kBK < n;
      if (more) fetch(k0 + kBK);
      const float* st = buf ? st1 : st0;
      if (active) {
        float acc[R4][4];
#pragma unroll
        for (int i = 0; i < R4; ++i)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[i][v] = 0.f;
#pragma unroll 4
        for (int kk = 0; kk < kBK; ++kk) {
          float a[R4];
          if (R4 == 2) {
            const float2 a2 = *reinterpret_cast<const float2*>(st + kk * RB + tx * 2);
            a[0] = a2.x;
            a[1] = a2.y;
          } else {
#pragma unroll
            for (int h = 0; h < R4 / 4; ++h) {   // conflict-free float4 rows 128 h + 4 tx .. + 3
              const float4 a4 = *reinterpret_cast<const float4*>(st + kk * RB + h * 128 + tx * 4);
              a[4 * h] = a4.x;
              a[4 * h + 1] = a4.y;
              a[4 * h + 2] = a4.z;
              a[4 * h + 3] = a4.w;
            }
          }
          const float4 b = *reinterpret_cast<const float4*>(st + kBK * RB + kk * kBXS + 4 * ty);
#pragma unroll
          for (int i = 0; i < R4; ++i) {
            acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
            acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
            acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
            acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
          }
        }
#pragma unroll
        for (int i = 0; i < R4; ++i)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float y = acc[i][v] - comp[i][v];
            const float s2 = sum[i][v] + y;
            comp[i][v] = (s2 - sum[i][v]) - y;
            sum[i][v] = s2;
          }
      }
      if (more) stash(buf ? st0 : st1);
      __syncthreads();
      buf ^= 1;
    }
    if (active) {
#pragma unroll
      for (int i = 0; i < R4; ++i) {
        const int64_t r = r0 + (R4 == 2 ? tx * 2 + i : (i / 4) * 128 + tx * 4 + (i % 4));
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = 4 * ty + v;
          if (r < n && c < p) q.G[r + (int64_t)c * q.ldw] = sum[i][v];
        }
      }
    }
  }
}

// ---------------------------------------------------------------- step 2: Grams into FP64
// Thread (ti, tj) = (t & 15, t >> 4) owns entries i = ti + 16a (a < 4), j = tj + 32b (b < 2).
// Y = G (C = X^T G) or X; with exact = true the products are formed in double (final step).
template <bool exact>
__device__ void batch_grams(const BatchDesc& q, const float* Y, int64_t ldy, float* stX, float* stY,
                            double (*Bout)[kBMaxP], double (*Cout)[kBMaxP]) {
  const int t = threadIdx.x, ti = t & 15, tj = t >> 4;
  const int64_t n = q.n;
  const int p = q.p;
  double dB[4][2], dC[4][2];
  float fB[4][2], fC[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) { dB[a][b] = dC[a][b] = 0.0; fB[a][b] = fC[a][b] = 0.f; }
  int stage = 0;
  for (int64_t r0 = 0; r0 < n; r0 += kBK, ++stage) {
    for (int e = t; e < kBK * kBMaxP; e += kBThreads) {
      const int rr = e % kBK, c = e / kBK;
      const int64_t r = r0 + rr;
      const bool ok = r < n && c < p;
      stX[rr * kBGS + c] = ok ? q.X[r + (int64_t)c * q.ldx] : 0.f;
      if (Y) stY[rr * kBGS + c] = ok ? Y[r + (int64_t)c * ldy] : 0.f;
    }
    __syncthreads();
    for (int rr = 0; rr < kBK; ++rr) {
      float xi[4], xj[2], yj[2];
#pragma unroll
      for (int a = 0; a < 4; ++a) xi[a] = stX[rr * kBGS + ti + 16 * a];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        xj[b] = stX[rr * kBGS + tj + 32 * b];
        yj[b] = Y ? stY[rr * kBGS + tj + 32 * b] : 0.f;
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          if (exact) {
            dB[a][b] = fma((double)xi[a], (double)xj[b], dB[a][b]);
          } else {
            fB[a][b] = fmaf(xi[a], xj[b], fB[a][b]);
            fC[a][b] = fmaf(xi[a], yj[b], fC[a][b]);
          }
        }
    }
    __syncthreads();
    if (!exact) {   // each 32-row stage's float sums into the FP64 totals
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          dB[a][b] += (double)fB[a][b];
          dC[a][b] += (double)fC[a][b];
          fB[a][b] = fC[a][b] = 0.f;
        }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = ti + 16 * a, j = tj + 32 * b;
      Bout[i][j] = dB[a][b];
      if (Cout) Cout[i][j] = dC[a][b];
    }
  __syncthreads();
}

// ---------------------------------------------------------------- one problem
template <int RB>
__device__ void batch_solve_one(const BatchDesc& q, const BatchParams& prm, plam_info_t* out,
                                BatchSmem& S, float* stA, float* stX) {
  constexpr int U = RB / 32;
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5, lane = t & 31;
  const int64_t n = q.n;
  const int p = q.p, V = (p + 15) / 16;
  // scalars kept by thread 0 across iterations
  double K0 = 0.0, eta0 = 0.0, eta = 0.0, kkt = NAN, feas = NAN, f = NAN;
  float ie_prev = 0.f;
  for (int c = t; c < kBMaxP; c += kBThreads) S.omn_prev[c] = 0.f;
  __syncthreads();
  int k = 0, stop = kRunning;
  for (;; ++k) {
    float* R = (k & 1) ? q.R1 : q.R0;
    const float* Rp = (k & 1) ? q.R0 : q.R1;
    // 1-2. gradient and Grams
    batch_ax<RB>(q, stA, stX);   // stA, stX: the two stage buffers
    __syncthreads();
    batch_grams<false>(q, q.G, q.ldw, stA, stX, S.B, S.C);
    // 3. p x p algebra in FP64
    double feas2 = 0.0, tr = 0.0;
    for (int e = t; e < p * p; e += kBThreads) {
      const int i = e % p, j = e / p;
      S.L[i][j] = (float)(0.5 * (S.C[i][j] + S.C[j][i]));
      const double bij = S.B[i][j] - (i == j ? 1.0 : 0.0);
      feas2 += bij * bij;
      if (i == j) tr += S.C[i][i];
    }
    feas2 = block_sum(feas2, S.scratch);
    tr = block_sum(tr, S.scratch);
    for (int i = t; i < p; i += kBThreads) {
      double di = 0.0;
      if (prm.lambda2) {            // d_i = C_ii - sum_k B_ik Psi(C)_ik + beta (sum_k B_ik^2 - B_ii)
        double s = 0.0, b2 = 0.0;
        for (int kk = 0; kk < p; ++kk) {
          const double bik = S.B[i][kk];
          s += bik * (0.5 * (S.C[i][kk] + S.C[kk][i]));
          b2 += bik * bik;
        }
        di = S.C[i][i] - s + prm.beta * (b2 - S.B[i][i]);
      }
      S.d[i] = di;
    }
    __syncthreads();
    for (int e = t; e < p * p; e += kBThreads) {
      const int i = e % p, j = e / p;
      const double l = 0.5 * (S.C[i][j] + S.C[j][i]);
      S.M[i][j] = (float)(l + (i == j ? S.d[i] : 0.0) - prm.beta * (S.B[i][j] - (i == j ? 1.0 : 0.0)));
    }
    __syncthreads();
    // 4. R = G - X M, K = G - X Psi(C), dots
    float cxx[4], cxr[4], crr[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) cxx[v] = cxr[v] = crr[v] = 0.f;
    float ss = 0.f, sy = 0.f, yy = 0.f, kk2 = 0.f, gg = 0.f;
    for (int64_t r0 = 0; r0 < n; r0 += RB) {
      float a1[U][4], a2[U][4];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) a1[u][v] = a2[u][v] = 0.f;
      for (int j0 = 0; j0 < p; j0 += kBK) {
        for (int e = t; e < kBK * RB; e += kBThreads) {
          const int i = e % RB, jj = e / RB;
          const int64_t r = r0 + i;
          const int j = j0 + jj;
          stA[jj * RB + i] = (r < n && j < p) ? q.X[r + (int64_t)j * q.ldx] : 0.f;
        }
        __syncthreads();
        const int jn = min(kBK, p - j0);
        for (int jj = 0; jj < jn; ++jj) {
          float xa[U], mb[4], lb[4];
#pragma unroll
          for (int u = 0; u < U; ++u) xa[u] = stA[jj * RB + tx + 32 * u];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            mb[v] = S.M[j0 + jj][(ty + 16 * v) & (kBMaxP - 1)];
            lb[v] = S.L[j0 + jj][(ty + 16 * v) & (kBMaxP - 1)];
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v)
              if (v < V) {
                a1[u][v] = fmaf(xa[u], mb[v], a1[u][v]);
                a2[u][v] = fmaf(xa[u], lb[v], a2[u][v]);
              }
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t r = r0 + tx + 32 * u;
        if (r >= n) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = ty + 16 * v;
          if (v >= V || c >= p) continue;
          const float x = q.X[r + (int64_t)c * q.ldx], g = q.G[r + (int64_t)c * q.ldw];
          const float rv = g - a1[u][v], kv = g - a2[u][v];
          R[r + (int64_t)c * q.ldw] = rv;
          cxx[v] = fmaf(x, x, cxx[v]);
          cxr[v] = fmaf(x, rv, cxr[v]);
          crr[v] = fmaf(rv, rv, crr[v]);
          kk2 = fmaf(kv, kv, kk2);
          gg = fmaf(g, g, gg);
          if (k > 0) {
            const float rp = Rp[r + (int64_t)c * q.ldw];
            const float sv = S.omn_prev[c] * x - rp * ie_prev, yv = rv - rp;
            ss = fmaf(sv, sv, ss);
            sy = fmaf(sv, yv, sy);
            yy = fmaf(yv, yv, yy);
          }
        }
      }
    }
    // warp ty owns columns ty + 16 v: the column sums are warp sums
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double s0 = warp_sum_d((double)cxx[v]), s1 = warp_sum_d((double)cxr[v]);
      const double s2 = warp_sum_d((double)crr[v]);
      const int c = ty + 16 * v;
      if (lane == 0 && c < p) { S.col[0][c] = s0; S.col[1][c] = s1; S.col[2][c] = s2; }
    }
    const double dss = block_sum((double)ss, S.scratch), dsy = block_sum((double)sy, S.scratch);
    const double dyy = block_sum((double)yy, S.scratch), dkk = block_sum((double)kk2, S.scratch);
    const double dgg = block_sum((double)gg, S.scratch);
    // 5. scalars (thread 0): the rules of the single-problem step-size kernel
    if (t == 0) {
      double xx_all = 0.0;
      for (int c = 0; c < p; ++c) xx_all += S.col[0][c];
      if (k == 0) {
        K0 = sqrt(dkk);
        eta0 = (prm.eta0_user > 0.0) ? prm.eta0_user
                                     : ((xx_all > 0.0 ? sqrt(dgg / xx_all) : 1.0) + prm.beta);
      }
      kkt = (K0 > 0.0) ? sqrt(dkk) / K0 : 0.0;
      feas = sqrt(feas2);
      f = 0.5 * tr;
      int st = kRunning;
      double e = eta;
      if (!isfinite(kkt)) st = kDiverged;
      else if (K0 == 0.0 || kkt < prm.tol) st = kConverged;
      else if (k >= prm.maxit) st = kMaxit;
      else {
        if (prm.eta_rule == 3) e = (prm.gamma > 0.0) ? prm.gamma : eta0;
        else if (k == 0) e = eta0;
        else if (prm.eta_rule == 4) e = (dss > 0.0 && dyy > 0.0) ? sqrt(dyy / dss) : eta;
        else if (dss == 0.0 || dsy == 0.0) e = eta;
        else {
          const double bb1 = fabs(dsy) / dss, bb2 = dyy / fabs(dsy);
          e = prm.eta_rule == 1 ? bb1 : prm.eta_rule == 2 ? bb2 : ((k & 1) ? bb1 : bb2);
        }
        if (!isfinite(e)) st = kDiverged;
        else e = eta_clamp(e, eta0, prm.eta_min, prm.eta_max);
      }
      eta = e;
      S.sc[0] = e;
      S.sc[1] = (double)st;
      S.flags[0] = 0;
    }
    __syncthreads();
    stop = (int)S.sc[1];
    if (stop != kRunning) break;
    const double ie = 1.0 / S.sc[0];
    for (int c = t; c < p; c += kBThreads) {
      const double q2 = S.col[0][c] - 2.0 * S.col[1][c] * ie + S.col[2][c] * ie * ie;
      double v = 1.0;
      if (prm.variant == 1) {
        v = sqrt(q2);
        if (!(v > 0.0) || !isfinite(v)) S.flags[0] = 1;
      } else if (!isfinite(q2)) {
        S.flags[0] = 1;
      }
      S.inv_nu[c] = (float)(1.0 / v);
      S.omn[c] = (float)(1.0 - v);
    }
    __syncthreads();
    if (S.flags[0]) { stop = kDiverged; break; }
    // 6. X <- (X - R / eta) / nu
    const float ief = (float)ie;
    for (int c = 0; c < p; ++c) {
      const float inu = S.inv_nu[c];
      for (int64_t r = t; r < n; r += kBThreads)
        q.X[r + (int64_t)c * q.ldx] = (q.X[r + (int64_t)c * q.ldx] - R[r + (int64_t)c * q.ldw] * ief) * inu;
    }
    for (int c = t; c < p; c += kBThreads) S.omn_prev[c] = S.omn[c];
    ie_prev = ief;
    __syncthreads();
  }
  // final orthonormalisation (Section 5.3): FP64 Gram of the float iterate, Cholesky, Q = X R^{-1}
  double feas_orth = NAN;
  int chol_fail = 0;
  if (q.Q != nullptr && stop != kDiverged) {
    batch_grams<true>(q, nullptr, 0, stA, stX, S.B, nullptr);
    for (int j = 0; j < p; ++j) {              // Cholesky B = L L^T, L in the lower triangle
      double s = 0.0;
      const int i = j + t;
      if (t < p - j) {
        s = S.B[i][j];
        for (int kk = 0; kk < j; ++kk) s -= S.B[i][kk] * S.B[j][kk];
      }
      __syncthreads();
      if (t == 0) {
        if (!(s > 0.0) || !isfinite(s)) S.flags[1] = 1;
        S.B[j][j] = sqrt(s);
      }
      __syncthreads();
      if (t > 0 && t < p - j) S.B[i][j] = s / S.B[j][j];
      __syncthreads();
    }
    chol_fail = S.flags[1];
    if (!chol_fail) {
      if (t < p) {                              // column t of L^{-1} into C[.][t]
        for (int i = 0; i < p; ++i) {
          double s = (i == t) ? 1.0 : 0.0;
          for (int kk = t; kk < i; ++kk) s -= S.B[i][kk] * S.C[kk][t];
          S.C[i][t] = (i < t) ? 0.0 : s / S.B[i][i];
        }
      }
      __syncthreads();
      // Q(r, c) = sum_{j <= c} X(r, j) (L^{-1})_{c j}
      for (int64_t e = t; e < n * p; e += kBThreads) {
        const int c = (int)(e / n);
        const int64_t r = e - (int64_t)c * n;
        double s = 0.0;
        for (int j = 0; j <= c; ++j) s = fma((double)q.X[r + (int64_t)j * q.ldx], S.C[c][j], s);
        q.Q[r + (int64_t)c * q.ldq] = s;
      }
      __syncthreads();
      // ||Q^T Q - I||_F: Q^T Q over 32-row stages of Q staged in shared memory (the stage
      // buffers), thread (ti, tj) owning entries i = ti + 16a, j = tj + 32b
      {
        double* qs = reinterpret_cast<double*>(stA);      // [32][65] doubles
        const int ti = t & 15, tj = t >> 4;
        double acc[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = 0.0;
        for (int64_t r0 = 0; r0 < n; r0 += kBK) {
          for (int e = t; e < kBK * kBMaxP; e += kBThreads) {
            const int rr = e % kBK, c = e / kBK;
            const int64_t r = r0 + rr;
            qs[rr * kBGS + c] = (r < n && c < p) ? q.Q[r + (int64_t)c * q.ldq] : 0.0;
          }
          __syncthreads();
          for (int rr = 0; rr < kBK; ++rr) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              const double qi = qs[rr * kBGS + ti + 16 * a];
              acc[a][0] = fma(qi, qs[rr * kBGS + tj], acc[a][0]);
              acc[a][1] = fma(qi, qs[rr * kBGS + tj + 32], acc[a][1]);
            }
          }
          __syncthreads();
        }
        double fe = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 2; ++b2) {
            const int i = ti + 16 * a, j = tj + 32 * b2;
            if (i < p && j < p) {
              const double e2 = acc[a][b2] - (i == j ? 1.0 : 0.0);
              fe += e2 * e2;
            }
          }
        feas_orth = sqrt(block_sum(fe, S.scratch));
      }
    }
  }
  if (t == 0) {
    plam_info_t inf;
    inf.iters = k;
    inf.status = stop == kConverged ? PLAM_OK : stop == kMaxit ? PLAM_ERR_NOT_CONVERGED
                                                               : PLAM_ERR_DIVERGED;
    if (chol_fail) inf.status = PLAM_ERR_CHOLESKY;
    inf.converged = stop == kConverged;
    inf.pad_ = 0;
    inf.f = f;
    inf.kkt_rel = kkt;
    inf.feas = feas;
    inf.eta = eta;
    inf.K0 = K0;
    inf.eta0 = eta0;
    inf.f_orth = NAN;
    inf.kkt_orth = NAN;
    inf.feas_orth = feas_orth;
    *out = inf;
    S.flags[1] = 0;
  }
  __syncthreads();
}

template <int RB>
__global__ void __launch_bounds__(kBThreads, 1)
batched_solve_kernel(const BatchDesc* __restrict__ desc, const int* __restrict__ order, int count,
                     int* next, plam_info_t* info, BatchParams prm) {
  extern __shared__ __align__(16) unsigned char bsm[];
  BatchSmem& S = *reinterpret_cast<BatchSmem*>(bsm);
  float* stA = reinterpret_cast<float*>(bsm + ((sizeof(BatchSmem) + 15) & ~(size_t)15));
  float* stX = stA + batch_stage_floats(RB);     // second stage buffer
  if (threadIdx.x == 0) S.flags[1] = 0;
  for (;;) {
    if (threadIdx.x == 0) S.problem = atomicAdd(next, 1);
    __syncthreads();
    const int b = S.problem;
    __syncthreads();
    if (b >= count) break;
    const int id = order[b];
    batch_solve_one<RB>(desc[id], prm, info + id, S, stA, stX);
  }
}

// ---------------------------------------------------------------- host side

size_t batch_smem_bytes(int rb) {
  return ((sizeof(BatchSmem) + 15) & ~(size_t)15) + 2 * batch_stage_floats(rb) * sizeof(float);
}

cudaError_t launch_batched(int rb, const BatchDesc* desc, const int* order, int count, int* next,
                           plam_info_t* info, BatchParams prm, int grid, cudaStream_t s) {
  const size_t smem = batch_smem_bytes(rb);
  cudaError_t e = cudaSuccess;
  switch (rb) {
    case 64:
      e = cudaFuncSetAttribute(batched_solve_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e == cudaSuccess)
        batched_solve_kernel<64><<<grid, kBThreads, smem, s>>>(desc, order, count, next, info, prm);
      break;
    case 128:
      e = cudaFuncSetAttribute(batched_solve_kernel<128>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        batched_solve_kernel<128><<<grid, kBThreads, smem, s>>>(desc, order, count, next, info, prm);
      break;
    case 256:
      e = cudaFuncSetAttribute(batched_solve_kernel<256>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        batched_solve_kernel<256><<<grid, kBThreads, smem, s>>>(desc, order, count, next, info, prm);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t preload_batched_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, batched_solve_kernel<64>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, batched_solve_kernel<128>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, batched_solve_kernel<256>);
  return e;
}

}  // namespace plam
