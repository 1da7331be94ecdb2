// Update GEMM of one PLAM / PCAL iteration on the 5th-generation tensor cores
// (tcgen05, kind::tf32, sm_103a):
//     R = G - X M        (eq. S1: grad_X L_beta with M = Lambda - beta (B - I))
//     K = G - X Psi(C)   (the KKT residual of the Section 3.3 shortcut; only
//                         its squared norm is kept)
// with the epilogue of the CUDA-core update kernel: per column c the partial
// dots ||X_c||^2, <X_c,R_c>, ||R_c||^2, and per tile <S,S>, <S,Y>, <Y,Y>,
// ||K||^2, ||G||^2, <X,G> for the Barzilai-Borwein step (Section 5.1), with
// S_c = (1 - nu^{k-1}_c) X^k_c - R^{k-1}_c / eta^{k-1}, Y = R^k - R^{k-1}.
//
// One CTA computes a 128-row x N-column tile of both products, with both
// accumulators (and their running totals) in tensor memory.  X is column-major,
// so for this product its contiguous index (the row) is an M index, not the
// contraction index.  TMA lands each 128-row x 32-column slice of X as it is,
// and converter warps transpose it into the canonical K-major 128-byte-swizzle
// layout while rounding it to nearest TF32 (and splitting off the TF32
// remainder in compensated mode), so that every MMA operand uses the K-major
// form.  M and Psi(C) arrive from a small kernel that stores their rounded
// TF32 parts (hi, lo) once per iteration, and TMA loads those in K-major form.
//   warp 0, one thread : TMA producer
//   warp 1, one thread : MMA issuer (2 products x 1 or 3 MMAs per 8 inner indices)
//   warps 2-3          : converters (transpose + round + split of X)
//   warps 4-7          : accumulator warps; epilogue
// Compensated (3xTF32) mode sums each 32-index segment from zero and adds it
// into the running total with round-to-nearest FP32 arithmetic, because the
// tensor-core accumulator truncates (see the Gram kernel).
//
// Every mbarrier wait is bounded; an expired wait raises *err, the CTA lets
// its copies in flight land, frees its tensor memory and returns.
#include "plam_device.cuh"
#include "tc_ptx.cuh"

namespace plam {

constexpr int kUpM = 128;          // rows of X per tile (TMEM lanes)
constexpr int kUpK = 32;           // inner indices per stage
constexpr int kUpThreads = 256;
constexpr int kUpConvThreads = 64;
constexpr int kUpMaxStages = 4;
constexpr int kUpAux = 256;        // barriers, TMEM address, counters

struct TcUpdateArgs {
  int64_t n;
  int p, N, nct;
  const float* X;
  int64_t ldx;
  const float* G;
  int64_t ldg;
  float* R0;
  float* R1;
  int64_t ldr;
  const float* coef;
  const DevState* st;
  float* colpart;
  float* totpart;
  int* err;
  uint32_t pipe_bytes;     // shared memory available to the stages
  double refine_switch;
  int force3;
};

// Sum of v[0..47] over the 32 lanes of a warp by recursive halving (48
// shuffles instead of 240): afterwards each even lane L holds the sums of
// entries b(L) .. b(L) + 2, with b = 24 bit4 + 12 bit3 + 6 bit2 + 3 bit1 of L.
__device__ __forceinline__ void warp_sum48(float (&v)[48], int lane) {
#pragma unroll
  for (int j = 0; j < 24; ++j) {
    const bool up = (lane & 16) != 0;
    const float send = up ? v[j] : v[j + 24];
    const float keep = up ? v[j + 24] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    const bool up = (lane & 8) != 0;
    const float send = up ? v[j] : v[j + 12];
    const float keep = up ? v[j + 12] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const bool up = (lane & 4) != 0;
    const float send = up ? v[j] : v[j + 6];
    const float keep = up ? v[j + 6] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const bool up = (lane & 2) != 0;
    const float send = up ? v[j] : v[j + 3];
    const float keep = up ? v[j + 3] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 1);
}

__device__ __forceinline__ uint32_t up_stage_bytes(int N, bool split) {
  const uint32_t XR = kUpM * kUpK * 4, A = kUpM * kUpK * 4, BT = (uint32_t)N * kUpK * 4;
  return split ? XR + 2 * A + 4 * BT : XR + A + 2 * BT;
}

__global__ void __launch_bounds__(kUpThreads, 1)
tc_update_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapMh,
                 const __grid_constant__ CUtensorMap mapMl, const __grid_constant__ CUtensorMap mapLh,
                 const __grid_constant__ CUtensorMap mapLl, TcUpdateArgs a) {
  if (a.st->stop != kRunning) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t pad = (1024u - (smem_addr(smem_raw) & 1023u)) & 1023u;
  unsigned char* base = smem_raw + pad;
  const bool split = a.force3 || (a.refine_switch > 0.0 && a.st->k > 0 &&
                                  a.st->kkt < a.refine_switch);
  const int N = a.N;
  const uint32_t XR = kUpM * kUpK * 4, AB = kUpM * kUpK * 4, BT = (uint32_t)N * kUpK * 4;
  const uint32_t STAGE = up_stage_bytes(N, split);
  int nst = (int)(a.pipe_bytes / STAGE);
  if (nst > kUpMaxStages) nst = kUpMaxStages;
  // stage layout: [X as landed][A hi][A lo][B1 hi][B2 hi][B1 lo][B2 lo] (lo parts: split only)
  const uint32_t oAh = XR, oAl = XR + AB;
  const uint32_t oB1h = split ? XR + 2 * AB : XR + AB;
  const uint32_t oB2h = oB1h + BT, oB1l = oB2h + BT, oB2l = oB1l + BT;
  const uint32_t tx_bytes = XR + (split ? 4 : 2) * BT;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + a.pipe_bytes);
  uint64_t* conv = full + kUpMaxStages;
  uint64_t* empty = conv + kUpMaxStages;
  uint64_t* acc_full = empty + kUpMaxStages;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* done = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* counters = reinterpret_cast<int*>(tmem_slot + 1);   // [issued, consumed]

  const int rb = blockIdx.x / a.nct, ct = blockIdx.x % a.nct;
  const int64_t r0 = (int64_t)rb * kUpM;
  const int c0 = ct * N;
  const int KT = (a.p + kUpK - 1) / kUpK;
  const int nseg = split ? KT : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols = tmem_cols_for(4 * N);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kUpMaxStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], kUpConvThreads);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 128);
    mbar_init(done, 1);
    counters[0] = 0;
    counters[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM columns: [acc X M][acc X Psi(C)][total X M][total X Psi(C)]
  const uint32_t cAcc1 = 0, cAcc2 = (uint32_t)N, cTot1 = 2u * N, cTot2 = 3u * N;

  if (warp == 0 && lane == 0) {
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % nst;
      const uint32_t ph = (uint32_t)(kt / nst) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, a.err)) break;
      unsigned char* sb = base + s * STAGE;
      mbar_arrive_expect_tx(&full[s], tx_bytes);
      const int k0 = kt * kUpK;
      tma_load_2d(sb, &mapX, &full[s], (int)r0, k0);
      tma_load_2d(sb + oB1h, &mapMh, &full[s], k0, c0);
      tma_load_2d(sb + oB2h, &mapLh, &full[s], k0, c0);
      if (split) {
        tma_load_2d(sb + oB1l, &mapMl, &full[s], k0, c0);
        tma_load_2d(sb + oB2l, &mapLl, &full[s], k0, c0);
      }
      counters[0] = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_tf32(kUpM, N);
    for (int kt = 0; kt < KT; ++kt) {
      const int seg = split ? kt : 0;
      const bool first = split || kt == 0;
      if (split && seg >= 1) {   // the accumulator warps have added the previous segment
        if (!mbar_wait(acc_empty, (uint32_t)(seg - 1) & 1u, a.err)) break;
        tc_fence_after();
      }
      const int s = kt % nst;
      const uint32_t ph = (uint32_t)(kt / nst) & 1u;
      if (!mbar_wait(&conv[s], ph, a.err)) break;
      tc_fence_after();
      const uint32_t sb = smem_addr(base + s * STAGE);
      const uint64_t ah = sdesc_k_sw128(sb + oAh), al = sdesc_k_sw128(sb + oAl);
      const uint64_t m1h = sdesc_k_sw128(sb + oB1h), m2h = sdesc_k_sw128(sb + oB2h);
      const uint64_t m1l = sdesc_k_sw128(sb + oB1l), m2l = sdesc_k_sw128(sb + oB2l);
#pragma unroll
      for (int k = 0; k < kUpK / 8; ++k) {
        const uint32_t acc = (first && k == 0) ? 0u : 1u;
        mma_tf32(tmem + cAcc1, ah + 2 * k, m1h + 2 * k, idesc, acc);
        mma_tf32(tmem + cAcc2, ah + 2 * k, m2h + 2 * k, idesc, acc);
        if (split) {
          mma_tf32(tmem + cAcc1, ah + 2 * k, m1l + 2 * k, idesc, 1);
          mma_tf32(tmem + cAcc1, al + 2 * k, m1h + 2 * k, idesc, 1);
          mma_tf32(tmem + cAcc2, ah + 2 * k, m2l + 2 * k, idesc, 1);
          mma_tf32(tmem + cAcc2, al + 2 * k, m2h + 2 * k, idesc, 1);
        }
      }
      mma_commit(&empty[s]);
      if (split || kt == KT - 1) mma_commit(acc_full);
      counters[1] = kt + 1;
    }
    mma_commit(done);
  } else if (warp == 2 || warp == 3) {
    // converters: X slice [32 columns][128 rows] -> K-major SW128 [128 rows][32 columns]
    const int tid = threadIdx.x - 64;
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % nst;
      const uint32_t ph = (uint32_t)(kt / nst) & 1u;
      if (!mbar_wait(&full[s], ph, a.err)) break;
      unsigned char* sb = base + s * STAGE;
      const float* xr = reinterpret_cast<const float*>(sb);
      for (int it = tid; it < kUpM * (kUpK / 4); it += kUpConvThreads) {
        const int m = it & (kUpM - 1), j = it >> 7;   // row, 16-byte chunk of 4 columns
        const float x0 = xr[(4 * j + 0) * kUpM + m], x1 = xr[(4 * j + 1) * kUpM + m];
        const float x2 = xr[(4 * j + 2) * kUpM + m], x3 = xr[(4 * j + 3) * kUpM + m];
        float4 h;
        h.x = __uint_as_float(tf32_rna(x0));
        h.y = __uint_as_float(tf32_rna(x1));
        h.z = __uint_as_float(tf32_rna(x2));
        h.w = __uint_as_float(tf32_rna(x3));
        const uint32_t off = (uint32_t)(m >> 3) * 1024u + (uint32_t)(m & 7) * 128u +
                             (uint32_t)((j ^ (m & 7)) * 16);
        *reinterpret_cast<float4*>(sb + oAh + off) = h;
        if (split) {
          float4 l;
          l.x = __uint_as_float(tf32_rna(x0 - h.x));
          l.y = __uint_as_float(tf32_rna(x1 - h.y));
          l.z = __uint_as_float(tf32_rna(x2 - h.z));
          l.w = __uint_as_float(tf32_rna(x3 - h.w));
          *reinterpret_cast<float4*>(sb + oAl + off) = l;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&conv[s]))
                   : "memory");
    }
  } else if (warp >= 4) {
    const int q = warp - 4;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int64_t r = r0 + q * 32 + lane;
    const bool row_ok = r < a.n;
    bool ok = true;
    for (int seg = 0; seg < nseg - 1; ++seg) {   // compensated mode: add the segment into the totals
      if (!mbar_wait_warp(acc_full, (uint32_t)seg & 1u, a.err)) { ok = false; break; }
      tc_fence_after();
      for (int j0 = 0; j0 < N; j0 += 16) {
        uint32_t v1[16], t1[16], v2[16], t2[16];
        tmem_ld16_nw(tmem + lane_off + cAcc1 + j0, v1);
        tmem_ld16_nw(tmem + lane_off + cAcc2 + j0, v2);
        if (seg > 0) {
          tmem_ld16_nw(tmem + lane_off + cTot1 + j0, t1);
          tmem_ld16_nw(tmem + lane_off + cTot2 + j0, t2);
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (seg > 0) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            v1[c] = __float_as_uint(__fadd_rn(__uint_as_float(t1[c]), __uint_as_float(v1[c])));
            v2[c] = __float_as_uint(__fadd_rn(__uint_as_float(t2[c]), __uint_as_float(v2[c])));
          }
        }
        tmem_st16(tmem + lane_off + cTot1 + j0, v1);
        tmem_st16(tmem + lane_off + cTot2 + j0, v2);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(acc_empty))
                   : "memory");
    }
    // every accumulator warp reaches the named barrier below exactly once
    int* bad = reinterpret_cast<int*>(counters + 2);
    if (threadIdx.x == 128) *bad = 0;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    ok = ok && mbar_wait_warp(acc_full, (uint32_t)(nseg - 1) & 1u, a.err);
    if (!ok && lane == 0) *bad = 1;
    {
      tc_fence_after();
      // epilogue; the stage buffers are idle now and hold the cross-warp sums
      float* colred = reinterpret_cast<float*>(base);              // [4][3][N]
      float* wsum = colred + 4 * 3 * N;                            // [4][6]
      const int k = a.st->k;
      float* R = (k & 1) ? a.R1 : a.R0;
      const float* Rp = (k & 1) ? a.R0 : a.R1;
      const float* cprev = a.coef + (size_t)((k + 1) & 1) * (2 * a.p + 1);
      const float inv_etap = k > 0 ? cprev[0] : 0.f;
      float ss = 0.f, sy = 0.f, yy = 0.f, kk = 0.f, gg = 0.f, xg = 0.f;
      for (int j0 = 0; ok && j0 < N; j0 += 16) {
        uint32_t v1[16], t1[16], v2[16], t2[16];
        tmem_ld16_nw(tmem + lane_off + cAcc1 + j0, v1);
        tmem_ld16_nw(tmem + lane_off + cAcc2 + j0, v2);
        if (nseg > 1) {
          tmem_ld16_nw(tmem + lane_off + cTot1 + j0, t1);
          tmem_ld16_nw(tmem + lane_off + cTot2 + j0, t2);
        }
        // all global loads of the chunk in flight together (one CTA per SM: the
        // epilogue hides latency by independent loads, not by other warps)
        float xv[16], gv[16], rpv[16], om[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = c0 + j0 + c;
          const bool v = row_ok && col < a.p;
          xv[c] = v ? __ldg(a.X + r + (int64_t)col * a.ldx) : 0.f;
          gv[c] = v ? __ldg(a.G + r + (int64_t)col * a.ldg) : 0.f;
        }
        if (k > 0) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int col = c0 + j0 + c;
            const bool v = row_ok && col < a.p;
            rpv[c] = v ? __ldg(Rp + r + (int64_t)col * a.ldr) : 0.f;
            om[c] = col < a.p ? __ldg(cprev + 1 + a.p + col) : 0.f;
          }
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c) { rpv[c] = 0.f; om[c] = 0.f; }
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float dv[48];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          float d1 = __uint_as_float(v1[c]), d2 = __uint_as_float(v2[c]);
          if (nseg > 1) {
            d1 = __fadd_rn(__uint_as_float(t1[c]), d1);
            d2 = __fadd_rn(__uint_as_float(t2[c]), d2);
          }
          const int col = c0 + j0 + c;
          float xx = 0.f, xrv = 0.f, rr = 0.f;
          if (row_ok && col < a.p) {
            const float x = xv[c], g = gv[c];
            const float rv = g - d1;
            const float kv = g - d2;
            R[r + (int64_t)col * a.ldr] = rv;
            xx = x * x;
            xrv = x * rv;
            rr = rv * rv;
            kk = fmaf(kv, kv, kk);
            gg = fmaf(g, g, gg);
            xg = fmaf(x, g, xg);
            if (k > 0) {
              const float rp = rpv[c];
              const float sv = om[c] * x - rp * inv_etap;
              const float yv = rv - rp;
              ss = fmaf(sv, sv, ss);
              sy = fmaf(sv, yv, sy);
              yy = fmaf(yv, yv, yy);
            }
          }
          dv[c] = xx;
          dv[16 + c] = xrv;
          dv[32 + c] = rr;
        }
        warp_sum48(dv, lane);
        if ((lane & 1) == 0) {
          const int b = 24 * ((lane >> 4) & 1) + 12 * ((lane >> 3) & 1) + 6 * ((lane >> 2) & 1) +
                        3 * ((lane >> 1) & 1);
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const int idx = b + e, d = idx >> 4, c = idx & 15;
            colred[(q * 3 + d) * N + j0 + c] = dv[e];
          }
        }
      }
      float tot[kTotDots] = {ss, sy, yy, kk, gg, xg};
#pragma unroll
      for (int d = 0; d < kTotDots; ++d) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot[d] += __shfl_xor_sync(0xffffffffu, tot[d], o);
      }
      if (ok && lane == 0) {
#pragma unroll
        for (int d = 0; d < kTotDots; ++d) wsum[q * kTotDots + d] = tot[d];
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");   // the four accumulator warps
      const int t = threadIdx.x - 128;
      const bool all_ok = *(volatile int*)bad == 0;
      for (int j = t; all_ok && j < N; j += 128) {
        const int col = c0 + j;
        if (col < a.p) {
          float* cp = a.colpart + (size_t)rb * kColDots * a.p;
#pragma unroll
          for (int d = 0; d < 3; ++d)
            cp[(size_t)d * a.p + col] = ((colred[(0 * 3 + d) * N + j] + colred[(1 * 3 + d) * N + j]) +
                                         colred[(2 * 3 + d) * N + j]) + colred[(3 * 3 + d) * N + j];
        }
      }
      if (all_ok && t < kTotDots)
        a.totpart[((size_t)rb * a.nct + ct) * kTotDots + t] =
            ((wsum[t] + wsum[kTotDots + t]) + wsum[2 * kTotDots + t]) + wsum[3 * kTotDots + t];
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (long long i = 0; i < kTcSpin && !mbar_try_wait(done, 0); ++i) {
    }
    for (int kt = counters[1]; kt < counters[0]; ++kt) {
      const int s = kt % nst;
      const uint32_t ph = (uint32_t)(kt / nst) & 1u;
      for (long long i = 0; i < kTcSpin && !mbar_try_wait(&full[s], ph); ++i) {
      }
    }
  }
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
}

// Rounded TF32 parts of M and Psi(C) (p x p, column-major, leading dimension
// p in the solver's buffers) into hi / lo arrays with leading dimension ldm:
// hi = RN_tf32(v), lo = RN_tf32(v - hi).
__global__ void tc_split_m_kernel(int p, const float* __restrict__ Mt, const float* __restrict__ L0t,
                                  int ldm, float* __restrict__ out, const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  const size_t plane = (size_t)ldm * p;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p * p; i += gridDim.x * blockDim.x) {
    const int r = i % p, c = i / p;
    const float m = Mt[i], l = L0t[i];
    const float mh = __uint_as_float(tf32_rna(m)), lh = __uint_as_float(tf32_rna(l));
    const size_t o = (size_t)c * ldm + r;
    out[o] = mh;
    out[plane + o] = __uint_as_float(tf32_rna(m - mh));
    out[2 * plane + o] = lh;
    out[3 * plane + o] = __uint_as_float(tf32_rna(l - lh));
  }
}

// ---------------------------------------------------------------- host side

static uint32_t up_stage_bytes_host(int N, bool split) {
  const uint32_t XR = kUpM * kUpK * 4, A = kUpM * kUpK * 4, BT = (uint32_t)N * kUpK * 4;
  return split ? XR + 2 * A + 4 * BT : XR + A + 2 * BT;
}

void tc_update_plan(int64_t n, int p, TcUpdatePlan* pl) {
  pl->N = p >= 128 ? 128 : ((p + 15) / 16) * 16;
  pl->nct = (p + pl->N - 1) / pl->N;
  pl->nrt = (int)((n + kUpM - 1) / kUpM);
  pl->ldm = ((p + 31) / 32) * 32;
  // stages: as many as fit (at most 4), with at least two in compensated mode
  const size_t limit = 232448 - 1024 - kUpAux;
  const uint32_t s3 = up_stage_bytes_host(pl->N, true);
  size_t pipe = 2 * (size_t)s3;
  const uint32_t s1 = up_stage_bytes_host(pl->N, false);
  size_t plain = (size_t)s1 * (limit / s1 < (size_t)kUpMaxStages ? limit / s1 : kUpMaxStages);
  if (plain > pipe) pipe = plain;
  size_t split4 = (size_t)s3 * (limit / s3 < (size_t)kUpMaxStages ? limit / s3 : kUpMaxStages);
  if (split4 > pipe) pipe = split4;
  pl->pipe_bytes = (uint32_t)pipe;
  pl->smem = 1024 + pipe + kUpAux;
}

bool tc_update_supported(const void* X, int64_t ldx) {
  return tma_encoder_available() && ((uintptr_t)X % 16) == 0 && (ldx % 4) == 0;
}

cudaError_t launch_tc_update(int64_t n, int p, const float* X, int64_t ldx, const float* G,
                             int64_t ldg, float* R0, float* R1, int64_t ldr, const float* Mt,
                             const float* L0t, const TcUpdatePlan& pl, float* msplit,
                             const float* coef, const DevState* st, float* colpart,
                             float* totpart, int* err, double refine_switch, int force3,
                             cudaStream_t s) {
  {
    int blocks = (p * p + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    tc_split_m_kernel<<<blocks, 256, 0, s>>>(p, Mt, L0t, pl.ldm, msplit, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t plane = (size_t)pl.ldm * p;
  CUtensorMap mX, mMh, mMl, mLh, mLl;
  if (!encode_map_f32(&mX, X, (uint64_t)n, (uint64_t)p, (uint64_t)ldx, kUpM, kUpK, false) ||
      !encode_map_f32(&mMh, msplit, p, p, pl.ldm, kUpK, pl.N, true) ||
      !encode_map_f32(&mMl, msplit + plane, p, p, pl.ldm, kUpK, pl.N, true) ||
      !encode_map_f32(&mLh, msplit + 2 * plane, p, p, pl.ldm, kUpK, pl.N, true) ||
      !encode_map_f32(&mLl, msplit + 3 * plane, p, p, pl.ldm, kUpK, pl.N, true))
    return cudaErrorInvalidValue;
  TcUpdateArgs a;
  a.n = n; a.p = p; a.N = pl.N; a.nct = pl.nct;
  a.X = X; a.ldx = ldx; a.G = G; a.ldg = ldg; a.R0 = R0; a.R1 = R1; a.ldr = ldr;
  a.coef = coef; a.st = st; a.colpart = colpart; a.totpart = totpart; a.err = err;
  a.pipe_bytes = pl.pipe_bytes; a.refine_switch = refine_switch; a.force3 = force3;
  cudaError_t e = cudaFuncSetAttribute(tc_update_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  tc_update_kernel<<<pl.nrt * pl.nct, kUpThreads, pl.smem, s>>>(mX, mMh, mMl, mLh, mLl, a);
  return cudaGetLastError();
}

cudaError_t preload_tc_update_kernels() {
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, tc_update_kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncGetAttributes(&at, tc_split_m_kernel);
}

}  // namespace plam
