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
// K is formed as R - X E with E = Psi(C) - M (= beta (B - I) - Diag(d)), which
// vanishes as the iterate converges: X E is then small against R and G, so it
// is taken in plain TF32 while X M is compensated (3xTF32) near convergence.
//
// The tensor cores' FP32 accumulation truncates (round toward zero), so a long
// sum loses up to an ulp of its running value per step.  M is dominated by its
// diagonal (Lambda's eigenvalue-like diagonal near a solution), so the MMAs
// take M without its diagonal and the epilogue adds X_rc M_cc in round-to-
// nearest FP32: R = G - fma(X, diag(M), acc).  The truncated running sums then
// carry only the off-diagonal terms, which at p = 1000 lowers the floor of the
// relative KKT value from ~1e-6 (and ~6e-6 with a dense Lambda) to the level of
// the CUDA-core FP32 update.
//
// Persistent and warp-specialised: one CTA per SM walks 128-row x N-column
// tiles of R; its tensor memory holds two tiles' accumulators (X M, X E), so
// the epilogue of one tile overlaps the loads and MMAs of the next.
//   warp 0, one thread   : TMA producer of the K-loop stages
//   warp 1, one thread   : MMA issuer
//   warps 2, 3, 8, 9     : converters.  X is column-major, so for this product
//                          its contiguous index (the row) is an M index; TMA
//                          lands each 128-row x 32-column slice as it is and
//                          the converters transpose it in place into the
//                          canonical K-major 128-byte-swizzle layout, rounded
//                          to nearest TF32 (and split into hi + lo when
//                          compensated)
//   warps 4-7, 10-13     : epilogue, two groups of four warps (TMEM lane
//                          quarter = warp mod 4).  The tile's X, G and R^{k-1}
//                          stream through a two-slot ring of 16-column TMA
//                          copies; group e takes the chunks in slot e (every
//                          other chunk), so two warps per scheduler share the
//                          epilogue arithmetic
// M (without its diagonal), its TF32 remainder, E and diag(M) arrive from a
// small kernel that stores them once per iteration.
//
// Every wait is bounded; an expired wait raises *err, every role leaves its
// loop at the same point of the protocol, the CTA lets its copies in flight
// land, frees its tensor memory and returns.
#include "plam_device.cuh"
#include "tc_ptx.cuh"

namespace plam {

constexpr int kUpM = 128;          // rows of X per tile (TMEM lanes)
constexpr int kUpK = 32;           // inner indices per stage
constexpr int kUpThreads = 448;    // 14 warps
constexpr int kUpConvThreads = 128;
constexpr int kUpMaxStages = 6;
constexpr int kUpChunk = 16;       // epilogue columns per ring slot
constexpr int kUpAux = 256;        // barriers, TMEM address, flags

struct TcUpdateArgs {
  int64_t n;
  int p, N, nct, ntiles;
  float* R0;
  float* R1;
  int64_t ldr;
  const float* coef;
  const DevState* st;
  float* colpart;
  float* totpart;
  int* err;
  uint32_t pipe_bytes;     // shared memory of the K-loop stages
  double refine_switch;
  int force3;
  const float* mdiag;      // M_cc, c < p (FP32), added by the epilogue
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

// Stage layout (bytes): plain [A hi = landed X][M hi][E hi];
// compensated [A hi][A lo = landed X][M hi][E hi][M lo].
__host__ __device__ inline uint32_t up_stage_bytes(int N, bool split) {
  const uint32_t A = kUpM * kUpK * 4, BT = (uint32_t)N * kUpK * 4;
  return split ? 2 * A + 3 * BT : A + 2 * BT;
}
__host__ __device__ inline uint32_t up_ring_bytes() { return 2u * 3u * kUpM * kUpChunk * 4u; }
__host__ __device__ inline uint32_t up_red_bytes(int N) { return (12u * N + 48u) * 4u; }

__device__ __forceinline__ void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Converter thread index (0..127) of warps 2, 3, 8, 9.
__device__ __forceinline__ int conv_tid(int warp, int lane) {
  return (warp < 8 ? warp - 2 : warp - 6) * 32 + lane;
}

// kPair = false: one CTA per 128-row x N-column tile.  kPair = true: a cluster of two CTAs
// per 256-row x N-column tile (tcgen05 cta_group::2, M = 256): each CTA stages and transposes
// its own 128 rows of X and N / 2 columns of M, E (and M lo), the even CTA issues the pair's
// MMAs and its commits release stages and accumulators in both CTAs, and each CTA's epilogue
// finishes its own 128 rows exactly as a single CTA does.  Per multiply-add this halves the
// bytes of the M / E operands each SM loads and reads, and a quarter of all its shared-memory
// traffic per stage.
template <bool kPair>
__global__ void __launch_bounds__(kUpThreads, 1)
tc_update_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapMh,
                 const __grid_constant__ CUtensorMap mapMl, const __grid_constant__ CUtensorMap mapEh,
                 const __grid_constant__ CUtensorMap mapXe, const __grid_constant__ CUtensorMap mapGe,
                 const __grid_constant__ CUtensorMap mapR0e, const __grid_constant__ CUtensorMap mapR1e,
                 TcUpdateArgs a) {
  if (a.st->stop != kRunning) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t pad = (1024u - (smem_addr(smem_raw) & 1023u)) & 1023u;
  unsigned char* base = smem_raw + pad;
  const bool split = a.force3 || (a.refine_switch > 0.0 && a.st->refine);
  const int N = a.N;
  const int NB = kPair ? N / 2 : N;                  // columns of M / E staged by this CTA
  const uint32_t A = kUpM * kUpK * 4, BT = (uint32_t)NB * kUpK * 4;
  const uint32_t STAGE = up_stage_bytes(NB, split);
  int nst = (int)(a.pipe_bytes / STAGE);
  if (nst > kUpMaxStages) nst = kUpMaxStages;
  const uint32_t oAh = 0, oAl = A, oRaw = split ? A : 0;
  const uint32_t oB1h = split ? 2 * A : A, oB2h = oB1h + BT, oB1l = oB2h + BT;
  const uint32_t tx_bytes = A + (split ? 3u : 2u) * BT;
  unsigned char* ring = base + a.pipe_bytes;                        // [2 slots][X | G | R^{k-1}]
  const uint32_t EPC = kUpM * kUpChunk * 4;                          // one 128 x 16 operand chunk
  float* colred = reinterpret_cast<float*>(ring + up_ring_bytes());  // [4][3][N]
  float* wsum = colred + 12 * N;                                     // [8][6]
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(colred) +
                                               up_red_bytes(N));
  uint64_t* conv = full + kUpMaxStages;
  uint64_t* empty = conv + kUpMaxStages;
  uint64_t* tfull = empty + kUpMaxStages;    // [2] accumulators of a tile complete
  uint64_t* tempty = tfull + 2;              // [2] epilogue has read them
  uint64_t* epfull = tempty + 2;             // [2] ring slot landed
  uint64_t* done = epfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* flags = reinterpret_cast<int*>(tmem_slot + 1);   // [epilogue abort, converter abort,
                                                        //  stages issued, chunks issued into
                                                        //  ring slot 0, into slot 1]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KT = (a.p + kUpK - 1) / kUpK;
  // tiles of this CTA (of its pair): rows rtile * kRows .. + kRows - 1, columns ctile * N ..;
  // this CTA's own rows start at rtile * kRows + rank * kUpM
  constexpr int kRows = kPair ? 2 * kUpM : kUpM;
  const uint32_t rank = kPair ? cluster_ctarank() : 0u;
  const int unit = kPair ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int nunits = kPair ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int ntl = (a.ntiles - unit + nunits - 1) / nunits;
  const int nrt128 = (int)((a.n + kUpM - 1) / kUpM);   // 128-row tiles of the partial dots
  const uint32_t ncols = tmem_cols_for(4 * N);
  const int kst = a.st->k;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kUpMaxStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], kPair ? 8 : 4);   // one arrival per converter warp (of both CTAs)
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kPair ? 16 : 8);   // one arrival per epilogue warp (of both CTAs)
      mbar_init(&epfull[b], 1);
    }
    mbar_init(done, 1);
    flags[0] = 0; flags[1] = 0; flags[2] = 0; flags[3] = 0; flags[4] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    if constexpr (kPair) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_addr(tmem_slot)),
                   "r"(ncols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_addr(tmem_slot)),
                   "r"(ncols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  if constexpr (kPair) {
    cluster_sync_all();   // both CTAs' barriers initialised and TMEM allocated
  } else {
    __syncthreads();
  }
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: the K-loop stages of every tile of this CTA
      int gs = 0;
      bool ok = true;
      for (int lt = 0; lt < ntl && ok; ++lt) {
        const int tile = unit + lt * nunits;
        const int r0 = (tile / a.nct) * kRows + (int)rank * kUpM;
        const int c0 = (tile % a.nct) * N + (int)rank * NB;
        for (int kt = 0; kt < KT; ++kt, ++gs) {
          const int s = gs % nst;
          if (!mbar_wait(&empty[s], ((uint32_t)(gs / nst) & 1u) ^ 1u, a.err)) { ok = false; break; }
          unsigned char* sb = base + s * STAGE;
          mbar_arrive_expect_tx(&full[s], tx_bytes);
          const int k0 = kt * kUpK;
          tma_load_2d(sb + oRaw, &mapX, &full[s], r0, k0);
          tma_load_2d(sb + oB1h, &mapMh, &full[s], k0, c0);
          tma_load_2d(sb + oB2h, &mapEh, &full[s], k0, c0);
          if (split) tma_load_2d(sb + oB1l, &mapMl, &full[s], k0, c0);
          flags[2] = gs + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---- MMA issuer (the even CTA of a pair)
      const uint32_t idesc = idesc_tf32(kPair ? 2 * kUpM : kUpM, N);
      int gs = 0;
      bool ok = true;
      for (int lt = 0; lt < ntl && ok; ++lt) {
        const int b = lt & 1;
        if (lt >= 2) {
          if (!mbar_wait(&tempty[b], (uint32_t)((lt >> 1) - 1) & 1u, a.err)) break;
          tc_fence_after();
        }
        const uint32_t d1 = tmem + (uint32_t)(b * 2 * N), d2 = d1 + (uint32_t)N;
        for (int kt = 0; kt < KT; ++kt, ++gs) {
          const int s = gs % nst;
          if (!mbar_wait(&conv[s], (uint32_t)(gs / nst) & 1u, a.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sb = smem_addr(base + s * STAGE);
          const uint64_t ah = sdesc_k_sw128(sb + oAh), al = sdesc_k_sw128(sb + oAl);
          const uint64_t mh = sdesc_k_sw128(sb + oB1h), eh = sdesc_k_sw128(sb + oB2h);
          const uint64_t ml = sdesc_k_sw128(sb + oB1l);
#pragma unroll
          for (int k = 0; k < kUpK / 8; ++k) {
            const uint32_t acc = (kt | k) != 0 ? 1u : 0u;
            if constexpr (kPair) {
              mma_tf32_pair(d1, ah + 2 * k, mh + 2 * k, idesc, acc);
              mma_tf32_pair(d2, ah + 2 * k, eh + 2 * k, idesc, acc);
              if (split) {
                mma_tf32_pair(d1, ah + 2 * k, ml + 2 * k, idesc, 1);
                mma_tf32_pair(d1, al + 2 * k, mh + 2 * k, idesc, 1);
              }
            } else {
              mma_tf32(d1, ah + 2 * k, mh + 2 * k, idesc, acc);
              mma_tf32(d2, ah + 2 * k, eh + 2 * k, idesc, acc);
              if (split) {
                mma_tf32(d1, ah + 2 * k, ml + 2 * k, idesc, 1);
                mma_tf32(d1, al + 2 * k, mh + 2 * k, idesc, 1);
              }
            }
          }
          if constexpr (kPair) mma_commit_pair(&empty[s], (uint16_t)3);
          else mma_commit(&empty[s]);
        }
        if (ok) {
          if constexpr (kPair) mma_commit_pair(&tfull[b], (uint16_t)3);
          else mma_commit(&tfull[b]);
        }
      }
      if constexpr (kPair) mma_commit_pair(done, (uint16_t)3);
      else mma_commit(done);
    }
  } else if (warp == 2 || warp == 3 || warp == 8 || warp == 9) {
    // ---- converters: landed X slice [32 columns][128 rows] -> K-major SW128 rows
    const int ct = conv_tid(warp, lane);
    int gs = 0;
    for (int lt = 0; lt < ntl; ++lt) {
      bool abort = false;
      for (int kt = 0; kt < KT; ++kt, ++gs) {
        const int s = gs % nst;
        if (!mbar_wait(&full[s], (uint32_t)(gs / nst) & 1u, a.err)) flags[1] = 1;
        named_bar(2, kUpConvThreads);
        if (*(volatile int*)&flags[1] != 0) { abort = true; break; }
        unsigned char* sb = base + s * STAGE;
        const float* xr = reinterpret_cast<const float*>(sb + oRaw);
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int it = ct + kUpConvThreads * i;
          const int m = it & (kUpM - 1), j = it >> 7;   // row, 16-byte chunk of 4 columns
          v[i].x = xr[(4 * j + 0) * kUpM + m];
          v[i].y = xr[(4 * j + 1) * kUpM + m];
          v[i].z = xr[(4 * j + 2) * kUpM + m];
          v[i].w = xr[(4 * j + 3) * kUpM + m];
        }
        named_bar(2, kUpConvThreads);   // the landed slice is read before it is overwritten
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int it = ct + kUpConvThreads * i;
          const int m = it & (kUpM - 1), j = it >> 7;
          const uint32_t off = (uint32_t)(m >> 3) * 1024u + (uint32_t)(m & 7) * 128u +
                               (uint32_t)((j ^ (m & 7)) * 16);
          float4 h;
          h.x = __uint_as_float(tf32_rna(v[i].x));
          h.y = __uint_as_float(tf32_rna(v[i].y));
          h.z = __uint_as_float(tf32_rna(v[i].z));
          h.w = __uint_as_float(tf32_rna(v[i].w));
          *reinterpret_cast<float4*>(sb + oAh + off) = h;
          if (split) {
            float4 l;
            l.x = __uint_as_float(tf32_rna(v[i].x - h.x));
            l.y = __uint_as_float(tf32_rna(v[i].y - h.y));
            l.z = __uint_as_float(tf32_rna(v[i].z - h.z));
            l.w = __uint_as_float(tf32_rna(v[i].w - h.w));
            *reinterpret_cast<float4*>(sb + oAl + off) = l;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if constexpr (kPair) mbar_arrive_remote(mapa_shared(smem_addr(&conv[s]), 0));
          else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&conv[s]))
                            : "memory");
        }
      }
      if (abort) break;
    }
  } else {
    // ---- epilogue: group e = 0 (warps 4-7) and e = 1 (warps 10-13).  Every named
    // barrier below is reached by every thread of its group (or of both groups)
    // whatever happens; after an expired wait only the work is skipped, and both
    // groups leave the tile loop together after an all-epilogue barrier.
    const int e = warp >= 10 ? 1 : 0;
    const int q = warp & 3;                    // TMEM lane quarter
    const int et = q * 32 + lane;              // TMEM lane = row in the tile
    const int el = (warp - (e ? 10 : 4)) * 32 + lane;   // 0 .. 127 within the group
    const int ea = e * 128 + el;               // 0 .. 255 over both groups
    const int gbar = e ? 3 : 1;                // named barrier of the group
    const bool leader = el == 0;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int nch = N / kUpChunk;
    float* R = (kst & 1) ? a.R1 : a.R0;
    const CUtensorMap* mapRp = (kst & 1) ? &mapR0e : &mapR1e;
    const float* cprev = a.coef + (size_t)((kst + 1) & 1) * (2 * a.p + 1);
    const float inv_etap = kst > 0 ? cprev[0] : 0.f;
    const uint32_t ep_bytes = (kst > 0 ? 3u : 2u) * EPC;
    // chunk g of this CTA's sequence (tiles in order, nch chunks each) into ring slot g & 1
    auto issue_seq = [&](int g) {
      const int lt2 = g / nch, jj = g - lt2 * nch;
      if (lt2 >= ntl) return;
      const int tile2 = unit + lt2 * nunits;
      const int r0c = (tile2 / a.nct) * kRows + (int)rank * kUpM;
      const int cc = (tile2 % a.nct) * N + jj * kUpChunk;
      unsigned char* sl = ring + (g & 1) * 3 * EPC;
      mbar_arrive_expect_tx(&epfull[g & 1], ep_bytes);
      tma_load_2d(sl, &mapXe, &epfull[g & 1], r0c, cc);
      tma_load_2d(sl + EPC, &mapGe, &epfull[g & 1], r0c, cc);
      if (kst > 0) tma_load_2d(sl + 2 * EPC, mapRp, &epfull[g & 1], r0c, cc);
      flags[3 + (g & 1)] = g + 1;
    };
    if (leader) issue_seq(e);
    bool aborted = false;
    for (int lt = 0; lt < ntl; ++lt) {
      const int tile = unit + lt * nunits;
      const int rb = (tile / a.nct) * (kRows / kUpM) + (int)rank;   // this CTA's 128-row tile
      const int ctl = tile % a.nct;
      const int r0 = rb * kUpM, c0 = ctl * N;
      const int b = lt & 1;
      if (!mbar_wait_warp(&tfull[b], (uint32_t)(lt >> 1) & 1u, a.err) && lane == 0) flags[0] = 1;
      named_bar(4, 256);
      if (*(volatile int*)&flags[0] != 0) break;
      tc_fence_after();
      const int64_t r = (int64_t)r0 + et;
      const bool row_ok = r < a.n;
      const uint32_t t1 = tmem + lane_off + (uint32_t)(b * 2 * N), t2 = t1 + (uint32_t)N;
      float ss = 0.f, sy = 0.f, yy = 0.f, kk = 0.f, gg = 0.f, xg = 0.f;
      // the chunks of this tile whose sequence number has parity e
      const int gbase = lt * nch;
      for (int j = ((gbase & 1) == e) ? 0 : 1; j < nch; j += 2) {
        const int gc = gbase + j;
        if (!aborted && !mbar_wait_warp(&epfull[e], (uint32_t)(gc >> 1) & 1u, a.err)) {
          if (lane == 0) flags[0] = 1;
        }
        named_bar(gbar, 128);
        if (*(volatile int*)&flags[0] != 0) aborted = true;
        if (!aborted) {
          const int j0 = j * kUpChunk;
          uint32_t v1[16], v2[16];
          tmem_ld16_nw(t1 + (uint32_t)j0, v1);
          tmem_ld16_nw(t2 + (uint32_t)j0, v2);
          const float* Xs = reinterpret_cast<const float*>(ring + e * 3 * EPC);
          const float* Gs = Xs + kUpM * kUpChunk;
          const float* Rs = Gs + kUpM * kUpChunk;
          float dv[48];
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int col = c0 + j0 + c;
            float xx = 0.f, xrv = 0.f, rr = 0.f;
            if (row_ok && col < a.p) {
              const float x = Xs[c * kUpM + et], g = Gs[c * kUpM + et];
              const float rv = g - fmaf(x, __ldg(a.mdiag + col), __uint_as_float(v1[c]));
              const float kv = rv - __uint_as_float(v2[c]);
              R[r + (int64_t)col * a.ldr] = rv;
              xx = x * x;
              xrv = x * rv;
              rr = rv * rv;
              kk = fmaf(kv, kv, kk);
              gg = fmaf(g, g, gg);
              xg = fmaf(x, g, xg);
              if (kst > 0) {
                const float rp = Rs[c * kUpM + et];
                const float sv = __ldg(cprev + 1 + a.p + col) * x - rp * inv_etap;
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
            const int bb = 24 * ((lane >> 4) & 1) + 12 * ((lane >> 3) & 1) + 6 * ((lane >> 2) & 1) +
                           3 * ((lane >> 1) & 1);
#pragma unroll
            for (int k3 = 0; k3 < 3; ++k3) {
              const int idx = bb + k3, d = idx >> 4, c = idx & 15;
              colred[(q * 3 + d) * N + j0 + c] = dv[k3];
            }
          }
        }
        named_bar(gbar, 128);   // every warp of the group is done with the slot
        if (leader && !aborted) issue_seq(gc + 2);
      }
      // the accumulators of buffer b are read: the MMA may reuse them
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (kPair) mbar_arrive_remote(mapa_shared(smem_addr(&tempty[b]), 0));
        else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&tempty[b]))
                          : "memory");
      }
      float tot[kTotDots] = {ss, sy, yy, kk, gg, xg};
#pragma unroll
      for (int d = 0; d < kTotDots; ++d) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot[d] += __shfl_xor_sync(0xffffffffu, tot[d], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < kTotDots; ++d) wsum[(e * 4 + q) * kTotDots + d] = tot[d];
      }
      named_bar(4, 256);
      const bool stop_all = *(volatile int*)&flags[0] != 0;
      if (!stop_all && rb < nrt128) {
        for (int jj = ea; jj < N; jj += 256) {
          const int col = c0 + jj;
          if (col < a.p) {
            float* cp = a.colpart + (size_t)rb * kColDots * a.p;
#pragma unroll
            for (int d = 0; d < 3; ++d)
              cp[(size_t)d * a.p + col] = ((colred[(0 * 3 + d) * N + jj] + colred[(1 * 3 + d) * N + jj]) +
                                           colred[(2 * 3 + d) * N + jj]) + colred[(3 * 3 + d) * N + jj];
          }
        }
        if (ea < kTotDots) {
          float t8 = wsum[ea];
          for (int w8 = 1; w8 < 8; ++w8) t8 += wsum[w8 * kTotDots + ea];
          a.totpart[((size_t)rb * a.nct + ctl) * kTotDots + ea] = t8;
        }
      }
      named_bar(4, 256);   // colred / wsum are free for the next tile
      if (stop_all) break;
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    // every issued MMA has completed and every issued copy has landed (bounded waits; in a
    // pair the even CTA's final commit arrives in both CTAs)
    for (long long i = 0; i < kTcSpin && !mbar_try_wait(done, 0); ++i) {
    }
    const int gs_issued = flags[2];
    for (int g = gs_issued > nst ? gs_issued - nst : 0; g < gs_issued; ++g)
      for (long long i = 0; i < kTcSpin && !mbar_try_wait(&full[g % nst], (uint32_t)(g / nst) & 1u);
           ++i) {
      }
    for (int sl = 0; sl < 2; ++sl) {   // the last chunk issued into each ring slot has landed
      const int g = flags[3 + sl] - 1;
      if (g < 0) continue;
      for (long long i = 0; i < kTcSpin && !mbar_try_wait(&epfull[sl], (uint32_t)(g >> 1) & 1u);
           ++i) {
      }
    }
  }
  __syncthreads();
  if constexpr (kPair) {
    tc_fence_before();
    cluster_sync_all();   // the peer no longer reads this CTA's shared memory or arrives here
  }
  if (warp == 2) {
    tc_fence_after();
    if constexpr (kPair) {
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(ncols)
                   : "memory");
    } else {
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(ncols)
                   : "memory");
    }
  }
}

// TF32 parts of M without its diagonal (M' = M - Diag(M)) and of E = Psi(C) - M
// (p x p, column-major, leading dimension p in the solver's buffers) into three
// planes of leading dimension ldm: M' hi = RN_tf32(M'), M' lo = RN_tf32(M' - M' hi),
// E hi = RN_tf32(E); the fourth plane starts with diag(M) in FP32.
__global__ void tc_split_m_kernel(int p, const float* __restrict__ Mt, const float* __restrict__ L0t,
                                  int ldm, float* __restrict__ out, const DevState* __restrict__ st) {
  if (st != nullptr && st->stop != kRunning) return;
  const size_t plane = (size_t)ldm * p;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p * p; i += gridDim.x * blockDim.x) {
    const int r = i % p, c = i / p;
    const float m = Mt[i];
    const float mo = (r == c) ? 0.f : m;
    const float mh = __uint_as_float(tf32_rna(mo));
    const size_t o = (size_t)c * ldm + r;
    out[o] = mh;
    out[plane + o] = __uint_as_float(tf32_rna(mo - mh));
    out[2 * plane + o] = __uint_as_float(tf32_rna(L0t[i] - m));
    if (r == c) out[3 * plane + c] = m;
  }
}

// ---------------------------------------------------------------- host side

void tc_update_plan(int64_t n, int p, TcUpdatePlan* pl, int allow_pair) {
  pl->N = p >= 128 ? 128 : ((p + 15) / 16) * 16;
  pl->nct = (p + pl->N - 1) / pl->N;
  pl->nrt = (int)((n + kUpM - 1) / kUpM);
  pl->ldm = ((p + 31) / 32) * 32;
  pl->pair = 0;
  pl->ncl = 0;
  // stage buffers: what is left after the epilogue ring and the reduction scratch,
  // at most kUpMaxStages stages of either mode (a pair stages N / 2 columns of M and E)
  auto size_pipe = [&](int nb) {
    const size_t fixed = 1024 + up_ring_bytes() + up_red_bytes(pl->N) + kUpAux;
    const size_t avail = 232448 - fixed;
    size_t pipe = 0;
    for (int split = 0; split < 2; ++split) {
      const size_t st = up_stage_bytes(nb, split != 0);
      size_t k = avail / st;
      if (k > (size_t)kUpMaxStages) k = kUpMaxStages;
      if (k * st > pipe) pipe = k * st;
    }
    pl->pipe_bytes = (uint32_t)pipe;
    pl->smem = fixed + pipe;
  };
  if (allow_pair && p >= 256) {
    size_pipe(pl->N / 2);
    int ncl = 0;
    cudaFuncAttributes at;
    if (cudaFuncGetAttributes(&at, tc_update_kernel<true>) == cudaSuccess &&
        cudaFuncSetAttribute(tc_update_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pl->smem) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(2, 1, 1);
      cfg.blockDim = dim3(kUpThreads, 1, 1);
      cfg.dynamicSmemBytes = pl->smem;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cudaOccupancyMaxActiveClusters(&ncl, tc_update_kernel<true>, &cfg) != cudaSuccess) ncl = 0;
    }
    cudaGetLastError();
    if (ncl >= 1) {
      pl->pair = 1;
      pl->ncl = ncl;
      return;
    }
  }
  size_pipe(pl->N);
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
  const uint32_t nb = pl.pair ? (uint32_t)pl.N / 2 : (uint32_t)pl.N;   // M / E columns per CTA
  CUtensorMap mX, mMh, mMl, mEh, mXe, mGe, mR0e, mR1e;
  if (!encode_map_f32(&mX, X, (uint64_t)n, (uint64_t)p, (uint64_t)ldx, kUpM, kUpK, false) ||
      !encode_map_f32(&mMh, msplit, p, p, pl.ldm, kUpK, nb, true) ||
      !encode_map_f32(&mMl, msplit + plane, p, p, pl.ldm, kUpK, nb, true) ||
      !encode_map_f32(&mEh, msplit + 2 * plane, p, p, pl.ldm, kUpK, nb, true) ||
      !encode_map_f32(&mXe, X, (uint64_t)n, (uint64_t)p, (uint64_t)ldx, kUpM, kUpChunk, false) ||
      !encode_map_f32(&mGe, G, (uint64_t)n, (uint64_t)p, (uint64_t)ldg, kUpM, kUpChunk, false) ||
      !encode_map_f32(&mR0e, R0, (uint64_t)n, (uint64_t)p, (uint64_t)ldr, kUpM, kUpChunk, false) ||
      !encode_map_f32(&mR1e, R1, (uint64_t)n, (uint64_t)p, (uint64_t)ldr, kUpM, kUpChunk, false))
    return cudaErrorInvalidValue;
  TcUpdateArgs a;
  a.n = n; a.p = p; a.N = pl.N; a.nct = pl.nct;
  a.ntiles = (pl.pair ? (pl.nrt + 1) / 2 : pl.nrt) * pl.nct;
  a.R0 = R0; a.R1 = R1; a.ldr = ldr;
  a.coef = coef; a.st = st; a.colpart = colpart; a.totpart = totpart; a.err = err;
  a.pipe_bytes = pl.pipe_bytes; a.refine_switch = refine_switch; a.force3 = force3;
  a.mdiag = msplit + 3 * plane;
  if (pl.pair) {
    cudaError_t e = cudaFuncSetAttribute(tc_update_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    const int units = pl.ncl < a.ntiles ? pl.ncl : a.ntiles;   // persistent: one pass of clusters
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * units), 1, 1);
    cfg.blockDim = dim3(kUpThreads, 1, 1);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, tc_update_kernel<true>, mX, mMh, mMl, mEh, mXe, mGe, mR0e, mR1e, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(tc_update_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  int grid = device_sm_count();
  if (grid > a.ntiles) grid = a.ntiles;
  tc_update_kernel<false><<<grid, kUpThreads, pl.smem, s>>>(mX, mMh, mMl, mEh, mXe, mGe, mR0e,
                                                            mR1e, a);
  return cudaGetLastError();
}

cudaError_t preload_tc_update_kernels() {
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, tc_update_kernel<false>);
  if (e != cudaSuccess) return e;
  e = cudaFuncGetAttributes(&at, tc_update_kernel<true>);
  if (e != cudaSuccess) return e;
  return cudaFuncGetAttributes(&at, tc_split_m_kernel);
}

}  // namespace plam
