// Tall-skinny Grams on CTA pairs (tcgen05 cta_group::2, sm_103a): partial sums
// of X^T [X | G] over row chunks for p >= 256 (Table "cost": X^T X and
// grad f^T X), kind::tf32 with FP32 accumulation in tensor memory.
//
// A cluster of two CTAs on the two SMs of a pair computes one 256 x 256 output
// tile (256 columns of X against 256 columns of X or G) over one chunk of rows:
// each CTA stages 128 columns of A and 128 columns of B per 32-row stage, and
// one MMA of the pair (M = 256, N = 256) multiplies both CTAs' A halves by the
// whole B tile, each CTA holding its 128 rows of the accumulator in its own
// tensor memory.  Against one CTA per 128 x 128 tile this halves both the
// operand bytes each SM brings in from L2 per multiply-add and the bytes its
// tensor core reads from shared memory per multiply-add.
//   warp 0, one thread   : TMA producer (both CTAs), ring of 6 (A, B) halves
//                          (3 stages of hi + lo halves in compensated mode)
//   warp 1, one thread   : MMA issuer (even CTA only), 4 pair MMAs (K = 8) per
//                          stage, 12 when compensated; commits release the
//                          stage in both CTAs
//   warps 2-7            : converters (both CTAs): round-to-nearest TF32 (and the
//                          TF32 remainder when compensated), then one arrival per
//                          warp on the even CTA's conversion barrier (CTA-scope
//                          release: no cluster-wide fence per stage)
//   warps 8-15           : accumulator warps (both CTAs): add each finished
//                          accumulation segment of their TMEM lanes into a
//                          running total held in registers (128 columns per
//                          thread), then write the chunk's partials
// Two 256-column accumulator regions fill the 512 TMEM columns, so the tensor
// cores fill one while the other is added; the running totals therefore live
// in registers (setmaxnreg: 176 per accumulator thread, 80 for the others).
// A segment is one stage when compensated and kTc2SegPlain stages otherwise:
// the accumulator of tcgen05.mma rounds toward zero and a long same-signed sum
// drifts low with the number of accumulation steps.
//
// Every mbarrier wait is bounded; after an expired wait the kernel raises *err,
// waits (bounded) for its own copies and MMAs, meets its peer at the final
// cluster barrier (which every path reaches), frees TMEM and returns.
#include <cuda.h>

#include "plam_device.cuh"
#include "tc_ptx.cuh"

namespace plam {

constexpr int kTc2K = 32;            // rows of X per stage
constexpr int kTc2Cols = 128;        // columns of A and of B staged by each CTA
constexpr int kTc2Stages = 6;        // (A, B) halves: 6 plain stages or 3 compensated
constexpr int kTc2Threads = 512;     // 16 warps
constexpr int kTc2SegPlain = 8;      // stages per accumulation segment, plain TF32
constexpr int kTc2RegsLow = 80;      // warps 0-7 after setmaxnreg
constexpr int kTc2RegsHigh = 176;    // warps 8-15 after setmaxnreg
constexpr uint32_t kTc2TmemCols = 512;

struct TcGram2Args {
  int64_t n;
  int p;
  int nsb;               // 256-column blocks of X (and of G)
  int nbt;               // tiles of B = X^T X at or above the diagonal
  int64_t rows_per_chunk;
  float* part;           // nchunks x 2p x p
  int* err;
  const DevState* st;
  double refine_switch;
  int force3;
};

__device__ __forceinline__ void tc2_tile(const TcGram2Args& a, int pair, int& mb, int& nb,
                                         int& isg) {
  if (pair < a.nbt) {
    int rem = pair;
    for (mb = 0; mb < a.nsb; ++mb) {
      const int cnt = a.nsb - mb;
      if (rem < cnt) { nb = mb + rem; break; }
      rem -= cnt;
    }
    isg = 0;
  } else {
    const int idx = pair - a.nbt;
    mb = idx % a.nsb;
    nb = idx / a.nsb;
    isg = 1;
  }
}

// The end of every role: all MMAs of the pair complete (bounded; the even CTA's final commit
// arrives in both CTAs), this CTA's own copies still in flight land after an expired wait,
// both CTAs meet (the peer then no longer reads this CTA's shared memory or arrives on its
// barriers), and TMEM is freed.  Each role calls it at its own end, so that no code after the
// roles runs under two register budgets.
__device__ __forceinline__ void tc2_teardown(uint64_t* done, uint64_t* full, const int* counters,
                                             int nst, uint32_t tmem, int warp) {
  __syncwarp();
  tc_fence_before();
  cta_sync_divergent();
  if (threadIdx.x == 0) {
    for (long long t2 = 0; t2 < kTcSpin && !mbar_try_wait(done, 0); ++t2) {
    }
    for (int kt = counters[1]; kt < counters[0]; ++kt) {
      const int s = kt % nst;
      const uint32_t ph = (uint32_t)(kt / nst) & 1u;
      for (long long t2 = 0; t2 < kTcSpin && !mbar_try_wait(&full[s], ph); ++t2) {
      }
    }
  }
  cta_sync_divergent();
  tc_fence_before();
  cluster_sync_divergent();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTc2TmemCols)
                 : "memory");
  }
}

__global__ void __launch_bounds__(kTc2Threads, 1)
tc_gram2_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapG,
                TcGram2Args a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t pad = (1024u - (smem_addr(smem_raw) & 1023u)) & 1023u;
  unsigned char* base = smem_raw + pad;
  const bool split = a.force3 || (a.refine_switch > 0.0 && a.st != nullptr && a.st->refine);
  constexpr uint32_t HALF_A = kTc2Cols * kTc2K * 4;   // 16 KB: 128 columns x 32 rows
  constexpr uint32_t HALF = 2 * HALF_A;               // this CTA's A half and B half
  const uint32_t STAGE = split ? 2 * HALF : HALF;     // split: hi halves, then lo halves
  const int nst = split ? kTc2Stages / 2 : kTc2Stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kTc2Stages * HALF);
  uint64_t* conv = full + kTc2Stages;
  uint64_t* empty = conv + kTc2Stages;
  uint64_t* acc_full = empty + kTc2Stages;   // [2]
  uint64_t* acc_empty = acc_full + 2;        // [2]
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* counters = reinterpret_cast<int*>(tmem_slot + 1);   // [copies issued, stages seen landed]

  const uint32_t rank = cluster_ctarank();
  int mb, nb, isg;
  tc2_tile(a, (int)(blockIdx.x >> 1), mb, nb, isg);
  const int64_t r0 = (int64_t)blockIdx.y * a.rows_per_chunk;
  const int64_t r1 = min(a.n, r0 + a.rows_per_chunk);
  const int KT = r1 > r0 ? (int)((r1 - r0 + kTc2K - 1) / kTc2K) : 0;
  const int segk = split ? 1 : kTc2SegPlain;
  const int nseg = (KT + segk - 1) / segk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTc2Stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 12);    // one arrival per converter warp of both CTAs
      mbar_init(&empty[s], 1);
    }
    for (int r = 0; r < 2; ++r) {
      mbar_init(&acc_full[r], 1);
      mbar_init(&acc_empty[r], 16);   // one arrival per accumulator warp of both CTAs
    }
    mbar_init(done, 1);
    counters[0] = 0;
    counters[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(kTc2TmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync_all();   // both CTAs' barriers initialised and TMEM allocated
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // Roles branch at warpgroup granularity first (warps 0-7 / 8-15), each branch with its own
  // register budget and its own teardown, so that the compiler allocates each under its limit.
  if (warp < 8) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kTc2RegsLow));
    if (warp == 0) {
      if (lane == 0) {
        // producer: this CTA's 128 columns of A and of B for every stage
        const int ca = mb * 256 + (int)rank * kTc2Cols;
        const int cb = nb * 256 + (int)rank * kTc2Cols;
        const CUtensorMap* mb_map = isg ? &mapG : &mapX;
        for (int kt = 0; kt < KT; ++kt) {
          const int s = kt % nst;
          const uint32_t ph = (uint32_t)(kt / nst) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, a.err)) break;
          unsigned char* sa = base + s * STAGE;
          mbar_arrive_expect_tx(&full[s], HALF);
          const int x = (int)(r0 + (int64_t)kt * kTc2K);
          tma_load_2d(sa, &mapX, &full[s], x, ca);
          tma_load_2d(sa + HALF_A, mb_map, &full[s], x, cb);
          counters[0] = kt + 1;
        }
      }
    } else if (warp == 1) {
      if (lane == 0 && rank == 0) {
        // MMA issuer of the pair
        const uint32_t idesc = idesc_tf32(256, 256);
        for (int kt = 0; kt < KT; ++kt) {
          const int seg = kt / segk;
          const bool first = (kt % segk) == 0;
          const bool last = (kt % segk) == segk - 1 || kt == KT - 1;
          const int r = seg & 1;
          if (first && seg >= 2) {   // both CTAs' accumulator warps have added region r
            if (!mbar_wait(&acc_empty[r], (uint32_t)((seg >> 1) - 1) & 1u, a.err)) break;
            tc_fence_after();
          }
          const int s = kt % nst;
          const uint32_t ph = (uint32_t)(kt / nst) & 1u;
          if (!mbar_wait(&conv[s], ph, a.err)) break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(r * 256);
          const uint32_t sa = smem_addr(base + s * STAGE);
          const uint64_t ah = sdesc_k_sw128(sa), bh = sdesc_k_sw128(sa + HALF_A);
          const uint64_t al = sdesc_k_sw128(sa + HALF), bl = sdesc_k_sw128(sa + HALF + HALF_A);
  #pragma unroll
          for (int k = 0; k < kTc2K / 8; ++k) {   // K = 8 tf32 (32 bytes) per instruction
            mma_tf32_pair(d, ah + 2 * k, bh + 2 * k, idesc, (first && k == 0) ? 0u : 1u);
            if (split) {
              mma_tf32_pair(d, ah + 2 * k, bl + 2 * k, idesc, 1);
              mma_tf32_pair(d, al + 2 * k, bh + 2 * k, idesc, 1);
            }
          }
          mma_commit_pair(&empty[s], (uint16_t)3);
          if (last) mma_commit_pair(&acc_full[r], (uint16_t)3);
        }
        mma_commit_pair(done, (uint16_t)3);   // arrives in both CTAs once every MMA completed
      }
    } else {
      // converters: round to TF32 (and split) this CTA's halves of each landed stage
      const int tid = (warp - 2) * 32 + lane;
      const uint32_t conv_leader = mapa_shared(smem_addr(conv), 0);
      for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % nst;
        const uint32_t ph = (uint32_t)(kt / nst) & 1u;
        if (!mbar_wait_warp(&full[s], ph, a.err)) break;
        if (tid == 0) counters[1] = kt + 1;
        unsigned char* sa = base + s * STAGE;
        convert_tile(reinterpret_cast<float*>(sa), reinterpret_cast<float*>(sa + HALF),
                     (int)(HALF / 16), tid, 192, split);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_remote(conv_leader + (uint32_t)(s * 8));
      }
    }
    tc2_teardown(done, full, counters, nst, tmem, warp);
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kTc2RegsHigh));
    // accumulator warps: warp 8 + 4h + q owns TMEM lanes 32q .. 32q + 31 and columns
    // 128h .. 128h + 127 of this CTA's accumulator rows
    const int q = warp & 3, hcol = (warp - 8) >> 2;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const uint32_t acc_empty_leader = mapa_shared(smem_addr(acc_empty), 0);
    float tot[128];
#pragma unroll
    for (int c = 0; c < 128; ++c) tot[c] = 0.f;
    bool ok = true;
    for (int seg = 0; seg < nseg; ++seg) {
      const int r = seg & 1;
      if (!mbar_wait_warp(&acc_full[r], (uint32_t)(seg >> 1) & 1u, a.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t acc = tmem + lane_off + (uint32_t)(r * 256 + hcol * 128);
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        uint32_t v[32];
        tmem_ld32_nw(acc + (uint32_t)(jj * 32), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 32; ++c)
          tot[jj * 32 + c] = __fadd_rn(tot[jj * 32 + c], __uint_as_float(v[c]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_remote(acc_empty_leader + (uint32_t)(r * 8));
    }
    if (ok) {
      const int gi = mb * 256 + (int)rank * kTc2Cols + q * 32 + lane;
      float* out = a.part + (size_t)blockIdx.y * 2 * a.p * a.p + (size_t)isg * a.p * a.p;
      if (gi < a.p) {
#pragma unroll
        for (int c = 0; c < 128; ++c) {
          const int gj = nb * 256 + hcol * 128 + c;
          if (gj < a.p) out[(size_t)gj * a.p + gi] = tot[c];
        }
      }
    }
    tc2_teardown(done, full, counters, nst, tmem, warp);
  }
}

// ---------------------------------------------------------------- host side

// The pair kernel needs the whole register file at launch (512 threads x 128) for its
// setmaxnreg split (256 x 80 + 256 x 176), and the device must fit a cluster of two.
static int tc_gram2_max_clusters(size_t smem) {
  static int cached = -1;
  static size_t cached_smem = 0;
  if (cached >= 0 && cached_smem == smem) return cached;
  int ncl = 0;
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, tc_gram2_kernel) == cudaSuccess &&
      at.numRegs * kTc2Threads >= 256 * (kTc2RegsLow + kTc2RegsHigh) &&
      cudaFuncSetAttribute(tc_gram2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(kTc2Threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&ncl, tc_gram2_kernel, &cfg) != cudaSuccess) ncl = 0;
  }
  cudaGetLastError();
  cached = ncl;
  cached_smem = smem;
  return ncl;
}

bool tc_gram2_plan(int64_t n, int p, int with_g, TcGramPlan* pl) {
  if (p < 256) return false;
  const size_t smem = 1024 + (size_t)kTc2Stages * 2 * kTc2Cols * kTc2K * 4 + 512;
  const int ncl = tc_gram2_max_clusters(smem);
  if (ncl < 1) return false;
  const int nsb = (p + 255) / 256;
  pl->pair = 1;
  pl->N = 256;
  pl->nmb = nsb;
  pl->nnb = nsb;
  pl->nbt = nsb * (nsb + 1) / 2;
  pl->ntiles = pl->nbt + (with_g ? nsb * nsb : 0);
  // chunks per tile: the fewest that fill at least 94% of whole waves of clusters
  int64_t nch = 1;
  double best = 0.0;
  for (int64_t c = 1; c <= 4 * (int64_t)ncl / pl->ntiles + 1 && c <= 1024; ++c) {
    const int64_t cl = c * pl->ntiles;
    const int64_t waves = (cl + ncl - 1) / ncl;
    const double eff = (double)cl / (double)(waves * ncl);
    if (eff > best + 1e-3) { best = eff; nch = c; }
    if (eff >= 0.94) break;
  }
  const int64_t max_ch = (n + kTc2K - 1) / kTc2K;
  if (nch > max_ch) nch = max_ch;
  if (nch < 1) nch = 1;
  int64_t rows = (n + nch - 1) / nch;
  rows = (rows + kTc2K - 1) / kTc2K * kTc2K;
  pl->rows_per_chunk = rows;
  pl->nchunks = (int)((n + rows - 1) / rows);
  pl->smem = smem;
  return true;
}

cudaError_t launch_tc_gram2(int64_t n, int p, const float* X, int64_t ldx, const float* G,
                            int64_t ldg, const TcGramPlan& pl, float* part, int* err,
                            const DevState* st, double refine_switch, int force3,
                            cudaStream_t s) {
  CUtensorMap mX, mG;
  if (!encode_map_f32(&mX, X, (uint64_t)n, (uint64_t)p, (uint64_t)ldx, kTc2K, kTc2Cols, true))
    return cudaErrorInvalidValue;
  if (G) {
    if (!encode_map_f32(&mG, G, (uint64_t)n, (uint64_t)p, (uint64_t)ldg, kTc2K, kTc2Cols, true))
      return cudaErrorInvalidValue;
  } else {
    mG = mX;
  }
  TcGram2Args a;
  a.n = n; a.p = p; a.nsb = pl.nmb; a.nbt = pl.nbt; a.rows_per_chunk = pl.rows_per_chunk;
  a.part = part; a.err = err; a.st = st; a.refine_switch = refine_switch; a.force3 = force3;
  cudaError_t e = cudaFuncSetAttribute(tc_gram2_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  const int pairs = pl.nbt + (G ? pl.nmb * pl.nmb : 0);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(2 * pairs), (unsigned)pl.nchunks, 1);
  cfg.blockDim = dim3(kTc2Threads, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, tc_gram2_kernel, mX, mG, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t preload_tc_gram2() {
  cudaFuncAttributes at;
  return cudaFuncGetAttributes(&at, tc_gram2_kernel);
}

}  // namespace plam
