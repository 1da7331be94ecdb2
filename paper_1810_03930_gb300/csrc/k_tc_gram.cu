// Tall-skinny Grams on the 5th-generation tensor cores (tcgen05, sm_103a):
// partial sums of X^T [X | G] over row chunks, kind::tf32 with FP32
// accumulation in tensor memory (Table "cost": X^T X and grad f^T X).
//
// One CTA computes one 128 x N output tile (128 columns of X against N
// columns of X or G) over one chunk of rows.  Both operands are K-major (the
// row index of X is the contraction index and is contiguous in column-major
// storage), so a TMA box of 32 rows x 128 (or N) columns with 128-byte
// swizzle lands in shared memory exactly in the canonical K-major SW128
// layout: one 128-byte line per column, 8-line atoms of 1024 bytes.
//   warp 0, one thread : TMA producer, ring of 6 (A, B) pairs (3 stages of
//                        hi + lo pairs in compensated mode)
//   warp 1, one thread : MMA issuer, 4 x tcgen05.mma (K = 8 each) per stage
//                        (12 when compensated), tcgen05.commit releases it
//   warps 2-3, 8-11    : convert each landed stage to round-to-nearest TF32 (and
//                        split it into hi + lo in compensated mode); warp 2
//                        also allocates / frees tensor memory (TMEM)
//   warps 4-7          : accumulator warps: add each finished accumulation
//                        segment into the running total (tcgen05.ld / st) and
//                        write the chunk's tile as float partials
//                        part[chunk][col][row] (the layout of the SIMT Gram,
//                        so the same fixed-order reduction follows)
// Tiles of B = X^T X that lie entirely below the diagonal are skipped.
//
// Every mbarrier wait is bounded (kTcSpin polls); when one expires the
// kernel raises *err, waits (bounded) for the copies it has in flight,
// frees its TMEM and returns; the host reports PLAM_ERR_TIMEOUT.
#include <cuda.h>

#include "plam_device.cuh"
#include "tc_ptx.cuh"

namespace plam {

constexpr int kTcM = 128;          // rows of the accumulator (columns of X per tile)
constexpr int kTcK = 32;           // rows of X per stage (128 bytes of FP32 per line)
constexpr int kTcStages = 6;        // (A, B) pairs of shared memory: 6 plain stages or 3 compensated

struct TcGramArgs {
  int64_t n;
  int p;
  int N;                 // accumulator columns (multiple of 16, <= 256)
  int nmb, nnb;          // 128-column blocks of X, N-column blocks of X / G
  int nbt;               // tiles of B = X^T X that are computed (at or above the diagonal)
  int with_g;
  int64_t rows_per_chunk;
  float* part;           // nchunks x 2p x p
  int* err;
  const DevState* st;    // iteration state (null outside the solver)
  double refine_switch;  // > 0: 3xTF32 once the step kernel latched DevState.refine (<= 0: never)
  int force3;            // 1: always 3xTF32
};

// Tile -> (m-block, n-block, source): the B tiles at or above the diagonal first.
__device__ __forceinline__ void tc_tile(const TcGramArgs& a, int tile, int& mb, int& nb, int& isg) {
  if (tile < a.nbt) {
    int rem = tile;
    for (mb = 0; mb < a.nmb; ++mb) {
      int first = (mb * kTcM) / a.N;          // n-blocks with (nb + 1) N > mb 128
      int cnt = a.nnb - first;
      if (rem < cnt) { nb = first + rem; break; }
      rem -= cnt;
    }
    isg = 0;
  } else {
    const int idx = tile - a.nbt;
    mb = idx % a.nmb;
    nb = idx / a.nmb;
    isg = 1;
  }
}

constexpr int kTcConvThreads = 192;  // warps 2, 3 and 8-11
constexpr int kTcThreads = 384;      // warps 0-11
constexpr int kTcSegSplit = 1;       // stages per accumulation segment in compensated mode

// TMEM columns: nacc accumulator regions of N columns, then one N-column
// running total, rounded up to the power of two that tcgen05.alloc takes.
__host__ __device__ inline int tc_nacc(int N) { return N <= 128 ? 2 : 1; }
__host__ __device__ inline uint32_t tc_tmem_cols(int N) { return tmem_cols_for((tc_nacc(N) + 1) * N); }

// The accumulator of tcgen05.mma rounds toward zero, so a long sum of
// same-signed terms (a diagonal of X^T X) drifts low by about 2^-25 per
// accumulation step relative to the running value.  The kernel therefore sums
// a chunk in segments: each segment starts from zero in an accumulator region
// of TMEM, and the accumulator warps add it, with round-to-nearest FP32
// arithmetic, into a running total that lives in TMEM as well.  Plain TF32
// mode uses one segment per chunk; compensated mode one per kTcSegSplit
// stages, with two accumulator regions when N <= 128 so that the tensor cores
// fill one while the other is added.
__global__ void __launch_bounds__(kTcThreads, 1)
tc_gram_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapXB,
               const __grid_constant__ CUtensorMap mapGB, TcGramArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t pad = (1024u - (smem_addr(smem_raw) & 1023u)) & 1023u;
  unsigned char* base = smem_raw + pad;
  // compensated (3xTF32) mode: decided once per launch from the device state
  const bool split = a.force3 || (a.refine_switch > 0.0 && a.st != nullptr && a.st->refine);
  const uint32_t A_BYTES = kTcM * kTcK * 4;
  const uint32_t B_BYTES = (uint32_t)a.N * kTcK * 4;
  const uint32_t HALF = A_BYTES + B_BYTES;           // one (A, B) pair
  const uint32_t STAGE = split ? 2 * HALF : HALF;   // split: hi pair then lo pair
  const int nst = split ? kTcStages / 2 : kTcStages;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kTcStages * HALF);
  uint64_t* conv = full + kTcStages;
  uint64_t* empty = conv + kTcStages;
  uint64_t* acc_full = empty + kTcStages;    // [2]
  uint64_t* acc_empty = acc_full + 2;        // [2]
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* counters = reinterpret_cast<int*>(tmem_slot + 1);   // [issued, consumed]

  int mb, nb, isg;
  tc_tile(a, blockIdx.x, mb, nb, isg);
  const int64_t r0 = (int64_t)blockIdx.y * a.rows_per_chunk;
  const int64_t r1 = min(a.n, r0 + a.rows_per_chunk);
  const int KT = (int)((r1 - r0 + kTcK - 1) / kTcK);
  const int segk = split ? kTcSegSplit : (KT > 0 ? KT : 1);
  const int nseg = (KT + segk - 1) / segk;
  const int nacc = tc_nacc(a.N);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols = tc_tmem_cols(a.N);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], kTcConvThreads);
      mbar_init(&empty[s], 1);
    }
    for (int r = 0; r < 2; ++r) {
      mbar_init(&acc_full[r], 1);
      mbar_init(&acc_empty[r], 128);
    }
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
  const uint32_t total_col = (uint32_t)(nacc * a.N);

  if (warp == 0 && lane == 0) {
    // producer: TMA of the (A, B) pair of each stage
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % nst;
      const uint32_t ph = (uint32_t)(kt / nst) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, a.err)) break;
      unsigned char* sa = base + s * STAGE;
      mbar_arrive_expect_tx(&full[s], HALF);
      const int x = (int)(r0 + (int64_t)kt * kTcK);
      tma_load_2d(sa, &mapA, &full[s], x, mb * kTcM);
      tma_load_2d(sa + A_BYTES, isg ? &mapGB : &mapXB, &full[s], x, nb * a.N);
      counters[0] = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_tf32(kTcM, a.N);
    bool ok = true;
    for (int kt = 0; kt < KT && ok; ++kt) {
      const int seg = kt / segk;
      const bool first = (kt % segk) == 0;
      const bool last = (kt % segk) == segk - 1 || kt == KT - 1;
      const int r = seg % nacc;
      if (first && seg >= nacc) {   // wait until the accumulator warps have added region r
        if (!mbar_wait(&acc_empty[r], (uint32_t)(seg / nacc - 1) & 1u, a.err)) break;
        tc_fence_after();
      }
      const int s = kt % nst;
      const uint32_t ph = (uint32_t)(kt / nst) & 1u;
      if (!mbar_wait(&conv[s], ph, a.err)) break;
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(r * a.N);
      const uint32_t sa = smem_addr(base + s * STAGE);
      const uint64_t ah = sdesc_k_sw128(sa), bh = sdesc_k_sw128(sa + A_BYTES);
      const uint64_t al = sdesc_k_sw128(sa + HALF), bl = sdesc_k_sw128(sa + HALF + A_BYTES);
#pragma unroll
      for (int k = 0; k < kTcK / 8; ++k) {   // K = 8 tf32 (32 bytes) per instruction
        mma_tf32(d, ah + 2 * k, bh + 2 * k, idesc, (first && k == 0) ? 0u : 1u);
        if (split) {
          mma_tf32(d, ah + 2 * k, bl + 2 * k, idesc, 1);
          mma_tf32(d, al + 2 * k, bh + 2 * k, idesc, 1);
        }
      }
      mma_commit(&empty[s]);
      if (last) mma_commit(&acc_full[r]);
      counters[1] = kt + 1;
    }
    mma_commit(done);   // arrives once every issued MMA has completed
  } else if (warp == 2 || warp == 3 || warp >= 8) {
    // converters: round to TF32 (and split) each landed stage in place
    const int tid = (warp < 8 ? warp - 2 : warp - 6) * 32 + lane;
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % nst;
      const uint32_t ph = (uint32_t)(kt / nst) & 1u;
      if (!mbar_wait(&full[s], ph, a.err)) break;
      unsigned char* sa = base + s * STAGE;
      convert_tile(reinterpret_cast<float*>(sa), reinterpret_cast<float*>(sa + HALF),
                   (int)(HALF / 16), tid, kTcConvThreads, split);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&conv[s]))
                   : "memory");
    }
  } else if (warp >= 4) {
    // accumulator warps: warp 4 + q owns TMEM lanes 32q .. 32q + 31 (rows of D)
    const int q = warp - 4;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int gi = mb * kTcM + q * 32 + lane;
    float* out = a.part + (size_t)blockIdx.y * 2 * a.p * a.p + (size_t)isg * a.p * a.p;
    bool ok = true;
    for (int seg = 0; seg < nseg; ++seg) {
      const int r = seg % nacc;
      if (!mbar_wait_warp(&acc_full[r], (uint32_t)(seg / nacc) & 1u, a.err)) { ok = false; break; }
      tc_fence_after();
      const uint32_t acc = tmem + lane_off + (uint32_t)(r * a.N);
      const uint32_t tot = tmem + lane_off + total_col;
      const bool final_seg = seg == nseg - 1;
      for (int j0 = 0; j0 < a.N; j0 += 16) {
        uint32_t v[16], t[16];
        tmem_ld16_nw(acc + (uint32_t)j0, v);
        if (seg > 0) tmem_ld16_nw(tot + (uint32_t)j0, t);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (seg > 0) {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            v[c] = __float_as_uint(__fadd_rn(__uint_as_float(t[c]), __uint_as_float(v[c])));
        }
        if (final_seg) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int gj = nb * a.N + j0 + c;
            if (gi < a.p && gj < a.p) out[(size_t)gj * a.p + gi] = __uint_as_float(v[c]);
          }
        } else {
          tmem_st16(tot + (uint32_t)j0, v);
        }
      }
      if (!final_seg) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&acc_empty[r]))
                   : "memory");
    }
    if (ok && KT == 0) {   // empty chunk: the partial is zero
      for (int j = 0; j < a.N; ++j) {
        const int gj = nb * a.N + j;
        if (gi < a.p && gj < a.p) out[(size_t)gj * a.p + gi] = 0.f;
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  // every issued MMA has completed (bounded), and after an expired wait the
  // copies still in flight land, before the CTA frees TMEM and exits
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
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool tma_encoder_available() { return encode_fn() != nullptr; }

int device_sm_count() {
  int dev = 0, cnt = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || cnt < 1)
    cnt = 1;
  return cnt;
}

bool encode_map_f32(CUtensorMap* m, const float* ptr, uint64_t dim0, uint64_t dim1, uint64_t ld,
                    uint32_t box0, uint32_t box1, bool swizzle128) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)dim0, (cuuint64_t)dim1};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {box0, box1};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D map of an n x p column-major float matrix: box of 32 rows x `cols` columns, 128-byte swizzle.
static bool encode_map(CUtensorMap* m, const float* ptr, int64_t n, int p, int64_t ld, int cols) {
  return encode_map_f32(m, ptr, (uint64_t)n, (uint64_t)p, (uint64_t)ld, (uint32_t)kTcK,
                        (uint32_t)cols, true);
}

void tc_gram_plan(int64_t n, int p, int with_g, TcGramPlan* pl, int allow_pair) {
  if (allow_pair && tc_gram2_plan(n, p, with_g, pl)) return;
  pl->pair = 0;
  pl->N = p >= 128 ? 128 : ((p + 15) / 16) * 16;
  pl->nmb = (p + kTcM - 1) / kTcM;
  pl->nnb = (p + pl->N - 1) / pl->N;
  int nbt = 0;
  for (int mb = 0; mb < pl->nmb; ++mb) nbt += pl->nnb - (mb * kTcM) / pl->N;
  pl->nbt = nbt;
  pl->ntiles = nbt + (with_g ? pl->nmb * pl->nnb : 0);
  // chunks per tile: the fewest that fill at least 94% of whole waves of one CTA per SM (a
  // last, partial wave costs as much as a full one; every chunk adds 2 p^2 partial sums)
  const int sms = device_sm_count();
  int64_t nch = 1;
  double best = 0.0;
  for (int64_t c = 1; c <= 4 * (int64_t)sms / pl->ntiles + 1 && c <= 1024; ++c) {
    const int64_t ctas = c * pl->ntiles;
    const int64_t waves = (ctas + sms - 1) / sms;
    const double eff = (double)ctas / (double)(waves * sms);
    if (eff > best + 1e-3) { best = eff; nch = c; }
    if (eff >= 0.94) break;
  }
  const int64_t max_ch = (n + kTcK - 1) / kTcK;
  if (nch > max_ch) nch = max_ch;
  if (nch < 1) nch = 1;
  int64_t rows = (n + nch - 1) / nch;
  rows = (rows + kTcK - 1) / kTcK * kTcK;
  pl->rows_per_chunk = rows;
  pl->nchunks = (int)((n + rows - 1) / rows);
  pl->smem = 1024 + (size_t)kTcStages * (kTcM + pl->N) * kTcK * 4 + 512;
}

bool tc_gram_supported(const void* X, int64_t ldx, const void* G, int64_t ldg) {
  return tma_encoder_available() && ((uintptr_t)X % 16) == 0 && (ldx % 4) == 0 &&
         (G == nullptr || (((uintptr_t)G % 16) == 0 && (ldg % 4) == 0));
}

cudaError_t launch_tc_gram(int64_t n, int p, const float* X, int64_t ldx, const float* G,
                           int64_t ldg, const TcGramPlan& pl, float* part, int* err,
                           const DevState* st, double refine_switch, int force3, cudaStream_t s) {
  if (pl.pair)
    return launch_tc_gram2(n, p, X, ldx, G, ldg, pl, part, err, st, refine_switch, force3, s);
  CUtensorMap mA, mXB, mGB;
  if (!encode_map(&mA, X, n, p, ldx, kTcM) || !encode_map(&mXB, X, n, p, ldx, pl.N))
    return cudaErrorInvalidValue;
  if (G) {
    if (!encode_map(&mGB, G, n, p, ldg, pl.N)) return cudaErrorInvalidValue;
  } else {
    mGB = mXB;
  }
  TcGramArgs a;
  a.n = n; a.p = p; a.N = pl.N; a.nmb = pl.nmb; a.nnb = pl.nnb; a.nbt = pl.nbt;
  a.with_g = G != nullptr; a.rows_per_chunk = pl.rows_per_chunk; a.part = part; a.err = err;
  a.st = st; a.refine_switch = refine_switch; a.force3 = force3;
  cudaError_t e = cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)pl.smem);
  if (e != cudaSuccess) return e;
  const int tiles = pl.nbt + (G ? pl.nmb * pl.nnb : 0);
  tc_gram_kernel<<<dim3(tiles, pl.nchunks), kTcThreads, pl.smem, s>>>(mA, mXB, mGB, a);
  return cudaGetLastError();
}

cudaError_t preload_tc_kernels() {
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, tc_gram_kernel);
  return e != cudaSuccess ? e : preload_tc_gram2();
}

}  // namespace plam
