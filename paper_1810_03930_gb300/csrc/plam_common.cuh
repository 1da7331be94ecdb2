// Shared declarations of the PLAM / PCAL CUDA kernels (sm_103a).
//
// Layout conventions: every n x p matrix is column-major with a leading
// dimension; p x p matrices are column-major with leading dimension p.  The
// element ("storage") type T is double in FP64 mode and float in FP32 mode.
// FP32 mode keeps double arithmetic to the O(p^2) algebra and the scalars,
// because GB300 runs FP64 at 1/64 of the FP32 rate.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/plam.h"

namespace plam {

constexpr int kThreads = 256;     // threads of the tiled kernels (16 x 16 micro-tile grid)
constexpr int kTile = 64;         // output tile edge of the tiled kernels
constexpr int kKStep = 32;        // rows (Gram) or inner index (update) per shared-memory stage
constexpr int kFlushRows = 256;   // FP32 running sums are flushed into a compensated sum after this many terms

// Stop codes written by the step-size kernel.
enum StopCode { kRunning = 0, kConverged = 1, kMaxit = 2, kDiverged = 3, kTimeout = 4 };

// Per-solve device state (one instance per handle, in device memory).
struct DevState {
  int k;          // updates performed
  int stop;       // StopCode
  int nrec;       // history records written
  int eta_rule_used;
  double K0;      // ||G0 - X0 Psi(G0^T X0)||_F
  double eta;     // eta used by the latest update
  double eta_prev;
  double eta0;
  double kkt;     // relative KKT value at the latest evaluated iterate
  double feas;    // ||X^T X - I||_F there
  double f;       // f there
  double ss, sy, yy;  // latest Barzilai-Borwein inner products
  int refine;     // 1 once the tensor-core kernels run compensated (latched for the run)
  int k_best;     // iteration of the last halving of the best relative KKT value
  double kkt_best;
};

// The plain-TF32 phase of the tensor-core kernels hands over to the compensated phase
// when the relative KKT value falls below refine_switch, or when it stalls: no halving of
// the best value seen for kStallIters iterations (TF32 rounding can floor the KKT value
// above refine_switch, and the Barzilai-Borwein steps are not monotone).
constexpr int kStallIters = 100;

// Parameters of one iteration, passed by value.
struct IterParams {
  int64_t n;
  int p;
  int variant;      // 0 PLAM, 1 PCAL
  int lambda2;      // 1: PCAL multiplier of eq. (lambda2)
  int eta_rule;     // PLAM_ETA_*
  int maxit;
  int hist_cap;     // records available in the history buffer
  double beta;
  double eta0_user; // <= 0: automatic
  double gamma;     // constant rule
  double tol;
  double hartree_alpha;  // f correction term for the Hartree objective (0 otherwise)
  double f_xg, f_part;   // f = f_xg <X, G> + f_part (sum of the objective's f partials)
  int lambda_da;         // 1: dual ascent Lambda^k = Lambda^{k-1} - beta (B^k - I) (PLAM-DA, PCAL-DA)
  double* lam;           // p x p FP64 multiplier carried across iterations (dual ascent only)
  double refine_switch;  // <= 0: the compensated phase never starts on its own (see DevState.refine)
  int moptqr;            // 1: MOptQR's update matrix, M = C^T (R = G - X G^T X), no penalty
  double feas_max;       // > 0: ||X^T X - I||_F above it stops the run as diverged
  double eta_min, eta_max;   // > 0: bounds of eta^k; 0: 1e-10 eta0 and 1e10 eta0
};

// MOptQR's Barzilai-Borwein sums of S = X - X_prev and Y = R^k - R^{k-1}, per tile of the
// update kernel that ran (tile_rows x tile_cols tiles, nct tile columns): written over the
// update's per-tile slots 0..2 of totpart (zeros at k = 0).
template <typename T>
cudaError_t launch_mopt_bb(int64_t n, int p, const T* X, int64_t ldx, const T* Xprev, int64_t ldxp,
                           const T* R0, const T* R1, int64_t ldr, int tile_rows, int tile_cols,
                           int nrt, int nct, T* totpart, const DevState* st, cudaStream_t s);

// Number of per-column dot products written by the update kernel and the
// number of whole-matrix sums (see update_kernel).
constexpr int kColDots = 3;   // ||X_c||^2, <X_c,R_c>, ||R_c||^2
constexpr int kTotDots = 6;   // <S,S>, <S,Y>, <Y,Y>, ||K||^2, ||G||^2, <X,G>

// ---------------------------------------------------------------- launchers
// Each returns the cudaError_t of the launch (cudaGetLastError).

// part: nchunks x 2p x p partial Grams in the arithmetic type T (Tin: input type).
template <typename Tin, typename T>
cudaError_t launch_gram_partial(int64_t n, int p, const Tin* X, int64_t ldx, const Tin* G,
                                int64_t ldg, int64_t rows_per_chunk, int nchunks, T* part,
                                const DevState* st, cudaStream_t s);
template <typename T>
cudaError_t launch_gram_reduce(int p, int nchunks, int with_g, const T* part, double* B,
                               double* C, cudaStream_t s);
// red: 2p x p doubles of scratch for the reduced Grams [B | C]; rowpart:
// gram_rowpart_doubles(p) doubles of scratch for the row sums.  stage 0: the chunk
// reduction and the p x p step (through red at small p, inside the tile kernel at
// large p); 1: the reduction into red only; 2: the p x p step from red only (a
// row-sharded solve sums red over the ranks in between).  gram_finalize_launches:
// the kernels one call launches.
template <typename T>
cudaError_t launch_gram_finalize(int p, int nchunks, const T* part, double* red, double* rowpart,
                                 T* Mt, T* L0t, double* feas_row, const DevState* st,
                                 IterParams prm, cudaStream_t s, int stage = 0);
size_t gram_rowpart_doubles(int p);
int gram_finalize_launches(int p, int stage);

// Row sharding: out[i] = sum over r = 0 .. size-1, in that order, of in[r * count + i]
// (in: the all-gathered buffers of every rank).  st (may be null): skipped once stopped.
cudaError_t launch_rank_sum(const double* in, int size, int64_t count, double* out,
                            const DevState* st, cudaStream_t s);

// R0/R1: the two residual buffers (R^k goes to buffer k mod 2).  nubuf: 2 x p
// column norms and coef: 2 x (2p + 1) scales [1/eta, 1/nu_c, 1 - nu_c] in the
// storage type (iteration k writes buffer k mod 2).  colpart: nrt x 3 x p,
// totpart: nrt x nct x 6 partial sums in the storage type.
template <typename T>
cudaError_t launch_update(int64_t n, int p, const T* X, int64_t ldx, const T* G, int64_t ldg,
                          T* R0, T* R1, int64_t ldr, const T* Mt, const T* L0t, const T* coef,
                          const DevState* st, T* colpart, T* totpart, cudaStream_t s);
// dsum: kStepRanges x (3p + 6) partial sums of scratch in the storage type;
// sums: 3p + 7 doubles of scratch; ticket: one zero-initialised counter.
// phase 0: the whole step; a row-sharded solve runs phase 1 (this rank's sums into
// sums[0 .. 3p + 6], with the objective's f partials at sums[3p + 6]), sums them over
// the ranks, then phase 2 (eta, the column scales and the stop test from those sums).
constexpr int kStepRanges = 32;
template <typename T>
cudaError_t launch_step_size(int nrt, int nct, const T* colpart, const T* totpart, T* dsum,
                             const double* feas_row, const double* fpart, int nfpart, double* sums,
                             unsigned int* ticket, DevState* st, double* nubuf, T* coef,
                             double* hist, IterParams prm, cudaStream_t s, int phase = 0);
template <typename T>
cudaError_t launch_primal_update(int64_t n, int p, T* X, int64_t ldx, const T* R0, const T* R1,
                                 int64_t ldr, const T* coef, const DevState* st, int variant,
                                 cudaStream_t s);

// Objectives.  `fpart` receives per-block partial sums that the step-size
// kernel adds into f (Hartree: rho^T y); may be null.
template <typename T>
cudaError_t launch_dense_grad(int64_t n, int p, const T* A, int64_t lda, const T* X, int64_t ldx,
                              T* G, int64_t ldg, const DevState* st, cudaStream_t s);
template <typename T>
cudaError_t launch_right_multiply(int64_t n, int p, const T* X, int64_t ldx, const T* Bm,
                                  int64_t ldb, T* Y, int64_t ldy, const DevState* st,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_hartree_grad(int64_t n, int p, double alpha, double q, double xc, const T* X,
                                int64_t ldx, T* G, int64_t ldg, double* rho, double* blk, double* y,
                                double* fpart, const DevState* st, cudaStream_t s);
int hartree_blocks(int64_t n);
// Block-diagonal 1D objective with an optional linear term (Section 5.4's Problems 1 and 2):
// row tiles of `tile` rows x `ncg` column groups of `cw` columns; the f partials are
// ntiles * ncg doubles and rho_part ncg * n doubles (when alpha or xc is nonzero).
constexpr int kChainMaxBlock = 64;
struct ChainPlan {
  int tile, ntiles, ncg, cw;
};
ChainPlan chain_plan(int64_t n, int p, int64_t block, bool need_y);
template <typename T>
cudaError_t launch_chain_grad(int64_t n, int p, int64_t block, double alpha, double q, double xc,
                              const T* X, int64_t ldx, const T* lin, int64_t ldl, T* G,
                              int64_t ldg, double* rho_part, double* fpart, const DevState* st,
                              cudaStream_t s, int* launches);
template <typename T>
cudaError_t launch_stencil_grad(int nx, int ny, int nz, int p, const T* V, const T* X, int64_t ldx,
                                T* G, int64_t ldg, const DevState* st, cudaStream_t s);

// Final orthonormalisation.  W: p x p work (B is copied into it), Z: p x p
// output R^{-1} (upper triangular), info: 0 or 1 + the failing pivot.
cudaError_t launch_cholesky_inverse(int p, const double* B, double* W, double* Z, int* info,
                                    cudaStream_t s);
int cholesky_inverse_launches(int p);   // kernels launch_cholesky_inverse launches
// scratch: p^2 doubles of workspace (a float X: Z split into two float planes; the Cholesky
// workspace W is free once Z is formed).
template <typename T>
cudaError_t launch_apply_rinv(int64_t n, int p, const T* X, int64_t ldx, const double* Z,
                              double* Q, int64_t ldq, double* scratch, cudaStream_t s);
// The same product written in the storage type (MOptQR's retraction X <- V R^{-1}); st (may
// be null): skipped once the run has stopped.
template <typename T>
cudaError_t launch_apply_rinv_same(int64_t n, int p, const T* X, int64_t ldx, const double* Z, T* Q,
                                   int64_t ldq, double* scratch, const DevState* st,
                                   cudaStream_t s);
// out[0] = ||B - I||_F (p x p, FP64); col: p doubles of per-column sums.
cudaError_t launch_feas(int p, const double* B, double* col, double* out, cudaStream_t s);

// Message returned by plam_last_error() on this host thread ("what: detail").
void set_last_error(const char* what, const char* detail);

// Row chunking of the CUDA-core split-K Grams (one rule for every entry point, so that
// plam_grams and plam_grams_noalloc reduce in the same order whenever max_chunks does not
// bind): about two CTAs per SM over the (upper) tiles of X^T X and, with_g, the tiles of
// X^T G; chunks are whole kKStep-row stages; at most max_chunks chunks (<= 0: no cap).
struct GramChunkPlan {
  int64_t rows_per_chunk;
  int nchunks;
};
inline GramChunkPlan gram_chunk_plan(int64_t n, int p, bool with_g, int sms, int64_t max_chunks) {
  const int nt = (p + kTile - 1) / kTile;
  const int64_t tiles = (int64_t)nt * (nt + 1) / 2 + (with_g ? (int64_t)nt * nt : 0);
  const int64_t target_ctas = 2 * (int64_t)(sms > 0 ? sms : 1);
  int64_t nch = (target_ctas + tiles - 1) / tiles;
  const int64_t by_rows = (n + kKStep - 1) / kKStep;
  if (nch > by_rows) nch = by_rows;
  if (max_chunks > 0 && nch > max_chunks) nch = max_chunks;
  if (nch < 1) nch = 1;
  int64_t rows = (n + nch - 1) / nch;
  rows = (rows + kKStep - 1) / kKStep * kKStep;
  GramChunkPlan pl;
  pl.rows_per_chunk = rows;
  pl.nchunks = (int)((n + rows - 1) / rows);
  return pl;
}

// Resident (persistent, cooperative) solve: FP32, p <= 64, Hartree or dense.
struct ResidentLaunch {
  int64_t n;
  int p, nblk, rows, rp;
  size_t smem;
  int kind;
  const float* A;
  int64_t lda;
  double alpha, q;
  float* X;
  int64_t ldx;
  float* R0;
  float* R1;
  int64_t ldr;
  float* halo;
  double* blk;
  float* part;
  float* red;
  float* dots;
  double* dred;
  unsigned int* bar;
  int bar_extra;   // 0; a test raises it so that no barrier is ever released (bounded wait expires)
  int* err;
  DevState* st;
  double* nubuf;
  float* coef;
  double* hist;
  IterParams prm;
};
void resident_plan(int64_t n, int p, int sms, size_t smem_limit, int* nblk, int* rows, int* rp,
                   size_t* smem);
cudaError_t launch_resident_solve(const ResidentLaunch& L, cudaStream_t s);
cudaError_t preload_resident_kernels();

// Tensor-core (tcgen05, kind::tf32) Grams: split-K partials in the layout of
// launch_gram_partial (float), reduced by launch_gram_finalize / _reduce.
struct TcGramPlan {
  int pair;              // 1: CTA-pair kernel (256 x 256 tiles, p >= 256); 0: one CTA per tile
  int N, nmb, nnb, nbt, ntiles;
  int64_t rows_per_chunk;
  int nchunks;
  size_t smem;
};
// allow_pair = 0 keeps one CTA per 128 x N tile for every p.
void tc_gram_plan(int64_t n, int p, int with_g, TcGramPlan* pl, int allow_pair = 1);
bool tc_gram2_plan(int64_t n, int p, int with_g, TcGramPlan* pl);
cudaError_t launch_tc_gram2(int64_t n, int p, const float* X, int64_t ldx, const float* G,
                            int64_t ldg, const TcGramPlan& pl, float* part, int* err,
                            const DevState* st, double refine_switch, int force3, cudaStream_t s);
cudaError_t preload_tc_gram2();
bool tc_gram_supported(const void* X, int64_t ldx, const void* G, int64_t ldg);
// st / refine_switch: compensated 3xTF32 once st->refine is latched (st may be
// null); force3 = 1 always uses it.
cudaError_t launch_tc_gram(int64_t n, int p, const float* X, int64_t ldx, const float* G,
                           int64_t ldg, const TcGramPlan& pl, float* part, int* err,
                           const DevState* st, double refine_switch, int force3, cudaStream_t s);
cudaError_t preload_tc_kernels();
bool tma_encoder_available();
int device_sm_count();   // SMs of the current device

// Tensor-core update GEMM (FP32 storage): R = G - X M and the KKT residual,
// with the column and tile dots of launch_update (nrt x 3 x p and
// nrt x nct x 6 partials, nrt = ceil(n / 128), nct = ceil(p / N)).
// msplit: 4 x ldm x p floats of scratch for the TF32 parts of M and Psi(C).
struct TcUpdatePlan {
  int pair;              // 1: CTA pairs on 256-row tiles (p >= 256); 0: one CTA per 128-row tile
  int N, nct, nrt, ldm;  // nrt: 128-row tiles of the partial dots (either kernel)
  int ncl;               // pair: clusters of two that fit at once
  uint32_t pipe_bytes;
  size_t smem;
};
// allow_pair = 0 keeps one CTA per 128-row tile for every p.
void tc_update_plan(int64_t n, int p, TcUpdatePlan* pl, int allow_pair = 1);
bool tc_update_supported(const void* X, int64_t ldx);
cudaError_t launch_tc_update(int64_t n, int p, const float* X, int64_t ldx, const float* G,
                             int64_t ldg, float* R0, float* R1, int64_t ldr, const float* Mt,
                             const float* L0t, const TcUpdatePlan& pl, float* msplit,
                             const float* coef, const DevState* st, float* colpart,
                             float* totpart, int* err, double refine_switch, int force3,
                             cudaStream_t s);
cudaError_t preload_tc_update_kernels();

// Batched dense trace problems (p <= 64), one persistent launch: each CTA takes
// problems from the queue `next` in the host's order and runs the whole loop.
struct BatchDesc {
  int64_t n;
  int p, pad_;
  const float* A;
  int64_t lda;
  float* X;
  int64_t ldx;
  float* G;
  float* R0;
  float* R1;
  int64_t ldw;
  double* Q;        // FP64 output of the final orthonormalisation (may be null)
  int64_t ldq;
};

struct BatchParams {
  int variant, lambda2, eta_rule, maxit;
  double beta, eta0_user, gamma, tol;
  double eta_min, eta_max;   // > 0: bounds of eta^k; 0: 1e-10 eta0 and 1e10 eta0
};

// The step-size interval: [eta_min, eta_max] where given, else [1e-10 eta0, 1e10 eta0].
__host__ __device__ inline double eta_clamp(double eta, double eta0, double eta_min,
                                            double eta_max) {
  const double lo = eta_min > 0.0 ? eta_min : 1e-10 * eta0;
  const double hi = eta_max > 0.0 ? eta_max : 1e10 * eta0;
  return fmin(fmax(eta, lo), hi);
}

size_t batch_smem_bytes(int rb);
cudaError_t launch_batched(int rb, const BatchDesc* desc, const int* order, int count, int* next,
                           plam_info_t* info, BatchParams prm, int grid, cudaStream_t s);
cudaError_t preload_batched_kernels();

// Force the module load of every kernel (lazy loading must not happen inside
// a stream capture).
// Q^T Q of a double Q for the feasibility report: entries split into float pairs (about 48
// bits), exact FP32 products and compensated sums; partials in the layout of launch_gram_partial.
cudaError_t launch_gram_report(int64_t n, int p, const double* Q, int64_t ldq,
                               int64_t rows_per_chunk, int nchunks, double* part, cudaStream_t s);
cudaError_t preload_gram_kernels();
cudaError_t preload_update_kernels();
cudaError_t preload_objective_kernels();

}  // namespace plam
