// Host side of the C ABI declared in include/plam.h: handle and workspace
// management, the launch sequence of one PLAM / PCAL iteration, the
// graph-captured solve loop and the final orthonormalisation.
//
// One iteration (Algorithms 2 and 3) is the kernel sequence
//   objective gradient  G = grad f(X)                        (k_objective.cu)
//   gram_partial        row-chunk partials of X^T [X | G]     (k_gram.cu)
//   gram_finalize       B, Psi(C), d (eq. lambda2), M, feasibility rows
//   update              R = G - X M, K = G - X Psi(C), dots   (k_update.cu)
//   step_size           KKT test, eta (Section 5.1), PCAL column norms
//   primal_update       X <- X - R/eta  or  (X - R/eta) / nu
// All control (iteration counter, stop flag, eta, buffer parity) lives in a
// device-side state record, so the sequence has no host synchronisation and
// plam_solve replays it from a captured CUDA graph, reading the stop flag
// back once per replay.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/plam.h"
#include "plam_common.cuh"

using namespace plam;

namespace {

thread_local char g_err[512] = "";

plam_status_t cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
  return PLAM_ERR_CUDA;
}

plam_status_t objective_fail() {
  snprintf(g_err, sizeof(g_err), "objective callback failed: the user gradient returned non-zero");
  return PLAM_ERR_CUDA;
}

}  // namespace

void plam::set_last_error(const char* what, const char* detail) {
  snprintf(g_err, sizeof(g_err), "%s: %s", what, detail);
}

namespace {

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
  } while (0)

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace

struct plam_handle_s {
  int64_t n = 0, p = 0;
  plam_objective_t obj{};
  plam_params_t prm{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int prec = 0;
  size_t esz = 8;
  int64_t ldw = 0;
  void* G = nullptr;
  void* R[2] = {nullptr, nullptr};
  void* part = nullptr;
  double* part64 = nullptr;
  int nchunks = 1;
  int64_t rows_per_chunk = 0;
  double* B = nullptr;      // p x p
  double* C = nullptr;      // p x p scratch for plam_grams
  double* red = nullptr;    // 2p x p reduced Grams [B | C] of the iteration
  double* rowpart = nullptr;   // row sums of the p x p step (gram_rowpart_doubles(p))
  void* Mt = nullptr;
  void* L0t = nullptr;
  double* feas_row = nullptr;
  void* colpart = nullptr;
  void* totpart = nullptr;
  int nrt = 0, nct = 0;
  double* sums = nullptr;
  void* dsum = nullptr;     // kStepRanges x (3p + 6) row-range sums of the dots
  unsigned int* ticket = nullptr;
  DevState* st = nullptr;
  double* nubuf = nullptr;
  void* coef = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  double* rho = nullptr;
  double* blk = nullptr;
  double* y = nullptr;
  double* fpart = nullptr;
  int nfpart = 0;
  double* W = nullptr;
  double* Z = nullptr;
  int* info = nullptr;
  double* feas_dev = nullptr;
  double* Qtmp = nullptr;
  double* dotpart = nullptr;
  DevState* st_host = nullptr;
  int* info_host = nullptr;
  double* scal_host = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void* graph_X = nullptr;
  int64_t graph_ldx = 0;
  int graph_variant = -1;
  int graph_kernels = 0;
  int64_t launches = 0;
  // resident engine (allocated at creation when the problem qualifies)
  int r_nblk = 0, r_rows = 0, r_rp = 0;
  size_t r_smem = 0;
  float* r_halo = nullptr;
  double* r_blk = nullptr;
  float* r_part = nullptr;
  float* r_red = nullptr;
  float* r_dots = nullptr;
  double* r_dred = nullptr;
  unsigned int* r_bar = nullptr;
  int* r_err = nullptr;
  // tensor-core Grams (FP32 mode)
  int use_tc = 0;
  TcGramPlan tc{};
  int* tc_err = nullptr;
  // tensor-core update GEMM (FP32 mode)
  TcUpdatePlan tcu{};
  float* msplit = nullptr;
  // KKT residual after the final orthonormalisation: per-CTA partial sums
  double* kkt_part = nullptr;
  // dual-ascent multiplier (PLAM_LAMBDA_DA), p x p FP64
  double* lam = nullptr;
  // row sharding (plam_create_sharded)
  int sharded = 0;
  plam_comm_t comm{};
  int64_t g_off = 0;        // rows of G before the first local row (the stencil's lower halo plane)
  int64_t plane = 0;        // rows of one halo plane (sharded stencil)
  void* vext = nullptr;     // the potential with zero halo planes (sharded stencil)
  void* halo = nullptr;     // 4 x plane x p staging: send_lo, send_hi, recv_lo, recv_hi
  double* gath = nullptr;   // size x max(2 p^2, 3p + 7) doubles: the all-gather's receive buffer
  void* qtmp = nullptr;     // n x p work of Problem 4's gradient (A X before the product with B)
  void* xprev = nullptr;    // MOptQR: the previous iterate (S = X - X_prev), leading dimension ldw
  void* vbuf = nullptr;     // MOptQR: the retraction's output before it is copied back to X
  cudaEvent_t tev[3] = {nullptr, nullptr, nullptr};   // plam_solve's phase timing
};

namespace {

constexpr int kDotBlocks = 256;

// ||.||-free helper: per-block partial sums of <X, G> (storage type per thread,
// double per block), then a fixed-order sum on the host side of the copy.
template <typename T>
__global__ void dot_partial_kernel(int64_t n, int p, const T* __restrict__ X, int64_t ldx,
                                   const T* __restrict__ G, int64_t ldg, double* __restrict__ out) {
  __shared__ double red[33];
  T s = T(0);
  const int64_t total = n * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, r = e - c * n;
    s = fma(X[r + c * ldx], G[r + c * ldg], s);
  }
  double v = (double)s;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    out[blockIdx.x] = t;
  }
}

// tensor_cores = 2 (or 2 | PLAM_TC_SINGLE_CTA): compensated 3xTF32 from the first iteration.
inline int tc_always3(const plam_params_t& prm) {
  return prm.tensor_cores >= 0 && (prm.tensor_cores & 3) == 2;
}

plam_status_t validate_params(const plam_params_t* prm) {
  if (!prm) return PLAM_ERR_INVALID;
  if (prm->variant < PLAM_VARIANT_PLAM || prm->variant > PLAM_VARIANT_MOPTQR) return PLAM_ERR_INVALID;
  if (prm->lambda_rule < PLAM_LAMBDA1 || prm->lambda_rule > PLAM_LAMBDA_DA) return PLAM_ERR_INVALID;
  if (prm->eta_rule < PLAM_ETA_ABB || prm->eta_rule > PLAM_ETA_DIFF) return PLAM_ERR_INVALID;
  if (prm->precision != PLAM_PREC_FP64 && prm->precision != PLAM_PREC_FP32) return PLAM_ERR_INVALID;
  if (!(prm->beta >= 0.0) || !std::isfinite(prm->beta)) return PLAM_ERR_INVALID;
  if (!(prm->tol >= 0.0) || prm->maxit < 0) return PLAM_ERR_INVALID;
  if (prm->final_orth < 0 || prm->final_orth > 2 || prm->graph_iters < 0) return PLAM_ERR_INVALID;
  if (prm->engine < PLAM_ENGINE_AUTO || prm->engine > PLAM_ENGINE_RESIDENT) return PLAM_ERR_INVALID;
  {
    const int tc = prm->tensor_cores;
    if (!(tc >= -1 && tc <= 2) && tc != (1 | PLAM_TC_SINGLE_CTA) && tc != (2 | PLAM_TC_SINGLE_CTA))
      return PLAM_ERR_INVALID;
  }
  if (!(prm->refine_switch >= 0.0)) return PLAM_ERR_INVALID;
  if (!(prm->feas_max >= 0.0)) return PLAM_ERR_INVALID;
  if (!(prm->eta_min >= 0.0) || !(prm->eta_max >= 0.0) || !std::isfinite(prm->eta_min) ||
      !std::isfinite(prm->eta_max) ||
      (prm->eta_min > 0.0 && prm->eta_max > 0.0 && prm->eta_min > prm->eta_max))
    return PLAM_ERR_INVALID;
  return PLAM_OK;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// The 1D objective with a block-diagonal L or a linear term runs on the chain kernels.
bool chain_objective(const plam_handle_s* h) {
  return h->obj.kind == PLAM_OBJ_HARTREE1D && (h->obj.block != 0 || h->obj.lin != nullptr);
}

// f = f_xg <X, grad f> + f_part (sum of the objective's f partials): 1/2 <X, A X>
// for the quadratic objectives; the Hartree term enters through its partials
// rho^T L^{-1} rho; a user objective supplies f itself.
void f_coefficients(const plam_handle_s* h, double* f_xg, double* f_part) {
  switch (h->obj.kind) {
    case PLAM_OBJ_HARTREE1D: *f_xg = 0.5; *f_part = 1.0; break;   // partials carry -alpha/4, xc/4
    case PLAM_OBJ_CALLBACK: *f_xg = 0.0; *f_part = 1.0; break;
    default: *f_xg = 0.5; *f_part = 0.0; break;
  }
}

template <typename T>
IterParams iter_params(const plam_handle_s* h, int variant, int lambda2) {
  IterParams ip{};
  ip.n = h->n;
  ip.p = (int)h->p;
  ip.variant = variant;
  ip.lambda2 = lambda2;
  ip.eta_rule = h->prm.eta_rule;
  ip.maxit = h->prm.maxit;
  ip.hist_cap = h->hist_cap;
  ip.beta = h->prm.beta;
  ip.eta0_user = h->prm.eta0;
  ip.gamma = h->prm.eta_gamma;
  ip.tol = h->prm.tol;
  ip.hartree_alpha = (h->obj.kind == PLAM_OBJ_HARTREE1D) ? h->obj.alpha : 0.0;
  f_coefficients(h, &ip.f_xg, &ip.f_part);
  ip.lambda_da = h->prm.lambda_rule == PLAM_LAMBDA_DA;
  ip.lam = h->lam;
  ip.refine_switch = h->use_tc ? h->prm.refine_switch : 0.0;
  ip.feas_max = h->prm.feas_max;
  ip.eta_min = h->prm.eta_min;
  ip.eta_max = h->prm.eta_max;
  if (variant == PLAM_VARIANT_MOPTQR) {   // no penalty, no column scaling, M = C^T
    ip.moptqr = 1;
    ip.variant = PLAM_VARIANT_PLAM;
    ip.lambda2 = 0;
    ip.lambda_da = 0;
    ip.beta = 0.0;
  }
  return ip;
}

// Objective gradient into G (ld ldg); returns the number of kernels launched or -1.
template <typename T>
int launch_objective(plam_handle_s* h, const T* X, int64_t ldx, T* G, int64_t ldg,
                     const DevState* st, cudaStream_t s, cudaError_t* err) {
  const int p = (int)h->p;
  switch (h->obj.kind) {
    case PLAM_OBJ_DENSE:
      *err = launch_dense_grad<T>(h->n, p, (const T*)h->obj.A, h->obj.lda, X, ldx, G, ldg, st, s);
      return 1;
    case PLAM_OBJ_HARTREE1D:
      if (chain_objective(h)) {
        int k = 0;
        *err = launch_chain_grad<T>(h->n, p, h->obj.block, h->obj.alpha, h->obj.quad_scale,
                                    h->obj.xc, X, ldx, (const T*)h->obj.lin, h->obj.ldlin, G, ldg,
                                    h->rho, h->fpart, st, s, &k);
        return k;
      }
      *err = launch_hartree_grad<T>(h->n, p, h->obj.alpha, h->obj.quad_scale, h->obj.xc, X, ldx, G,
                                    ldg, h->rho,
                                    h->blk, h->y, h->fpart, st, s);
      return 2;
    case PLAM_OBJ_STENCIL3D:
      *err = launch_stencil_grad<T>(h->obj.nx, h->obj.ny, h->obj.nz, p, (const T*)h->obj.V, X, ldx,
                                    G, ldg, st, s);
      return 1;
    case PLAM_OBJ_QAP:   // A X into the handle's n x p work, then (A X) B
      *err = launch_dense_grad<T>(h->n, p, (const T*)h->obj.A, h->obj.lda, X, ldx, (T*)h->qtmp,
                                  h->ldw, st, s);
      if (*err == cudaSuccess)
        *err = launch_right_multiply<T>(h->n, p, (const T*)h->qtmp, h->ldw, (const T*)h->obj.Bq,
                                        h->obj.ldbq, G, ldg, st, s);
      return 2;
    case PLAM_OBJ_CALLBACK:
      if (h->obj.grad(h->obj.grad_ctx, X, ldx, G, ldg, h->fpart, (void*)s) != 0) {
        *err = cudaSuccess;
        return -2;   // the message is set by objective_fail
      }
      *err = cudaGetLastError();
      return 0;
  }
  *err = cudaErrorInvalidValue;
  return -1;
}

plam_status_t comm_fail(const char* what) {
  snprintf(g_err, sizeof(g_err), "communicator callback failed: %s", what);
  return PLAM_ERR_CUDA;
}

// Sum `count` doubles at buf over the ranks (all-gather, then the rank-order sum) in place.
// st: the iteration's state (the sum is skipped once the run has stopped, like every kernel
// of an iteration), or null outside the iteration (the final orthonormalisation).
plam_status_t shard_allreduce(plam_handle_s* h, double* buf, int64_t count, cudaStream_t s,
                              int* nk, const DevState* st) {
  if (h->comm.size == 1) return PLAM_OK;
  if (h->comm.allgather(h->comm.ctx, buf, h->gath, count, (void*)s) != 0) return comm_fail("allgather");
  CK(launch_rank_sum(h->gath, h->comm.size, count, buf, st, s));
  *nk += 1;
  return PLAM_OK;
}

// The stencil's halo planes of X: this rank's first and last planes to its neighbours, theirs
// into the rows before X and after X + n (zeros at the global boundary: Dirichlet).
template <typename T>
plam_status_t shard_halo(plam_handle_s* h, T* X, int64_t ldx, cudaStream_t s) {
  const int64_t pl = h->plane, n = h->n;
  const size_t w = sizeof(T), pitch = (size_t)ldx * w, cnt = (size_t)pl * h->p;
  T* buf = (T*)h->halo;
  T *send_lo = buf, *send_hi = buf + cnt, *recv_lo = buf + 2 * cnt, *recv_hi = buf + 3 * cnt;
  const int r = h->comm.rank, P = h->comm.size;
  if (P > 1) {
    CK(cudaMemcpy2DAsync(send_lo, pl * w, X, pitch, pl * w, h->p, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpy2DAsync(send_hi, pl * w, X + (n - pl), pitch, pl * w, h->p,
                         cudaMemcpyDeviceToDevice, s));
    if (h->comm.exchange(h->comm.ctx, send_lo, send_hi, recv_lo, recv_hi, (int64_t)cnt, (void*)s) != 0)
      return comm_fail("exchange");
  }
  if (r > 0)
    CK(cudaMemcpy2DAsync(X - pl, pitch, recv_lo, pl * w, pl * w, h->p, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemset2DAsync(X - pl, pitch, 0, pl * w, h->p, s));
  if (r < P - 1)
    CK(cudaMemcpy2DAsync(X + n, pitch, recv_hi, pl * w, pl * w, h->p, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemset2DAsync(X + n, pitch, 0, pl * w, h->p, s));
  return PLAM_OK;
}

// MOptQR's retraction after the step-size kernel (Table "cost"): X_prev <- X (the
// Barzilai-Borwein S of the next iteration), X <- V = X - D/eta (the PLAM form of the primal
// update), then X <- V R^{-1} with V^T V = R^T R, the Gram, Cholesky and product in FP64
// arithmetic (from a copy of V, so that X stays the converged iterate once the run stopped:
// the kernels that write X skip then).  Returns kernels launched in *nk.
template <typename T>
plam_status_t moptqr_retract(plam_handle_s* h, T* X, int64_t ldx, cudaStream_t s, int* nk) {
  const int p = (int)h->p;
  const size_t w = sizeof(T);
  CK(cudaMemcpy2DAsync(h->xprev, (size_t)h->ldw * w, X, (size_t)ldx * w, (size_t)h->n * w, p,
                       cudaMemcpyDeviceToDevice, s));
  CK(launch_primal_update<T>(h->n, p, X, ldx, (const T*)h->R[0], (const T*)h->R[1], h->ldw,
                             (const T*)h->coef, h->st, PLAM_VARIANT_PLAM, s));
  CK(cudaMemcpy2DAsync(h->vbuf, (size_t)h->ldw * w, X, (size_t)ldx * w, (size_t)h->n * w, p,
                       cudaMemcpyDeviceToDevice, s));
  CK((launch_gram_partial<T, double>(h->n, p, (const T*)h->vbuf, h->ldw, (const T*)nullptr, 0,
                                      h->rows_per_chunk, h->nchunks, h->part64, h->st, s)));
  CK(launch_gram_reduce<double>(p, h->nchunks, 0, h->part64, h->B, nullptr, s));
  CK(launch_cholesky_inverse(p, h->B, h->W, h->Z, h->info, s));
  CK(launch_apply_rinv_same<T>(h->n, p, (const T*)h->vbuf, h->ldw, h->Z, X, ldx, h->W, h->st, s));
  *nk += 4 + cholesky_inverse_launches(p) + (sizeof(T) == 4 ? 1 : 0);
  return PLAM_OK;
}

// The kernel sequence of one iteration on stream s; returns kernels launched.
// When `ev` is given, ev[i] is recorded before kernel group i and ev[6] after
// the last one (kernel attribution, plam_time_kernels).
template <typename T>
plam_status_t launch_iteration(plam_handle_s* h, T* X, int64_t ldx, int variant, int lambda2,
                               cudaStream_t s, int* nk, cudaEvent_t* ev = nullptr) {
  const int p = (int)h->p;
  const IterParams ip = iter_params<T>(h, variant, lambda2);
  T* G = (T*)h->G + h->g_off;
  cudaError_t e;
  if (ev) CK(cudaEventRecord(ev[0], s));
  int k = 0;
  if (h->sharded && h->obj.kind == PLAM_OBJ_STENCIL3D) {
    // the halo planes, then the stencil on the slab extended by them (the outputs on the
    // halo planes themselves are not used)
    plam_status_t hs = shard_halo<T>(h, X, ldx, s);
    if (hs != PLAM_OK) return hs;
    e = launch_stencil_grad<T>(h->obj.nx, h->obj.ny, h->obj.nz + 2, p, (const T*)h->vext,
                               X - h->plane, ldx, (T*)h->G, h->ldw, h->st, s);
    k = 1;
  } else {
    k = launch_objective<T>(h, X, ldx, G, h->ldw, h->st, s, &e);
  }
  if (k == -2) return objective_fail();
  if (k < 0 || e != cudaSuccess) return cuda_fail(e, "objective gradient");
  if (ev) CK(cudaEventRecord(ev[1], s));
  int nch = h->nchunks;
  if (sizeof(T) == 4 && h->use_tc && tc_gram_supported(X, ldx, G, h->ldw)) {
    CK(launch_tc_gram(h->n, p, (const float*)X, ldx, (const float*)G, h->ldw, h->tc, (float*)h->part,
                      h->tc_err, h->st, h->prm.refine_switch, tc_always3(h->prm), s));
    nch = h->tc.nchunks;
  } else {
    CK((launch_gram_partial<T, T>(h->n, p, X, ldx, G, h->ldw, h->rows_per_chunk, h->nchunks,
                                   (T*)h->part, h->st, s)));
  }
  if (ev) CK(cudaEventRecord(ev[2], s));
  // the fixed count below takes two launches for this stage
  if (h->sharded) {
    CK(launch_gram_finalize<T>(p, nch, (const T*)h->part, h->red, h->rowpart, (T*)h->Mt,
                               (T*)h->L0t, h->feas_row, h->st, ip, s, 1));
    plam_status_t as = shard_allreduce(h, h->red, (int64_t)2 * p * p, s, &k, h->st);
    if (as != PLAM_OK) return as;
    CK(launch_gram_finalize<T>(p, nch, (const T*)h->part, h->red, h->rowpart, (T*)h->Mt,
                               (T*)h->L0t, h->feas_row, h->st, ip, s, 2));
    k += gram_finalize_launches(p, 1) + gram_finalize_launches(p, 2) - 2;
  } else {
    CK(launch_gram_finalize<T>(p, nch, (const T*)h->part, h->red, h->rowpart, (T*)h->Mt,
                               (T*)h->L0t, h->feas_row, h->st, ip, s));
    k += gram_finalize_launches(p, 0) - 2;
  }
  if (ev) CK(cudaEventRecord(ev[3], s));
  int nrt = h->nrt, nct = h->nct;
  bool tc_upd = false;
  if (sizeof(T) == 4 && h->use_tc && tc_update_supported(X, ldx)) {
    tc_upd = true;
    CK(launch_tc_update(h->n, p, (const float*)X, ldx, (const float*)G, h->ldw, (float*)h->R[0],
                        (float*)h->R[1], h->ldw, (const float*)h->Mt, (const float*)h->L0t, h->tcu,
                        h->msplit, (const float*)h->coef, h->st, (float*)h->colpart,
                        (float*)h->totpart, h->tc_err, h->prm.refine_switch,
                        tc_always3(h->prm), s));
    nrt = h->tcu.nrt;
    nct = h->tcu.nct;
    k += 1;   // the TF32 split of M and Psi(C)
  } else {
    CK(launch_update<T>(h->n, p, X, ldx, G, h->ldw, (T*)h->R[0], (T*)h->R[1], h->ldw,
                        (const T*)h->Mt, (const T*)h->L0t, (const T*)h->coef, h->st,
                        (T*)h->colpart, (T*)h->totpart, s));
  }
  if (ip.moptqr) {   // the update's S/Y sums assume the PLAM/PCAL step: MOptQR's own
    CK(launch_mopt_bb<T>(h->n, p, X, ldx, (const T*)h->xprev, h->ldw, (const T*)h->R[0],
                         (const T*)h->R[1], h->ldw, tc_upd ? 128 : kTile, tc_upd ? h->tcu.N : kTile,
                         nrt, nct, (T*)h->totpart, h->st, s));
    k += 1;
  }
  if (ev) CK(cudaEventRecord(ev[4], s));
  if (h->sharded) {
    CK(launch_step_size<T>(nrt, nct, (const T*)h->colpart, (const T*)h->totpart, (T*)h->dsum,
                           h->feas_row, h->fpart, h->nfpart, h->sums, h->ticket, h->st, h->nubuf,
                           (T*)h->coef, h->hist, ip, s, 1));
    plam_status_t as = shard_allreduce(h, h->sums, (int64_t)kColDots * p + kTotDots + 1, s, &k,
                                       h->st);
    if (as != PLAM_OK) return as;
    CK(launch_step_size<T>(nrt, nct, (const T*)h->colpart, (const T*)h->totpart, (T*)h->dsum,
                           h->feas_row, h->fpart, h->nfpart, h->sums, h->ticket, h->st, h->nubuf,
                           (T*)h->coef, h->hist, ip, s, 2));
    k += 1;
  } else {
    CK(launch_step_size<T>(nrt, nct, (const T*)h->colpart, (const T*)h->totpart, (T*)h->dsum,
                           h->feas_row,
                           h->fpart, h->nfpart, h->sums,
                           h->ticket, h->st, h->nubuf, (T*)h->coef, h->hist, ip, s));
  }
  if (ev) CK(cudaEventRecord(ev[5], s));
  if (ip.moptqr) {
    int nr = 0;
    plam_status_t rs = moptqr_retract<T>(h, X, ldx, s, &nr);
    if (rs != PLAM_OK) return rs;
    k += nr - 1;
  } else {
    CK(launch_primal_update<T>(h->n, p, X, ldx, (const T*)h->R[0], (const T*)h->R[1], h->ldw,
                               (const T*)h->coef, h->st, variant, s));
  }
  if (ev) CK(cudaEventRecord(ev[6], s));
  *nk = k + 6;
  return PLAM_OK;
}

plam_status_t dispatch_iteration(plam_handle_s* h, void* X, int64_t ldx, int variant, int lambda2,
                                 cudaStream_t s, int* nk, cudaEvent_t* ev = nullptr) {
  if (h->prec == PLAM_PREC_FP64)
    return launch_iteration<double>(h, (double*)X, ldx, variant, lambda2, s, nk, ev);
  return launch_iteration<float>(h, (float*)X, ldx, variant, lambda2, s, nk, ev);
}

plam_status_t reset_state(plam_handle_s* h) {
  CK(cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream));
  CK(cudaMemsetAsync(h->ticket, 0, sizeof(unsigned int), h->stream));
  CK(cudaMemsetAsync(h->nubuf, 0, 2 * h->p * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->coef, 0, 2 * (2 * h->p + 1) * h->esz, h->stream));
  if (h->tc_err) CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
  return PLAM_OK;
}

plam_status_t read_state(plam_handle_s* h, plam_info_t* info, int* stop) {
  CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  if (h->tc_err) CK(cudaMemcpyAsync(h->info_host, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->tc_err && *h->info_host != 0) h->st_host->stop = kTimeout;
  const DevState& s = *h->st_host;
  if (stop) *stop = s.stop;
  if (info) {
    info->ms_iterations = info->ms_orth = NAN;
    info->iters = s.k;
    info->converged = (s.stop == kConverged);
    info->f = s.f;
    info->kkt_rel = s.kkt;
    info->feas = s.feas;
    info->eta = s.eta;
    info->K0 = s.K0;
    info->eta0 = s.eta0;
    info->status = (s.stop == kDiverged) ? PLAM_ERR_DIVERGED
                   : (s.stop == kMaxit)  ? PLAM_ERR_NOT_CONVERGED
                   : (s.stop == kTimeout) ? PLAM_ERR_TIMEOUT
                                         : PLAM_OK;
  }
  return PLAM_OK;
}

// X of a sharded stencil handle carries a halo plane before and after the local rows.
bool halo_rows_ok(const plam_handle_s* h, int64_t ldx) {
  return h->plane == 0 || ldx >= h->n + 2 * h->plane;
}

plam_status_t step_common(plam_handle_t h, void* X, int64_t ldx, plam_info_t* info, int variant,
                          int lambda2) {
  if (!h || !X || ldx < h->n || !aligned(X, h->esz) || !halo_rows_ok(h, ldx))
    return PLAM_ERR_INVALID;
  int nk = 0;
  plam_status_t st = dispatch_iteration(h, X, ldx, variant, lambda2, h->stream, &nk);
  if (st != PLAM_OK) return st;
  h->launches += nk;
  int stop = 0;
  if (info) {
    info->f_orth = info->kkt_orth = info->feas_orth = NAN;
  }
  st = read_state(h, info, &stop);
  if (st != PLAM_OK) return st;
  if (stop == kDiverged) return PLAM_ERR_DIVERGED;
  return PLAM_OK;
}

void free_handle(plam_handle_s* h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  void* dev[] = {h->G, h->R[0], h->R[1], h->part, h->part64, h->B, h->C, h->red, h->rowpart, h->Mt,
                 h->L0t, h->feas_row, h->colpart, h->totpart, h->sums, h->dsum, h->ticket, h->st, h->nubuf,
                 h->coef, h->hist,
                 h->rho, h->blk, h->y, h->fpart, h->W, h->Z, h->info, h->feas_dev, h->Qtmp,
                 h->dotpart, h->r_halo, h->r_blk, h->r_part, h->r_red, h->r_dots, h->r_dred,
                 h->r_bar, h->r_err, h->tc_err, h->msplit, h->kkt_part, h->lam, h->vext,
                 h->halo, h->gath, h->qtmp, h->xprev, h->vbuf};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->info_host) cudaFreeHost(h->info_host);
  if (h->scal_host) cudaFreeHost(h->scal_host);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaEvent_t e : h->tev)
    if (e) cudaEventDestroy(e);
  delete h;
}

template <typename T>
plam_status_t orthonormalize_impl(plam_handle_s* h, const T* X, int64_t ldx, double* Xout,
                                  int64_t ldo, int passes, double* feas) {
  const int p = (int)h->p;
  cudaStream_t s = h->stream;
  const double* src64 = nullptr;
  for (int pass = 0; pass < passes; ++pass) {
    if (pass == 0) {
      CK((launch_gram_partial<T, double>(h->n, p, X, ldx, (const T*)nullptr, 0, h->rows_per_chunk,
                                          h->nchunks, h->part64, nullptr, s)));
    } else {
      CK((launch_gram_partial<double, double>(h->n, p, src64, h->ldw, (const double*)nullptr, 0,
                                               h->rows_per_chunk, h->nchunks, h->part64, nullptr,
                                               s)));
    }
    CK(launch_gram_reduce<double>(p, h->nchunks, 0, h->part64, h->B, nullptr, s));
    if (h->sharded) {
      int nk = 0;
      plam_status_t as = shard_allreduce(h, h->B, (int64_t)p * p, s, &nk, nullptr);   // all rows
      if (as != PLAM_OK) return as;
      h->launches += nk;
    }
    CK(launch_cholesky_inverse(p, h->B, h->W, h->Z, h->info, s));
    CK(cudaMemcpyAsync(h->info_host, h->info, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->launches += 2 + cholesky_inverse_launches(p);
    if (*h->info_host != 0) {
      snprintf(g_err, sizeof(g_err), "Cholesky pivot %d not positive", *h->info_host);
      return PLAM_ERR_CHOLESKY;
    }
    if (pass == 0) {
      if (passes == 1) {
        CK(launch_apply_rinv<T>(h->n, p, X, ldx, h->Z, Xout, ldo, h->W, s));
      } else {
        CK(launch_apply_rinv<T>(h->n, p, X, ldx, h->Z, h->Qtmp, h->ldw, h->W, s));
        src64 = h->Qtmp;
      }
    } else {
      CK(launch_apply_rinv<double>(h->n, p, src64, h->ldw, h->Z, Xout, ldo, h->W, s));
    }
    h->launches += (pass == 0 && sizeof(T) == 4) ? 2 : 1;   // a float X: split Z, then apply
  }
  if (feas) {
    CK(launch_gram_report(h->n, p, Xout, ldo, h->rows_per_chunk, h->nchunks, h->part64, s));
    CK(launch_gram_reduce<double>(p, h->nchunks, 0, h->part64, h->B, nullptr, s));
    if (h->sharded) {
      int nk = 0;
      plam_status_t as = shard_allreduce(h, h->B, (int64_t)p * p, s, &nk, nullptr);
      if (as != PLAM_OK) return as;
      h->launches += nk;
    }
    CK(launch_feas(p, h->B, h->feas_row, h->feas_dev, s));
    CK(cudaMemcpyAsync(h->scal_host, h->feas_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->launches += 4;
    *feas = h->scal_host[0];
  }
  return PLAM_OK;
}

template <typename T>
plam_status_t energy_impl(plam_handle_s* h, const T* X, int64_t ldx, T* G, int64_t ldg, double* f) {
  cudaError_t e;
  const int k = launch_objective<T>(h, X, ldx, G, ldg, nullptr, h->stream, &e);
  if (k == -2) return objective_fail();
  if (k < 0 || e != cudaSuccess) return cuda_fail(e, "objective gradient");
  h->launches += k;
  if (f) {
    dot_partial_kernel<T><<<kDotBlocks, 256, 0, h->stream>>>(h->n, (int)h->p, X, ldx, G, ldg,
                                                              h->dotpart);
    CK(cudaGetLastError());
    h->launches += 1;
    const int nf = h->nfpart;
    CK(cudaMemcpyAsync(h->scal_host, h->dotpart, kDotBlocks * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    if (nf > 0)
      CK(cudaMemcpyAsync(h->scal_host + kDotBlocks, h->fpart, nf * sizeof(double),
                         cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double xg = 0.0, hy = 0.0;
    for (int i = 0; i < kDotBlocks; ++i) xg += h->scal_host[i];
    for (int i = 0; i < nf; ++i) hy += h->scal_host[kDotBlocks + i];
    double cx = 0.0, cf = 0.0;
    f_coefficients(h, &cx, &cf);
    *f = cx * xg + cf * hy;
  }
  return PLAM_OK;
}

// ||G - Q Psi(Q^T G)||_F^2 after the final orthonormalisation (Section 3.3's
// KKT measure; C = Q^T G in FP64 column-major): each CTA owns 128 rows of a
// kKktCols-column block, keeps Psi(C) for the block in shared memory and forms
// the residual elementwise; per-CTA partial sums in a fixed order.
constexpr int kKktCols = 16;
constexpr int kKktBlocksX = 256;

template <typename T>
__global__ void __launch_bounds__(128)
kkt_norm_kernel(int64_t n, int p, const T* __restrict__ Q, int64_t ldq, const T* __restrict__ G,
                int64_t ldg, const double* __restrict__ C, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char kkt_smem[];
  T* L = reinterpret_cast<T*>(kkt_smem);           // [p][kKktCols]
  const int c0 = blockIdx.y * kKktCols;
  for (int i = threadIdx.x; i < p * kKktCols; i += blockDim.x) {
    const int j = i / kKktCols, c = c0 + i % kKktCols;
    L[i] = c < p ? (T)(0.5 * (C[j + (size_t)c * p] + C[c + (size_t)j * p])) : T(0);
  }
  __syncthreads();
  double s = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    T acc[kKktCols];
#pragma unroll
    for (int c = 0; c < kKktCols; ++c) acc[c] = T(0);
    for (int j = 0; j < p; ++j) {
      const T q = Q[r + (int64_t)j * ldq];
#pragma unroll
      for (int c = 0; c < kKktCols; ++c) acc[c] = fma(q, L[j * kKktCols + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kKktCols; ++c) {
      if (c0 + c < p) {
        const double k = (double)(G[r + (int64_t)(c0 + c) * ldg] - acc[c]);
        s += k * k;
      }
    }
  }
  __shared__ double red[4];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0)
    part[blockIdx.y * gridDim.x + blockIdx.x] = ((red[0] + red[1]) + red[2]) + red[3];
}

__global__ void round_to_float_kernel(int64_t n, int p, const double* __restrict__ X, int64_t ldx,
                                      float* __restrict__ Y, int64_t ldy) {
  const int c = blockIdx.y;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    Y[r + (int64_t)c * ldy] = (float)X[r + (int64_t)c * ldx];
}

// f and the relative KKT value of the orthonormalised output Q (storage type
// T: the FP64 output itself, or its rounding to FP32 in FP32 mode).
template <typename T>
plam_status_t post_orth_metrics(plam_handle_s* h, const T* Q, int64_t ldq, double* f,
                                double* kkt_rel) {
  const int p = (int)h->p;
  T* G = (T*)h->G;
  plam_status_t st = energy_impl<T>(h, Q, ldq, G, h->ldw, f);
  if (st != PLAM_OK) return st;
  CK((launch_gram_partial<T, T>(h->n, p, Q, ldq, G, h->ldw, h->rows_per_chunk, h->nchunks,
                                 (T*)h->part, nullptr, h->stream)));
  CK(launch_gram_reduce<T>(p, h->nchunks, 1, (const T*)h->part, h->W, h->C, h->stream));
  const int gy = (p + kKktCols - 1) / kKktCols;
  int64_t gx = (h->n + 127) / 128;
  if (gx > kKktBlocksX) gx = kKktBlocksX;
  const size_t smem = (size_t)p * kKktCols * sizeof(T);
  if (smem > 232448) {   // Psi(C) block does not fit in shared memory: not evaluated
    *kkt_rel = NAN;
    return PLAM_OK;
  }
  CK(cudaFuncSetAttribute(kkt_norm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem));
  kkt_norm_kernel<T><<<dim3((unsigned)gx, (unsigned)gy), 128, smem, h->stream>>>(
      h->n, p, Q, ldq, G, h->ldw, h->C, h->kkt_part);
  CK(cudaGetLastError());
  h->launches += 3;
  const size_t np = (size_t)gx * gy;
  std::vector<double> hp(np);
  CK(cudaMemcpyAsync(hp.data(), h->kkt_part, np * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  double s = 0.0;
  for (size_t i = 0; i < np; ++i) s += hp[i];
  const double K0 = h->st_host->K0;
  *kkt_rel = K0 > 0 ? std::sqrt(s) / K0 : 0.0;
  return PLAM_OK;
}

// f(X) into device memory without a host synchronisation: the gradient goes
// to the handle's G buffer, f = f_xg <X, G> + f_part (sum of the f partials).
__global__ void energy_finalize_kernel(const double* __restrict__ dotpart, int ndot,
                                       const double* __restrict__ fpart, int nf, double f_xg,
                                       double f_part, double* __restrict__ f) {
  if (threadIdx.x == 0) {
    double xg = 0.0, hy = 0.0;
    for (int i = 0; i < ndot; ++i) xg += dotpart[i];
    for (int i = 0; i < nf; ++i) hy += fpart[i];
    *f = f_xg * xg + f_part * hy;
  }
}

template <typename T>
__global__ void scale_columns_kernel(int64_t n, int p, const double* __restrict__ s, T* G,
                                     int64_t ldg) {
  const T sc = (T)*s;
  const int c = blockIdx.y;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    G[r + (int64_t)c * ldg] *= sc;
}

template <typename T>
plam_status_t energy_device_impl(plam_handle_s* h, const T* X, int64_t ldx, double* f) {
  cudaError_t e;
  T* G = (T*)h->G;
  const int k = launch_objective<T>(h, X, ldx, G, h->ldw, nullptr, h->stream, &e);
  if (k == -2) return objective_fail();
  if (k < 0 || e != cudaSuccess) return cuda_fail(e, "objective gradient");
  double cx = 0.0, cf = 0.0;
  f_coefficients(h, &cx, &cf);
  int ndot = 0;
  if (cx != 0.0) {
    dot_partial_kernel<T><<<kDotBlocks, 256, 0, h->stream>>>(h->n, (int)h->p, X, ldx, G, h->ldw,
                                                              h->dotpart);
    CK(cudaGetLastError());
    ndot = kDotBlocks;
  }
  energy_finalize_kernel<<<1, 32, 0, h->stream>>>(h->dotpart, ndot, h->fpart, h->nfpart, cx, cf, f);
  CK(cudaGetLastError());
  h->launches += k + (ndot > 0 ? 2 : 1);
  return PLAM_OK;
}

template <typename T>
plam_status_t energy_backward_impl(plam_handle_s* h, const T* X, int64_t ldx, const double* s,
                                   T* G, int64_t ldg) {
  cudaError_t e;
  const int k = launch_objective<T>(h, X, ldx, G, ldg, nullptr, h->stream, &e);
  if (k == -2) return objective_fail();
  if (k < 0 || e != cudaSuccess) return cuda_fail(e, "objective gradient");
  h->launches += k;
  if (s) {
    int64_t bx = (h->n + 255) / 256;
    if (bx > 64) bx = 64;
    scale_columns_kernel<T><<<dim3((unsigned)bx, (unsigned)h->p), 256, 0, h->stream>>>(
        h->n, (int)h->p, s, G, ldg);
    CK(cudaGetLastError());
    h->launches += 1;
  }
  return PLAM_OK;
}

}  // namespace

extern "C" {

plam_status_t plam_default_params(plam_params_t* prm) {
  if (!prm) return PLAM_ERR_INVALID;
  memset(prm, 0, sizeof(*prm));
  prm->variant = PLAM_VARIANT_PCAL;
  prm->lambda_rule = PLAM_LAMBDA2;
  prm->beta = 1.0;
  prm->eta_rule = PLAM_ETA_ABB;
  prm->eta0 = 0.0;
  prm->eta_gamma = 0.0;
  prm->tol = 1e-8;
  prm->maxit = 3000;
  prm->precision = PLAM_PREC_FP64;
  prm->final_orth = 1;
  prm->graph_iters = 16;
  prm->engine = PLAM_ENGINE_AUTO;
  prm->tensor_cores = -1;
  prm->refine_switch = 1e-3;
  prm->feas_max = 1e6;
  prm->eta_min = 0.0;
  prm->eta_max = 0.0;
  prm->orth_metrics = 1;
  return PLAM_OK;
}

}  // extern "C"

namespace {

// plam_create and plam_create_sharded (comm != nullptr).
plam_status_t create_impl(plam_handle_t* out, int64_t n, int64_t p, const plam_objective_t* obj,
                          const plam_params_t* prm_in, void* stream, const plam_comm_t* comm) {
  if (!out) return PLAM_ERR_INVALID;
  *out = nullptr;
  const int64_t n_all = comm ? comm->n_global : n;
  if (!obj || p < 1 || n < 1 || n_all < 2 * p || p > 65535) return PLAM_ERR_INVALID;
  if (validate_params(prm_in) != PLAM_OK) return PLAM_ERR_INVALID;
  plam_params_t prm_local = *prm_in;
  const plam_params_t* prm = &prm_local;
  int64_t plane = 0;
  if (comm) {
    if (comm->size < 1 || comm->rank < 0 || comm->rank >= comm->size || comm->row0 < 0 ||
        comm->row0 + n > comm->n_global || (comm->size > 1 && !comm->allgather))
      return PLAM_ERR_INVALID;
    if (obj->kind == PLAM_OBJ_STENCIL3D) {
      plane = (int64_t)obj->nx * obj->ny;
      if (plane < 1 || comm->row0 % plane != 0 || (comm->size > 1 && !comm->exchange))
        return PLAM_ERR_INVALID;
    } else if (obj->kind == PLAM_OBJ_HARTREE1D) {
      if (obj->block < 1) return PLAM_ERR_UNSUPPORTED;   // one global L couples every row
      if (comm->row0 % obj->block != 0 ||
          (comm->rank < comm->size - 1 && n % obj->block != 0))
        return PLAM_ERR_INVALID;
    } else {
      return PLAM_ERR_UNSUPPORTED;
    }
    if (prm->engine == PLAM_ENGINE_RESIDENT || prm->variant == PLAM_VARIANT_MOPTQR)
      return PLAM_ERR_UNSUPPORTED;
    prm_local.engine = PLAM_ENGINE_GRAPH;
    prm_local.graph_iters = 0;
    prm_local.orth_metrics = 0;
  }
  const size_t esz = prm->precision == PLAM_PREC_FP64 ? 8 : 4;
  switch (obj->kind) {
    case PLAM_OBJ_DENSE:
      if (!obj->A || obj->lda < n || !aligned(obj->A, esz)) return PLAM_ERR_INVALID;
      break;
    case PLAM_OBJ_HARTREE1D: {
      if (!std::isfinite(obj->alpha) || !std::isfinite(obj->quad_scale) || !std::isfinite(obj->xc) ||
          obj->block < 0)
        return PLAM_ERR_INVALID;
      if (obj->lin && (obj->ldlin < n || !aligned(obj->lin, esz))) return PLAM_ERR_INVALID;
      const int64_t blk = obj->block >= n ? 0 : obj->block;
      if ((blk != 0 || obj->lin) && obj->alpha != 0.0 && (blk < 1 || blk > kChainMaxBlock))
        return PLAM_ERR_INVALID;
      break;
    }
    case PLAM_OBJ_STENCIL3D:
      if (obj->nx < 1 || obj->ny < 1 || obj->nz < 1 ||
          (int64_t)obj->nx * obj->ny * obj->nz != n || n > 2147483647 ||
          (obj->V && !aligned(obj->V, esz)))
        return PLAM_ERR_INVALID;
      break;
    case PLAM_OBJ_CALLBACK:
      if (!obj->grad) return PLAM_ERR_INVALID;
      if (prm->engine == PLAM_ENGINE_RESIDENT) return PLAM_ERR_UNSUPPORTED;
      break;
    case PLAM_OBJ_QAP:
      if (!obj->A || obj->lda < n || !aligned(obj->A, esz) || !obj->Bq || obj->ldbq < p ||
          !aligned(obj->Bq, esz))
        return PLAM_ERR_INVALID;
      if (prm->engine == PLAM_ENGINE_RESIDENT) return PLAM_ERR_UNSUPPORTED;
      break;
    default:
      return PLAM_ERR_INVALID;
  }
  plam_handle_s* h = new (std::nothrow) plam_handle_s();
  if (!h) return PLAM_ERR_NOMEM;
  h->n = n;
  h->p = p;
  h->obj = *obj;
  if (h->obj.kind == PLAM_OBJ_HARTREE1D && h->obj.block >= n && !comm) h->obj.block = 0;
  h->prm = *prm;
  h->stream = (cudaStream_t)stream;
  h->prec = prm->precision;
  h->esz = esz;
  h->ldw = round_up(n, 32);
  if (comm) {
    h->sharded = 1;
    h->comm = *comm;
    h->plane = plane;
    h->g_off = plane;
    h->ldw = round_up(n + 2 * plane, 32);
  }
  const int pi = (int)p;
  const int nt = (pi + kTile - 1) / kTile;
  const GramChunkPlan gcp = gram_chunk_plan(n, pi, true, device_sm_count(), 0);
  h->rows_per_chunk = gcp.rows_per_chunk;
  h->nchunks = gcp.nchunks;
  h->nrt = (int)((n + kTile - 1) / kTile);
  h->nct = nt;
  h->hist_cap = prm->maxit + 2;
  if (prm->precision == PLAM_PREC_FP32 &&
      (prm->tensor_cores >= 1 || (prm->tensor_cores == -1 && p >= 128))) {
    tc_gram_plan(n, (int)p, 1, &h->tc, !(prm->tensor_cores >= 0 &&
                                         (prm->tensor_cores & PLAM_TC_SINGLE_CTA)));
    tc_update_plan(n, (int)p, &h->tcu, !(prm->tensor_cores >= 0 &&
                                         (prm->tensor_cores & PLAM_TC_SINGLE_CTA)));
    h->use_tc = 1;
  }
  const int part_chunks = h->use_tc && h->tc.nchunks > h->nchunks ? h->tc.nchunks : h->nchunks;
  const size_t np_bytes = (size_t)h->ldw * p * esz;
  const size_t pp = (size_t)p * p;
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    return cudaMalloc(ptr, bytes == 0 ? 16 : bytes) == cudaSuccess;
  };
  bool ok = alloc(&h->G, np_bytes) && alloc(&h->R[0], np_bytes) && alloc(&h->R[1], np_bytes) &&
            alloc(&h->part, (size_t)part_chunks * 2 * pp * esz) &&
            alloc((void**)&h->tc_err, sizeof(int)) &&
            (!h->use_tc || alloc((void**)&h->msplit, (size_t)4 * h->tcu.ldm * p * sizeof(float))) &&
            alloc((void**)&h->part64, (size_t)h->nchunks * 2 * pp * sizeof(double)) &&
            alloc((void**)&h->B, pp * sizeof(double)) &&
            alloc((void**)&h->C, pp * sizeof(double)) && alloc(&h->Mt, pp * esz) &&
            alloc((void**)&h->red, 2 * pp * sizeof(double)) &&
            alloc((void**)&h->rowpart, gram_rowpart_doubles((int)p) * sizeof(double)) &&
            alloc(&h->L0t, pp * esz) && alloc((void**)&h->feas_row, p * sizeof(double)) &&
            alloc(&h->colpart, (size_t)h->nrt * kColDots * p * esz) &&
            alloc(&h->totpart, (size_t)h->nrt * h->nct * kTotDots * esz) &&
            alloc((void**)&h->sums, (kColDots * p + kTotDots + 1) * sizeof(double)) &&
            alloc(&h->dsum, (size_t)kStepRanges * (kColDots * p + kTotDots) * esz) &&
            alloc((void**)&h->ticket, sizeof(unsigned int)) &&
            alloc((void**)&h->st, sizeof(DevState)) &&
            alloc((void**)&h->nubuf, 2 * p * sizeof(double)) &&
            alloc(&h->coef, 2 * (2 * p + 1) * esz) &&
            alloc((void**)&h->hist, (size_t)h->hist_cap * 5 * sizeof(double)) &&
            alloc((void**)&h->W, pp * sizeof(double)) && alloc((void**)&h->Z, pp * sizeof(double)) &&
            alloc((void**)&h->info, sizeof(int)) && alloc((void**)&h->feas_dev, sizeof(double)) &&
            alloc((void**)&h->dotpart, kDotBlocks * sizeof(double)) &&
            alloc((void**)&h->kkt_part, (size_t)kKktBlocksX * ((p + kKktCols - 1) / kKktCols) *
                                            sizeof(double));
  if (ok && chain_objective(h)) {
    const ChainPlan c = chain_plan(n, (int)p, h->obj.block, h->obj.alpha != 0.0);
    h->nfpart = c.ntiles * c.ncg;
    ok = alloc((void**)&h->fpart, (size_t)h->nfpart * sizeof(double));
    if (ok && (h->obj.alpha != 0.0 || h->obj.xc != 0.0))
      ok = alloc((void**)&h->rho, (size_t)c.ncg * n * sizeof(double));
  } else if (ok && obj->kind == PLAM_OBJ_HARTREE1D) {
    h->nfpart = hartree_blocks(n);
    ok = alloc((void**)&h->rho, n * sizeof(double)) && alloc((void**)&h->y, n * sizeof(double)) &&
         alloc((void**)&h->blk, 2 * (size_t)h->nfpart * sizeof(double)) &&
         alloc((void**)&h->fpart, (size_t)h->nfpart * sizeof(double));
  }
  if (ok && prm->lambda_rule == PLAM_LAMBDA_DA) ok = alloc((void**)&h->lam, pp * sizeof(double));
  if (ok && obj->kind == PLAM_OBJ_CALLBACK) {
    h->nfpart = 1;
    ok = alloc((void**)&h->fpart, sizeof(double));
  }
  if (ok && prm->final_orth == 2) ok = alloc((void**)&h->Qtmp, (size_t)h->ldw * p * sizeof(double));
  if (ok && obj->kind == PLAM_OBJ_QAP) ok = alloc(&h->qtmp, np_bytes);
  if (ok && prm->variant == PLAM_VARIANT_MOPTQR) ok = alloc(&h->xprev, np_bytes) && alloc(&h->vbuf, np_bytes);
  if (ok && h->sharded) {
    const size_t gcount = std::max((size_t)2 * p * p, (size_t)kColDots * p + kTotDots + 1);
    ok = alloc((void**)&h->gath, (size_t)comm->size * gcount * sizeof(double));
    if (ok && plane > 0) {
      // the potential on the slab and its two halo planes (zero there: only the outputs of
      // interior planes are used)
      ok = alloc(&h->vext, (size_t)(n + 2 * plane) * esz) &&
           alloc(&h->halo, (size_t)4 * plane * p * esz);
      if (ok) ok = cudaMemsetAsync(h->vext, 0, (size_t)(n + 2 * plane) * esz, h->stream) == cudaSuccess;
      if (ok && obj->V)
        ok = cudaMemcpyAsync((char*)h->vext + plane * esz, obj->V, (size_t)n * esz,
                             cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess;
    }
  }
  if (ok && prm->engine != PLAM_ENGINE_GRAPH && prm->precision == PLAM_PREC_FP32 &&
      prm->lambda_rule != PLAM_LAMBDA_DA && prm->variant != PLAM_VARIANT_MOPTQR &&
      ((obj->kind == PLAM_OBJ_HARTREE1D && obj->xc == 0.0 && !chain_objective(h)) ||
       obj->kind == PLAM_OBJ_DENSE)) {
    int dev = 0, sms = 0, optin = 0, coop = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop) {
      resident_plan(n, (int)p, sms, (size_t)optin, &h->r_nblk, &h->r_rows, &h->r_rp, &h->r_smem);
    }
    if (h->r_nblk > 0) {
      const size_t S = 3 * (size_t)p + 7;
      ok = alloc((void**)&h->r_halo, (size_t)h->r_nblk * 2 * p * sizeof(float)) &&
           alloc((void**)&h->r_blk, (size_t)h->r_nblk * 2 * sizeof(double)) &&
           alloc((void**)&h->r_part, (size_t)h->r_nblk * 2 * pp * sizeof(float)) &&
           alloc((void**)&h->r_red, 2 * pp * sizeof(float)) &&
           alloc((void**)&h->r_dots, (size_t)h->r_nblk * S * sizeof(float)) &&
           alloc((void**)&h->r_dred, S * sizeof(double)) &&
           alloc((void**)&h->r_bar, 2 * sizeof(unsigned int)) && alloc((void**)&h->r_err, sizeof(int));
    }
  }
  if (ok && prm->engine == PLAM_ENGINE_RESIDENT && h->r_nblk == 0) {
    free_handle(h);
    snprintf(g_err, sizeof(g_err), "resident engine does not apply to this problem");
    return PLAM_ERR_UNSUPPORTED;
  }
  if (ok) {
    ok = cudaMallocHost((void**)&h->st_host, sizeof(DevState)) == cudaSuccess &&
         cudaMallocHost((void**)&h->info_host, sizeof(int)) == cudaSuccess &&
         cudaMallocHost((void**)&h->scal_host,
                        (kDotBlocks + (size_t)h->nfpart + 8) * sizeof(double)) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_handle(h);
    return PLAM_ERR_NOMEM;
  }
  {
    cudaError_t e = preload_gram_kernels();
    if (e == cudaSuccess) e = preload_update_kernels();
    if (e == cudaSuccess) e = preload_objective_kernels();
    if (e == cudaSuccess && h->r_nblk > 0) e = preload_resident_kernels();
    if (e == cudaSuccess && h->use_tc) e = preload_tc_kernels();
    if (e == cudaSuccess && h->use_tc) e = preload_tc_update_kernels();
    if (e != cudaSuccess) {
      free_handle(h);
      return cuda_fail(e, "kernel preload");
    }
  }
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    free_handle(h);
    return cuda_fail(cudaGetLastError(), "cudaStreamCreate");
  }
  if (reset_state(h) != PLAM_OK || cudaStreamSynchronize(h->stream) != cudaSuccess) {
    free_handle(h);
    return PLAM_ERR_CUDA;
  }
  *out = h;
  return PLAM_OK;
}

}  // namespace

extern "C" {

plam_status_t plam_create(plam_handle_t* out, int64_t n, int64_t p, const plam_objective_t* obj,
                          const plam_params_t* prm, void* stream) {
  return create_impl(out, n, p, obj, prm, stream, nullptr);
}

plam_status_t plam_create_sharded(plam_handle_t* out, int64_t n_local, int64_t p,
                                  const plam_objective_t* obj, const plam_params_t* prm,
                                  const plam_comm_t* comm, void* stream) {
  if (!comm) {
    if (out) *out = nullptr;
    return PLAM_ERR_INVALID;
  }
  return create_impl(out, n_local, p, obj, prm, stream, comm);
}

plam_status_t plam_destroy(plam_handle_t h) {
  if (!h) return PLAM_ERR_INVALID;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
  return PLAM_OK;
}

plam_status_t plam_reset(plam_handle_t h) {
  if (!h) return PLAM_ERR_INVALID;
  return reset_state(h);
}

plam_status_t plam_step(plam_handle_t h, void* X, int64_t ldx, plam_info_t* info) {
  return step_common(h, X, ldx, info, PLAM_VARIANT_PLAM, 0);
}

plam_status_t pcal_step(plam_handle_t h, void* X, int64_t ldx, plam_info_t* info) {
  if (!h) return PLAM_ERR_INVALID;
  return step_common(h, X, ldx, info, PLAM_VARIANT_PCAL, h->prm.lambda_rule == PLAM_LAMBDA2);
}

plam_status_t plam_orthonormalize(plam_handle_t h, const void* X, int64_t ldx, double* Xout,
                                  int64_t ldo, int passes, double* feas) {
  if (!h || !X || !Xout || ldx < h->n || ldo < h->n || passes < 1 || passes > 2)
    return PLAM_ERR_INVALID;
  if (!aligned(X, h->esz) || !aligned(Xout, 8)) return PLAM_ERR_INVALID;
  if (h->prec == PLAM_PREC_FP32 && (const void*)Xout == X) return PLAM_ERR_INVALID;
  if (passes == 2 && !h->Qtmp) {
    if (cudaMalloc((void**)&h->Qtmp, (size_t)h->ldw * h->p * sizeof(double)) != cudaSuccess)
      return PLAM_ERR_NOMEM;
  }
  if (h->prec == PLAM_PREC_FP64)
    return orthonormalize_impl<double>(h, (const double*)X, ldx, Xout, ldo, passes, feas);
  return orthonormalize_impl<float>(h, (const float*)X, ldx, Xout, ldo, passes, feas);
}

static plam_status_t solve_impl(plam_handle_t h, void* X, int64_t ldx, double* Xout, int64_t ldo,
                                plam_info_t* info) {
  if (!h || !X || ldx < h->n || !aligned(X, h->esz) || !halo_rows_ok(h, ldx))
    return PLAM_ERR_INVALID;
  if (Xout && ldo < h->n) return PLAM_ERR_INVALID;
  const int variant = h->prm.variant;
  const int lambda2 = (variant == PLAM_VARIANT_PCAL && h->prm.lambda_rule == PLAM_LAMBDA2);
  plam_status_t st = reset_state(h);
  if (st != PLAM_OK) return st;
  if (!h->tev[0]) {
    for (int i = 0; i < 3; ++i) CK(cudaEventCreate(&h->tev[i]));
  }
  CK(cudaEventRecord(h->tev[0], h->stream));
  // a user gradient runs on the host between the kernels, and MOptQR's retraction checks its
  // Cholesky factorisation on the host: no graph capture
  const int gi = (h->obj.kind == PLAM_OBJ_CALLBACK || variant == PLAM_VARIANT_MOPTQR)
                     ? 0 : h->prm.graph_iters;
  int stop = kRunning;
  if (h->r_nblk > 0) {
    // resident engine: the whole loop in one cooperative launch
    ResidentLaunch L{};
    L.n = h->n; L.p = (int)h->p; L.nblk = h->r_nblk; L.rows = h->r_rows; L.rp = h->r_rp;
    L.smem = h->r_smem; L.kind = h->obj.kind; L.A = (const float*)h->obj.A; L.lda = h->obj.lda;
    L.alpha = h->obj.alpha; L.q = h->obj.quad_scale; L.X = (float*)X; L.ldx = ldx;
    L.R0 = (float*)h->R[0]; L.R1 = (float*)h->R[1]; L.ldr = h->ldw;
    L.halo = h->r_halo; L.blk = h->r_blk; L.part = h->r_part; L.red = h->r_red; L.dots = h->r_dots;
    L.dred = h->r_dred; L.bar = h->r_bar; L.err = h->r_err; L.st = h->st; L.nubuf = h->nubuf;
    L.coef = (float*)h->coef; L.hist = h->hist;
    L.prm = iter_params<float>(h, variant, lambda2);
    if (h->obj.kind == PLAM_OBJ_HARTREE1D) L.prm.f_part = -0.25 * h->obj.alpha;   // its own rho^T y sum
    // failure-detection test hook: extra expected arrivals that never come, so the
    // bounded barrier wait runs out (no fault; the kernel returns a status)
    const char* extra = getenv("PLAM_TEST_BARRIER_EXTRA");
    L.bar_extra = extra ? atoi(extra) : 0;
    CK(cudaMemsetAsync(h->r_bar, 0, 2 * sizeof(unsigned int), h->stream));
    CK(cudaMemsetAsync(h->r_err, 0, sizeof(int), h->stream));
    CK(launch_resident_solve(L, h->stream));
    h->launches += 1;
    st = read_state(h, nullptr, &stop);
    if (st != PLAM_OK) return st;
    if (stop == kTimeout) {
      snprintf(g_err, sizeof(g_err), "resident engine: a grid barrier wait expired");
      return PLAM_ERR_TIMEOUT;
    }
  } else if (gi > 0) {
    if (!h->graph || h->graph_X != X || h->graph_ldx != ldx || h->graph_variant != variant) {
      if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
      }
      // capture graph_iters iterations on the private capture stream
      CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      int total = 0;
      for (int i = 0; i < gi; ++i) {
        int nk = 0;
        st = dispatch_iteration(h, X, ldx, variant, lambda2, h->cap_stream, &nk);
        if (st != PLAM_OK) break;
        total += nk;
      }
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
      if (st != PLAM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
      ce = cudaGraphInstantiate(&h->graph, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
      h->graph_X = X;
      h->graph_ldx = ldx;
      h->graph_variant = variant;
      h->graph_kernels = total;
    }
    const int max_launch = h->prm.maxit / gi + 2;
    for (int l = 0; l < max_launch; ++l) {
      CK(cudaGraphLaunch(h->graph, h->stream));
      h->launches += h->graph_kernels;
      st = read_state(h, nullptr, &stop);
      if (st != PLAM_OK) return st;
      if (stop != kRunning) break;
    }
  } else {
    for (int it = 0; it <= h->prm.maxit; ++it) {
      int nk = 0;
      st = dispatch_iteration(h, X, ldx, variant, lambda2, h->stream, &nk);
      if (st != PLAM_OK) return st;
      h->launches += nk;
      if ((it & 15) == 15 || it == h->prm.maxit || variant == PLAM_VARIANT_MOPTQR) {
        st = read_state(h, nullptr, &stop);
        if (st != PLAM_OK) return st;
        if (stop != kRunning) break;
        if (variant == PLAM_VARIANT_MOPTQR) {   // the retraction's Cholesky of V^T V
          CK(cudaMemcpyAsync(h->info_host, h->info, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
          CK(cudaStreamSynchronize(h->stream));
          if (*h->info_host != 0) {
            snprintf(g_err, sizeof(g_err), "MOptQR retraction: Cholesky pivot %d not positive",
                     *h->info_host);
            return PLAM_ERR_CHOLESKY;
          }
        }
      }
    }
    st = read_state(h, nullptr, &stop);
    if (st != PLAM_OK) return st;
  }
  nvtxRangePop();   // the iterations (profiler timelines: "Func" + "BLAS3")
  nvtxRangePushA("plam_solve: final orthonormalisation");
  plam_info_t tmp;
  plam_info_t* inf = info ? info : &tmp;
  CK(cudaEventRecord(h->tev[1], h->stream));
  st = read_state(h, inf, &stop);
  if (st != PLAM_OK) return st;
  inf->f_orth = inf->kkt_orth = inf->feas_orth = NAN;
  {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->tev[0], h->tev[1]));
    inf->ms_iterations = ms;
    inf->ms_orth = 0.0;
  }
  if (stop == kDiverged) return PLAM_ERR_DIVERGED;
  if (h->prm.final_orth > 0 && Xout) {
    double feas = NAN;
    st = plam_orthonormalize(h, X, ldx, Xout, ldo, h->prm.final_orth,
                             h->prm.orth_metrics ? &feas : nullptr);
    if (st != PLAM_OK) return st;
    inf->feas_orth = feas;
    // Table "orth step": f and KKT of the orthonormalised output
    if (!h->prm.orth_metrics) {
    } else if (h->prec == PLAM_PREC_FP64) {
      st = post_orth_metrics<double>(h, Xout, ldo, &inf->f_orth, &inf->kkt_orth);
    } else {
      float* Qf = (float*)h->R[0];
      int64_t bx = (h->n + 255) / 256;
      if (bx > 64) bx = 64;
      round_to_float_kernel<<<dim3((unsigned)bx, (unsigned)h->p), 256, 0, h->stream>>>(
          h->n, (int)h->p, Xout, ldo, Qf, h->ldw);
      CK(cudaGetLastError());
      h->launches += 1;
      st = post_orth_metrics<float>(h, Qf, h->ldw, &inf->f_orth, &inf->kkt_orth);
    }
    if (st != PLAM_OK) return st;
    CK(cudaEventRecord(h->tev[2], h->stream));
    CK(cudaEventSynchronize(h->tev[2]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->tev[1], h->tev[2]));
    inf->ms_orth = ms;
  }
  return stop == kConverged ? PLAM_OK : PLAM_ERR_NOT_CONVERGED;
}

plam_status_t plam_solve(plam_handle_t h, void* X, int64_t ldx, double* Xout, int64_t ldo,
                         plam_info_t* info) {
  // NVTX ranges for profiler timelines (no cost without a profiler attached): the iterations,
  // then the final orthonormalisation (the paper's "Orth" category, Section 5.4)
  nvtxRangePushA("plam_solve");
  nvtxRangePushA("plam_solve: iterations");
  // solve_impl swaps the inner range for "final orthonormalisation" on its way out: two pops
  // here on every path
  plam_status_t st = solve_impl(h, X, ldx, Xout, ldo, info);
  nvtxRangePop();
  nvtxRangePop();
  return st;
}

int plam_solve_engine(plam_handle_t h) {
  if (!h) return -1;
  if (h->r_nblk > 0) return PLAM_ENGINE_RESIDENT;
  const int gi = (h->obj.kind == PLAM_OBJ_CALLBACK || h->prm.variant == PLAM_VARIANT_MOPTQR)
                     ? 0 : h->prm.graph_iters;
  return gi > 0 ? PLAM_ENGINE_GRAPH : 0;
}

plam_status_t plam_energy(plam_handle_t h, const void* X, int64_t ldx, double* f_dev) {
  if (!h || !X || !f_dev || ldx < h->n || !aligned(X, h->esz)) return PLAM_ERR_INVALID;
  if (h->sharded) return PLAM_ERR_UNSUPPORTED;
  plam_status_t st = h->prec == PLAM_PREC_FP64
                         ? energy_device_impl<double>(h, (const double*)X, ldx, f_dev)
                         : energy_device_impl<float>(h, (const float*)X, ldx, f_dev);
  return st;
}

plam_status_t plam_energy_backward(plam_handle_t h, const void* X, int64_t ldx,
                                   const double* scale_dev, void* G, int64_t ldg) {
  if (!h || !X || !G || ldx < h->n || ldg < h->n) return PLAM_ERR_INVALID;
  if (h->sharded) return PLAM_ERR_UNSUPPORTED;
  if (!aligned(X, h->esz) || !aligned(G, h->esz)) return PLAM_ERR_INVALID;
  return h->prec == PLAM_PREC_FP64
             ? energy_backward_impl<double>(h, (const double*)X, ldx, scale_dev, (double*)G, ldg)
             : energy_backward_impl<float>(h, (const float*)X, ldx, scale_dev, (float*)G, ldg);
}

plam_status_t plam_energy_grad(plam_handle_t h, const void* X, int64_t ldx, void* G, int64_t ldg,
                               double* f) {
  if (!h || !X || !G || ldx < h->n || ldg < h->n) return PLAM_ERR_INVALID;
  if (h->sharded) return PLAM_ERR_UNSUPPORTED;
  if (!aligned(X, h->esz) || !aligned(G, h->esz)) return PLAM_ERR_INVALID;
  if (h->prec == PLAM_PREC_FP64)
    return energy_impl<double>(h, (const double*)X, ldx, (double*)G, ldg, f);
  return energy_impl<float>(h, (const float*)X, ldx, (float*)G, ldg, f);
}

plam_status_t plam_grams(plam_handle_t h, const void* X, int64_t ldx, const void* G, int64_t ldg,
                         double* B, double* C) {
  if (!h || !X || !B || ldx < h->n || (G && (ldg < h->n || !C))) return PLAM_ERR_INVALID;
  if (h->sharded) return PLAM_ERR_UNSUPPORTED;
  const int p = (int)h->p;
  if (h->prec == PLAM_PREC_FP64) {
    CK((launch_gram_partial<double, double>(h->n, p, (const double*)X, ldx, (const double*)G, ldg,
                                             h->rows_per_chunk, h->nchunks, (double*)h->part,
                                             nullptr, h->stream)));
    CK(launch_gram_reduce<double>(p, h->nchunks, G != nullptr, (const double*)h->part, B, C,
                                  h->stream));
  } else if (h->use_tc && tc_gram_supported(X, ldx, G, ldg)) {
    TcGramPlan pl = h->tc;
    if (!G) tc_gram_plan(h->n, p, 0, &pl, pl.pair);
    if (pl.nchunks > h->tc.nchunks) pl = h->tc;   // the workspace is sized for the with-G plan
    CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
    CK(launch_tc_gram(h->n, p, (const float*)X, ldx, (const float*)G, ldg, pl, (float*)h->part,
                      h->tc_err, nullptr, 0.0, tc_always3(h->prm), h->stream));
    CK(launch_gram_reduce<float>(p, pl.nchunks, G != nullptr, (const float*)h->part, B, C,
                                 h->stream));
    CK(cudaMemcpyAsync(h->info_host, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->launches += 2;
    if (*h->info_host != 0) {
      snprintf(g_err, sizeof(g_err), "tensor-core Gram: a pipeline wait expired");
      return PLAM_ERR_TIMEOUT;
    }
    return PLAM_OK;
  } else {
    CK((launch_gram_partial<float, float>(h->n, p, (const float*)X, ldx, (const float*)G, ldg,
                                           h->rows_per_chunk, h->nchunks, (float*)h->part, nullptr,
                                           h->stream)));
    CK(launch_gram_reduce<float>(p, h->nchunks, G != nullptr, (const float*)h->part, B, C,
                                 h->stream));
  }
  h->launches += 2;
  CK(cudaStreamSynchronize(h->stream));
  return PLAM_OK;
}

plam_status_t plam_time_kernels(plam_handle_t h, void* X, int64_t ldx, int iters, double* ms,
                                int* done) {
  if (!h || !X || !ms || !done || iters < 0 || ldx < h->n || !aligned(X, h->esz))
    return PLAM_ERR_INVALID;
  const int variant = h->prm.variant;
  const int lambda2 = (variant == PLAM_VARIANT_PCAL && h->prm.lambda_rule == PLAM_LAMBDA2);
  cudaEvent_t ev[7];
  for (int i = 0; i < 7; ++i) CK(cudaEventCreate(&ev[i]));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  int it = 0;
  plam_status_t st = PLAM_OK;
  for (; it < iters; ++it) {
    int stop = 0;
    st = read_state(h, nullptr, &stop);
    if (st != PLAM_OK || stop != kRunning) break;
    int nk = 0;
    st = dispatch_iteration(h, X, ldx, variant, lambda2, h->stream, &nk, ev);
    if (st != PLAM_OK) break;
    h->launches += nk;
    cudaError_t e = cudaEventSynchronize(ev[6]);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cudaEventSynchronize");
      break;
    }
    for (int i = 0; i < 6; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      acc[i] += t;
    }
  }
  for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
  for (int i = 0; i < 6; ++i) ms[i] = it > 0 ? acc[i] / it : 0.0;
  *done = it;
  return st;
}

plam_status_t plam_last_iteration(plam_handle_t h, void* R, int64_t ldr, void* M,
                                  double* colsums, double* bb) {
  if (!h || (R && (ldr < h->n || !aligned(R, h->esz))) || (M && !aligned(M, h->esz)))
    return PLAM_ERR_INVALID;
  CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const DevState s = *h->st_host;
  if (s.nrec == 0) return PLAM_ERR_INVALID;            // no iterate evaluated since the reset
  // the latest evaluated iterate: k - 1 after an update, k when the run stopped at k
  const int k_last = s.k - (s.stop == kRunning ? 1 : 0);
  const int64_t n = h->n, p = h->p;
  if (R) {
    const void* src = h->R[k_last & 1];
    CK(cudaMemcpy2DAsync(R, (size_t)ldr * h->esz, src, (size_t)h->ldw * h->esz, (size_t)n * h->esz,
                         (size_t)p, cudaMemcpyDeviceToDevice, h->stream));
  }
  if (M)
    CK(cudaMemcpyAsync(M, h->Mt, (size_t)p * p * h->esz, cudaMemcpyDeviceToDevice, h->stream));
  if (colsums)
    CK(cudaMemcpyAsync(colsums, h->sums, (size_t)kColDots * p * sizeof(double),
                       cudaMemcpyDeviceToHost, h->stream));
  if (bb)
    CK(cudaMemcpyAsync(bb, h->sums + kColDots * p, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PLAM_OK;
}

}  // extern "C"

namespace {

// Layout of a checkpoint (plam_get_state): this header, the DevState, both parity halves of
// the column scales (storage type) and of the column norms (double), the residual R^{k-1}
// that the next iteration's Barzilai-Borwein differences read (n x p, packed), and, when the
// handle has them, the dual-ascent multiplier (p x p double) and MOptQR's X^{k-1} (n x p).
struct StateHeader {
  uint32_t magic, version;
  int64_t n, p;
  int32_t prec, variant, has_lam, has_xprev;
  uint64_t bytes;
};
constexpr uint32_t kStateMagic = 0x4d414c50u;   // "PLAM"

size_t state_bytes(const plam_handle_s* h) {
  const size_t np = (size_t)h->n * h->p * h->esz;
  size_t b = sizeof(StateHeader) + sizeof(DevState) + 2 * (2 * (size_t)h->p + 1) * h->esz +
             2 * (size_t)h->p * sizeof(double) + np;
  if (h->lam) b += (size_t)h->p * h->p * sizeof(double);
  if (h->xprev) b += np;
  return b;
}

}  // namespace

extern "C" {

size_t plam_state_bytes(plam_handle_t h) { return h ? state_bytes(h) : 0; }

plam_status_t plam_get_state(plam_handle_t h, void* buf, size_t bytes) {
  if (!h || !buf || bytes < state_bytes(h)) return PLAM_ERR_INVALID;
  CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const DevState ds = *h->st_host;
  unsigned char* o = (unsigned char*)buf;
  StateHeader hd{kStateMagic, 1u, h->n, h->p, h->prec, h->prm.variant, h->lam != nullptr,
                 h->xprev != nullptr, (uint64_t)state_bytes(h)};
  memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  memcpy(o, &ds, sizeof(ds));
  o += sizeof(ds);
  const size_t w = h->esz, cb = 2 * (2 * (size_t)h->p + 1) * w, nb = 2 * (size_t)h->p * 8;
  CK(cudaMemcpyAsync(o, h->coef, cb, cudaMemcpyDeviceToHost, h->stream));
  o += cb;
  CK(cudaMemcpyAsync(o, h->nubuf, nb, cudaMemcpyDeviceToHost, h->stream));
  o += nb;
  // R^{k-1}: the buffer the next iteration (k = ds.k) reads as the previous residual
  const void* rprev = h->R[(ds.k + 1) & 1];
  CK(cudaMemcpy2DAsync(o, (size_t)h->n * w, rprev, (size_t)h->ldw * w, (size_t)h->n * w,
                       (size_t)h->p, cudaMemcpyDeviceToHost, h->stream));
  o += (size_t)h->n * h->p * w;
  if (h->lam) {
    CK(cudaMemcpyAsync(o, h->lam, (size_t)h->p * h->p * 8, cudaMemcpyDeviceToHost, h->stream));
    o += (size_t)h->p * h->p * 8;
  }
  if (h->xprev)
    CK(cudaMemcpy2DAsync(o, (size_t)h->n * w, h->xprev, (size_t)h->ldw * w, (size_t)h->n * w,
                         (size_t)h->p, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PLAM_OK;
}

plam_status_t plam_set_state(plam_handle_t h, const void* buf, size_t bytes) {
  if (!h || !buf || bytes < sizeof(StateHeader)) return PLAM_ERR_INVALID;
  StateHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != 1u || hd.n != h->n || hd.p != h->p ||
      hd.prec != h->prec || hd.variant != h->prm.variant || hd.has_lam != (h->lam != nullptr) ||
      hd.has_xprev != (h->xprev != nullptr) || hd.bytes != state_bytes(h) || bytes < hd.bytes)
    return PLAM_ERR_INVALID;
  const unsigned char* o = (const unsigned char*)buf + sizeof(hd);
  DevState ds;
  memcpy(&ds, o, sizeof(ds));
  o += sizeof(ds);
  const size_t w = h->esz, cb = 2 * (2 * (size_t)h->p + 1) * w, nb = 2 * (size_t)h->p * 8;
  CK(cudaStreamSynchronize(h->stream));
  *h->st_host = ds;
  CK(cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->coef, o, cb, cudaMemcpyHostToDevice, h->stream));
  o += cb;
  CK(cudaMemcpyAsync(h->nubuf, o, nb, cudaMemcpyHostToDevice, h->stream));
  o += nb;
  CK(cudaMemcpy2DAsync(h->R[(ds.k + 1) & 1], (size_t)h->ldw * w, o, (size_t)h->n * w,
                       (size_t)h->n * w, (size_t)h->p, cudaMemcpyHostToDevice, h->stream));
  o += (size_t)h->n * h->p * w;
  if (h->lam) {
    CK(cudaMemcpyAsync(h->lam, o, (size_t)h->p * h->p * 8, cudaMemcpyHostToDevice, h->stream));
    o += (size_t)h->p * h->p * 8;
  }
  if (h->xprev)
    CK(cudaMemcpy2DAsync(h->xprev, (size_t)h->ldw * w, o, (size_t)h->n * w, (size_t)h->n * w,
                         (size_t)h->p, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(h->ticket, 0, sizeof(unsigned int), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PLAM_OK;
}

plam_status_t plam_history(plam_handle_t h, double* out, int cap, int* count) {
  if (!h || !out || !count || cap < 0) return PLAM_ERR_INVALID;
  CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int nrec = h->st_host->nrec;
  if (nrec > cap) nrec = cap;
  if (nrec > 0)
    CK(cudaMemcpy(out, h->hist, (size_t)nrec * 5 * sizeof(double), cudaMemcpyDeviceToHost));
  *count = nrec;
  return PLAM_OK;
}

int64_t plam_kernel_launches(plam_handle_t h) { return h ? h->launches : -1; }

const char* plam_last_error(void) { return g_err; }

int plam_version(void) { return 100; }

}  // extern "C"

// ---------------------------------------------------------------- batched solves

struct plam_batch_s {
  int count = 0;
  cudaStream_t stream = nullptr;
  plam::BatchParams prm{};
  int tile = 128;
  int grid = 1;
  plam::BatchDesc* desc = nullptr;        // device
  int* order = nullptr;                   // device
  int* next = nullptr;                    // device
  plam_info_t* info = nullptr;            // device
  plam_info_t* info_host = nullptr;       // pinned
  float* work = nullptr;                  // device: G, R0, R1 of every problem
  std::vector<plam::BatchDesc> hdesc;
  cudaGraphExec_t graph = nullptr;
  int graph_tile = 0;
};

namespace {

void free_batch(plam_batch_s* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  void* dev[] = {b->desc, b->order, b->next, b->info, b->work};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (b->info_host) cudaFreeHost(b->info_host);
  delete b;
}

}  // namespace

extern "C" {

plam_status_t plam_batch_create(plam_batch_t* out, const plam_batch_problem_t* probs, int count,
                                const plam_params_t* prm, void* stream) {
  using namespace plam;
  if (!out) return PLAM_ERR_INVALID;
  *out = nullptr;
  if (!probs || count < 1 || !prm || validate_params(prm) != PLAM_OK) return PLAM_ERR_INVALID;
  if (prm->precision != PLAM_PREC_FP32 || prm->lambda_rule == PLAM_LAMBDA_DA) {
    snprintf(g_err, sizeof(g_err), "plam_batch_create: FP32 mode with a closed-form multiplier only");
    return PLAM_ERR_UNSUPPORTED;
  }
  size_t work = 0;
  for (int i = 0; i < count; ++i) {
    const plam_batch_problem_t& q = probs[i];
    if (q.p < 1 || q.p > 64 || q.n < 2 * q.p || !q.A || !q.X || q.lda < q.n || q.ldx < q.n ||
        !aligned(q.A, 4) || !aligned(q.X, 4) || (q.Q && (q.ldq < q.n || !aligned(q.Q, 8))))
      return PLAM_ERR_INVALID;
    work += 3 * (size_t)round_up(q.n, 32) * (size_t)q.p;
  }
  plam_batch_s* b = new (std::nothrow) plam_batch_s();
  if (!b) return PLAM_ERR_NOMEM;
  b->count = count;
  b->stream = (cudaStream_t)stream;
  b->prm.variant = prm->variant;
  b->prm.lambda2 = prm->variant == PLAM_VARIANT_PCAL && prm->lambda_rule == PLAM_LAMBDA2;
  b->prm.eta_rule = prm->eta_rule;
  b->prm.maxit = prm->maxit;
  b->prm.beta = prm->beta;
  b->prm.eta0_user = prm->eta0;
  b->prm.gamma = prm->eta_gamma;
  b->prm.tol = prm->tol;
  b->prm.eta_min = prm->eta_min;
  b->prm.eta_max = prm->eta_max;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = count < sms ? count : sms;
  bool ok = cudaMalloc((void**)&b->desc, count * sizeof(BatchDesc)) == cudaSuccess &&
            cudaMalloc((void**)&b->order, count * sizeof(int)) == cudaSuccess &&
            cudaMalloc((void**)&b->next, sizeof(int)) == cudaSuccess &&
            cudaMalloc((void**)&b->info, count * sizeof(plam_info_t)) == cudaSuccess &&
            cudaMalloc((void**)&b->work, work * sizeof(float)) == cudaSuccess &&
            cudaMallocHost((void**)&b->info_host, count * sizeof(plam_info_t)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_batch(b);
    return PLAM_ERR_NOMEM;
  }
  b->hdesc.resize(count);
  float* w = b->work;
  for (int i = 0; i < count; ++i) {
    const plam_batch_problem_t& q = probs[i];
    BatchDesc& d = b->hdesc[i];
    d.n = q.n; d.p = (int)q.p; d.pad_ = 0;
    d.A = (const float*)q.A; d.lda = q.lda; d.X = (float*)q.X; d.ldx = q.ldx;
    d.ldw = round_up(q.n, 32);
    d.G = w; w += d.ldw * q.p;
    d.R0 = w; w += d.ldw * q.p;
    d.R1 = w; w += d.ldw * q.p;
    d.Q = q.Q; d.ldq = q.ldq;
  }
  // the queue: largest n^2 p first, so that the longest problems start first
  std::vector<int> ord(count);
  for (int i = 0; i < count; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    const double cx = (double)probs[x].n * probs[x].n * probs[x].p;
    const double cy = (double)probs[y].n * probs[y].n * probs[y].p;
    return cx > cy;
  });
  ok = cudaMemcpy(b->desc, b->hdesc.data(), count * sizeof(BatchDesc), cudaMemcpyHostToDevice) ==
           cudaSuccess &&
       cudaMemcpy(b->order, ord.data(), count * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       preload_batched_kernels() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_batch(b);
    return PLAM_ERR_CUDA;
  }
  *out = b;
  return PLAM_OK;
}

plam_status_t plam_batch_set_tile(plam_batch_t b, int tile_rows) {
  if (!b || (tile_rows != 64 && tile_rows != 128 && tile_rows != 256)) return PLAM_ERR_INVALID;
  b->tile = tile_rows;
  return PLAM_OK;
}

plam_status_t plam_batch_solve(plam_batch_t b, plam_info_t* infos) {
  using namespace plam;
  if (!b) return PLAM_ERR_INVALID;
  if (!b->graph || b->graph_tile != b->tile) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(b->next, 0, sizeof(int), cs);
    if (ce == cudaSuccess)
      ce = launch_batched(b->tile, b->desc, b->order, b->count, b->next, b->info, b->prm, b->grid,
                          cs);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(b->info_host, b->info, b->count * sizeof(plam_info_t),
                           cudaMemcpyDeviceToHost, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "batched solve graph");
    b->graph_tile = b->tile;
  }
  CK(cudaGraphLaunch(b->graph, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  if (infos) {
    memcpy(infos, b->info_host, b->count * sizeof(plam_info_t));
    for (int i = 0; i < b->count; ++i) infos[i].ms_iterations = infos[i].ms_orth = NAN;
  }
  return PLAM_OK;
}

plam_status_t plam_batch_autotune(plam_batch_t b, int iters, int* tile_rows, double* ms) {
  using namespace plam;
  if (!b || iters < 1) return PLAM_ERR_INVALID;
  // back up every start, time each tile height from the same starts, restore
  size_t tot = 0;
  for (const BatchDesc& d : b->hdesc) tot += (size_t)d.n * d.p;
  float* bak = nullptr;
  if (cudaMalloc((void**)&bak, tot * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return PLAM_ERR_NOMEM;
  }
  auto copy_all = [&](bool save) -> cudaError_t {
    size_t off = 0;
    for (const BatchDesc& d : b->hdesc) {
      cudaError_t e = save ? cudaMemcpy2DAsync(bak + off, d.n * sizeof(float), d.X,
                                               d.ldx * sizeof(float), d.n * sizeof(float), d.p,
                                               cudaMemcpyDeviceToDevice, b->stream)
                           : cudaMemcpy2DAsync(d.X, d.ldx * sizeof(float), bak + off,
                                               d.n * sizeof(float), d.n * sizeof(float), d.p,
                                               cudaMemcpyDeviceToDevice, b->stream);
      if (e != cudaSuccess) return e;
      off += (size_t)d.n * d.p;
    }
    return cudaSuccess;
  };
  BatchParams tp = b->prm;
  tp.maxit = iters;
  tp.tol = 0.0;
  const int tiles[3] = {64, 128, 256};
  int best = b->tile;
  double best_ms = INFINITY;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t ce = copy_all(true);
  for (int i = 0; i < 3 && ce == cudaSuccess; ++i) {
    for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {   // first run warms up
      ce = cudaMemsetAsync(b->next, 0, sizeof(int), b->stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, b->stream);
      if (ce == cudaSuccess)
        ce = launch_batched(tiles[i], b->desc, b->order, b->count, b->next, b->info, tp, b->grid,
                            b->stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, b->stream);
      if (ce == cudaSuccess) ce = copy_all(false);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
      float t = 0.f;
      if (ce == cudaSuccess && rep == 1 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
          t < best_ms) {
        best_ms = t;
        best = tiles[i];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(bak);
  if (ce != cudaSuccess) return cuda_fail(ce, "batched autotune");
  b->tile = best;
  if (tile_rows) *tile_rows = best;
  if (ms) *ms = best_ms;
  return PLAM_OK;
}

plam_status_t plam_batch_destroy(plam_batch_t b) {
  if (!b) return PLAM_ERR_INVALID;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_batch(b);
  return PLAM_OK;
}

}  // extern "C"
