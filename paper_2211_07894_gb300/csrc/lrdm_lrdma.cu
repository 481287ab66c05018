// The accumulated LRDM driver (LRDMA, §II.B.1) behind lrdm_lrdma_*: a
// history of directions and Gateaux derivatives kept across SCF steps,
// independently of any context (each step brings a new subspace).
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "api_common.h"

using namespace lrdm;
using namespace lrdm::api;

struct lrdm_lrdma {
  long long n = 0;
  int io = LRDM_DTYPE_F64;
  double w = 0.0;
  int cap = 0;
  int m = 0;                         // kept directions
  bool clear_next = false;
  bool have_lin = false;
  int device = 0;
  void* U = nullptr;                 // [cap][n]
  void* T = nullptr;                 // [cap][n]
  void* R_lin = nullptr;             // [n]
  double* gs = nullptr;              // Gram-Schmidt / norm scratch
  double* norm = nullptr;            // [2]
  double* ls_partial = nullptr;
  double* ls_coef = nullptr;
  double* ls_scal = nullptr;
  double* upd_partial = nullptr;
  int* status = nullptr;
  std::vector<void*> allocs;
};

namespace {

template <typename T>
lrdm_status lalloc(lrdm_lrdma* a, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, (count ? count : 1) * sizeof(T)) != cudaSuccess) return LRDM_ERR_OOM;
  a->allocs.push_back(q);
  if (cudaMemset(q, 0, (count ? count : 1) * sizeof(T)) != cudaSuccess) return LRDM_ERR_CUDA;
  *p = static_cast<T*>(q);
  return LRDM_OK;
}

void lrdma_free(lrdm_lrdma* a) {
  if (!a) return;
  for (void* p : a->allocs) cudaFree(p);
  delete a;
}

// s_rel of the low-rank model over the first m kept pairs on R; with rho and
// alpha != 0 also rho <- rho - alpha sum a_k v_k (v = U or, for the linear
// prediction, T).  Host value of s_rel.
lrdm_status lrdma_ls(lrdm_lrdma* a, const void* R, const void* v, int m, double alpha, void* rho,
                     double rcond, double* s_rel, cudaStream_t st, const AllReduce* ar) {
  int ar_failed = 0;
  LRDM_CU(launch_ls(R, v, a->T, a->io, m, a->n, a->w, alpha, rcond, rho, a->ls_coef, nullptr,
                    nullptr, a->ls_partial, a->ls_scal, a->upd_partial, a->status, st, ar,
                    &ar_failed));
  if (ar_failed) return LRDM_ERR_COLLECTIVE;
  LRDM_CU(cudaMemcpyAsync(s_rel, a->ls_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  LRDM_CU(cudaStreamSynchronize(st));
  return LRDM_OK;
}

}  // namespace

extern "C" {

void lrdm_lrdma_default_params(lrdm_lrdma_params* p) {
  if (!p) return;
  p->s_tol = 0.3;
  p->beta_tol = 0.1;
  p->r_norm_clear = 1.0;
  p->alpha = -1.0;
  p->r_max_iter = 5;
  p->r_max = KMAX_LIMIT;
}

lrdm_status lrdm_lrdma_create(lrdm_lrdma** out, long long n, int io_dtype, double w, int capacity) {
  if (!out) return LRDM_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || !(w > 0.0) || capacity < 1 || capacity > KMAX_LIMIT) return LRDM_ERR_INVALID_ARG;
  if (io_dtype != LRDM_DTYPE_F64 && io_dtype != LRDM_DTYPE_F32) return LRDM_ERR_INVALID_ARG;
  lrdm_lrdma* a = new (std::nothrow) lrdm_lrdma();
  if (!a) return LRDM_ERR_OOM;
  a->n = n;
  a->io = io_dtype;
  a->w = w;
  a->cap = capacity;
  cudaGetDevice(&a->device);
  const size_t isz = io_size(io_dtype);
  const int maxval = KMAX_LIMIT * (KMAX_LIMIT + 1) / 2 + KMAX_LIMIT + 1;
  lrdm_status rc;
  char* u = nullptr;
  char* t = nullptr;
  char* r = nullptr;
  if ((rc = lalloc(a, &u, (size_t)capacity * n * isz)) != LRDM_OK ||
      (rc = lalloc(a, &t, (size_t)capacity * n * isz)) != LRDM_OK ||
      (rc = lalloc(a, &r, (size_t)n * isz)) != LRDM_OK ||
      (rc = lalloc(a, &a->gs, gram_schmidt_scratch())) != LRDM_OK ||
      (rc = lalloc(a, &a->norm, 2)) != LRDM_OK ||
      (rc = lalloc(a, &a->ls_partial, (size_t)LS_BLOCKS * maxval)) != LRDM_OK ||
      (rc = lalloc(a, &a->ls_coef, KMAX_LIMIT)) != LRDM_OK ||
      (rc = lalloc(a, &a->ls_scal, 4)) != LRDM_OK ||
      (rc = lalloc(a, &a->upd_partial, UPD_BLOCKS)) != LRDM_OK ||
      (rc = lalloc(a, &a->status, 1)) != LRDM_OK) {
    lrdma_free(a);
    return rc;
  }
  a->U = u;
  a->T = t;
  a->R_lin = r;
  *out = a;
  return LRDM_OK;
}

lrdm_status lrdm_lrdma_get_state(const lrdm_lrdma* a, int* m, int* flags) {
  if (!a || !m || !flags) return LRDM_ERR_INVALID_ARG;
  *m = a->m;
  *flags = (a->clear_next ? LRDM_LRDMA_CLEAR_NEXT : 0) | (a->have_lin ? LRDM_LRDMA_HAVE_LIN : 0);
  return LRDM_OK;
}

lrdm_status lrdm_lrdma_export(const lrdm_lrdma* a, void* U, void* T, void* R_lin, void* stream) {
  if (!a || !U || !T || !R_lin) return LRDM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vb = (size_t)a->n * io_size(a->io);
  if (a->m > 0) {
    LRDM_CU(cudaMemcpyAsync(U, a->U, a->m * vb, cudaMemcpyDefault, st));
    LRDM_CU(cudaMemcpyAsync(T, a->T, a->m * vb, cudaMemcpyDefault, st));
  }
  LRDM_CU(cudaMemcpyAsync(R_lin, a->R_lin, vb, cudaMemcpyDefault, st));
  return from_cuda(cudaStreamSynchronize(st));
}

lrdm_status lrdm_lrdma_import(lrdm_lrdma* a, int m, int flags, const void* U, const void* T,
                              const void* R_lin, void* stream) {
  if (!a || m < 0 || m > a->cap || (m > 0 && (!U || !T)) || !R_lin) return LRDM_ERR_INVALID_ARG;
  if (flags & ~(LRDM_LRDMA_CLEAR_NEXT | LRDM_LRDMA_HAVE_LIN)) return LRDM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vb = (size_t)a->n * io_size(a->io);
  if (m > 0) {
    LRDM_CU(cudaMemcpyAsync(a->U, U, m * vb, cudaMemcpyDefault, st));
    LRDM_CU(cudaMemcpyAsync(a->T, T, m * vb, cudaMemcpyDefault, st));
  }
  LRDM_CU(cudaMemcpyAsync(a->R_lin, R_lin, vb, cudaMemcpyDefault, st));
  LRDM_CU(cudaStreamSynchronize(st));
  a->m = m;
  a->clear_next = (flags & LRDM_LRDMA_CLEAR_NEXT) != 0;
  a->have_lin = (flags & LRDM_LRDMA_HAVE_LIN) != 0;
  return LRDM_OK;
}

lrdm_status lrdm_lrdma_clear(lrdm_lrdma* a) {
  if (!a) return LRDM_ERR_INVALID_ARG;
  a->m = 0;
  a->clear_next = false;
  a->have_lin = false;
  return LRDM_OK;
}

void lrdm_lrdma_destroy(lrdm_lrdma* a) {
  if (!a) return;
  cudaDeviceSynchronize();
  lrdma_free(a);
}

lrdm_status lrdm_lrdma_step(lrdm_lrdma* a, lrdm_ctx* ctx, int sys, const void* R, void* rho_inout,
                            const lrdm_lrdma_params* params, lrdm_lrdma_report* report,
                            void* stream) {
  NvtxRange nvtx_("lrdm_lrdma_step");
  if (!a || !ctx || sys < 0 || sys >= ctx->nsys || !R) return LRDM_ERR_INVALID_ARG;
  lrdm_lrdma_params p;
  if (params) p = *params;
  else lrdm_lrdma_default_params(&p);
  SysState& S = ctx->sys[sys];
  if ((long long)S.nspin * S.Ng != a->n || ctx->opt.io_dtype != a->io ||
      std::fabs(S.w - a->w) > 1e-12 * a->w)
    return LRDM_ERR_SHAPE;
  if (p.r_max > a->cap) p.r_max = a->cap;
  if (p.r_max < 1 || p.r_max_iter < 1 || !(p.s_tol >= 0.0) || !isfinite(p.alpha))
    return LRDM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vb = (size_t)a->n * io_size(a->io);
  const double rcond = ctx->opt.pinv_rcond;
  char* U = static_cast<char*>(a->U);
  char* T = static_cast<char*>(a->T);
  // a row-sharded context: the history holds this rank's rows, and every grid
  // sum of the step is summed over the ranks
  const AllReduce* ar = ctx->rows ? &ctx->ar : nullptr;
  int arf = 0;
  // ||R|| and, with a history, ||R_lin||
  LRDM_CU(launch_norm(R, a->io, a->n, a->w, a->gs, a->norm, st, ar, &arf));
  if (a->m > 0 && a->have_lin)
    LRDM_CU(launch_norm(a->R_lin, a->io, a->n, a->w, a->gs, a->norm + 1, st, ar, &arf));
  if (arf) return LRDM_ERR_COLLECTIVE;
  double nrm[2] = {0.0, 0.0};
  LRDM_CU(cudaMemcpyAsync(nrm, a->norm, sizeof(nrm), cudaMemcpyDeviceToHost, st));
  LRDM_CU(cudaStreamSynchronize(st));
  const double r_norm = nrm[0];
  if (!(r_norm > 0.0) || !isfinite(r_norm)) return LRDM_ERR_INVALID_ARG;
  // decisions (§II.B.1)
  int event;
  double beta = -1.0;
  if (a->clear_next) {
    event = LRDMA_CLEAR_TRUNCATED;
  } else if (a->m > 0) {
    beta = std::fabs(nrm[1] / r_norm - 1.0);
    if (beta > p.beta_tol) {
      event = LRDMA_CLEAR_LINEARITY;
    } else {
      double s_hist = 0.0;
      LRDM_CK(lrdma_ls(a, R, U, a->m, 0.0, nullptr, rcond, &s_hist, st, ar));
      if (s_hist < p.s_tol) event = LRDMA_REUSE;
      else if (r_norm > p.r_norm_clear) event = LRDMA_CLEAR_RESIDUAL;
      else event = LRDMA_ACCUMULATE;
    }
  } else {
    event = LRDMA_FRESH;
  }
  if (event == LRDMA_CLEAR_TRUNCATED || event == LRDMA_CLEAR_LINEARITY || event == LRDMA_CLEAR_RESIDUAL)
    a->m = 0;
  a->clear_next = false;
  int n_new = 0;
  double s_rel = 0.0;
  if (event != LRDMA_REUSE) {
    const bool fresh = a->m == 0;
    int limit = fresh ? p.r_max : std::min(p.r_max_iter, p.r_max - a->m);
    if (limit < 1) {                  // the history is full: rebuild afresh
      a->m = 0;
      limit = p.r_max;
    }
    // first new direction: R normalised, or its complement to the history
    LRDM_CU(launch_gram_schmidt(U, a->m, R, a->io, a->n, a->w, U + a->m * vb, a->gs, a->norm, st, ar,
                                &arf));
    if (arf) return LRDM_ERR_COLLECTIVE;
    std::vector<const void*> v(ctx->nsys, nullptr);
    std::vector<void*> f(ctx->nsys, nullptr);
    std::vector<int> K(ctx->nsys, 0);
    for (;;) {
      v[sys] = U + a->m * vb;
      f[sys] = T + a->m * vb;
      K[sys] = 1;
      LRDM_CK(forward_one(ctx, sys, v.data(), K.data(), f.data(), st));
      ++a->m;
      ++n_new;
      LRDM_CK(lrdma_ls(a, R, U, a->m, 0.0, nullptr, rcond, &s_rel, st, ar));
      if (s_rel < p.s_tol || n_new == limit) break;
      LRDM_CU(launch_gram_schmidt(U, a->m, T + (a->m - 1) * vb, a->io, a->n, a->w, U + a->m * vb,
                                  a->gs, a->norm, st, ar, &arf));
      if (arf) return LRDM_ERR_COLLECTIVE;
    }
    if (!fresh && s_rel >= p.s_tol) a->clear_next = true;
  }
  const double alpha = p.alpha < 0.0 ? (r_norm < 2.0 ? 0.5 : 0.1) : p.alpha;
  // linear prediction of the next residual: R_lin = R - alpha sum a_k t_k
  LRDM_CU(cudaMemcpyAsync(a->R_lin, R, vb, cudaMemcpyDeviceToDevice, st));
  LRDM_CK(lrdma_ls(a, R, T, a->m, alpha, a->R_lin, rcond, &s_rel, st, ar));
  a->have_lin = true;
  if (rho_inout) LRDM_CK(lrdma_ls(a, R, U, a->m, alpha, rho_inout, rcond, &s_rel, st, ar));
  if (report) {
    report->event = event;
    report->rank = a->m;
    report->rank_new = n_new;
    report->s_rel = s_rel;
    report->beta = beta;
    report->r_norm = r_norm;
    report->alpha = alpha;
  }
  return LRDM_OK;
}

}  // extern "C"
