// Helpers shared by the host-side files of the C ABI (lrdm_api.cu: contexts,
// forward, least squares, adjoint; lrdm_lrdma.cu: the accumulated LRDM
// driver; lrdm_kpoint_api.cu: Brillouin-zone-sampled systems).  Not part of
// the public interface.
#pragma once

#include <vector>

#include "lrdm_internal.h"

namespace lrdm {
namespace api {

// CUDA / cuFFT result -> lrdm_status (LRDM_DEBUG=1 prints the CUDA error)
lrdm_status from_cuda(cudaError_t e);
lrdm_status from_cufft(cufftResult r);

#define LRDM_CK(expr)                          \
  do {                                         \
    lrdm_status _s = (expr);                   \
    if (_s != LRDM_OK) return _s;              \
  } while (0)
#define LRDM_CU(expr) LRDM_CK(from_cuda(expr))
#define LRDM_FFT(expr) LRDM_CK(from_cufft(expr))

// Device allocation owned by the context (freed by lrdm_destroy), zeroed
// unless zero == false.
template <typename T>
lrdm_status dalloc(lrdm_ctx* ctx, T** p, size_t count, bool zero = true) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return from_cuda(e);
  ctx->allocs.push_back(q);
  if (zero) {
    e = cudaMemset(q, 0, count * sizeof(T));
    if (e != cudaSuccess) return from_cuda(e);
  }
  *p = static_cast<T*>(q);
  return LRDM_OK;
}

inline bool is_tc(int prec) { return prec == LRDM_TF32 || prec == LRDM_BF16X3; }
size_t io_size(int io);
// numerically stable Fermi function f = 1/(1 + exp(x))
double fermi_host(double x);

// profiling records (lrdm_profile_enable): event pairs and launch counts
int prof_begin(lrdm_ctx* ctx, int kind, cudaStream_t st);
void prof_end(lrdm_ctx* ctx, int i, cudaStream_t st);
void count(lrdm_ctx* ctx, int n);

// Poisson transforms, symbol table and buffers of system S; V_H in place in
// S.fft_real for all k_max slots
lrdm_status setup_poisson(lrdm_ctx* ctx, SysState& S, cudaStream_t st);
lrdm_status hartree(lrdm_ctx* ctx, SysState& S, int K, cudaStream_t st);
// grouped tensor-core launch of ctx->tc_entries (gemm 1: projection, 2: response)
lrdm_status tc_group(lrdm_ctx* ctx, int gemm, int out_is_io, cudaStream_t st);
// launch-shape tuner of the tensor-core contractions (options.autotune)
lrdm_status autotune(lrdm_ctx* ctx, cudaStream_t st);
void free_ctx(lrdm_ctx* ctx);

// the forward of every system of a context; one forward call of the direction
// drivers (system sys only; k-point contexts run kp_forward)
lrdm_status forward_all(lrdm_ctx* ctx, const void* const* v, const int* K, void* const* f,
                        double* dmu_out, cudaStream_t st);
lrdm_status forward_one(lrdm_ctx* ctx, int sys, const void* const* v, const int* K, void* const* f,
                        cudaStream_t st);
// Brillouin-zone-sampled contexts (lrdm_kpoint_api.cu)
lrdm_status kp_forward(lrdm_ctx* ctx, const void* v, int K, void* f_out, double* dmu_out, cudaStream_t st);
lrdm_status kp_backward(lrdm_ctx* ctx, const void* const* f_bar, void* const* v_bar,
                        double* const* eps_bar, double* const* occ_bar, cudaStream_t st);

// CUDA graph of a forward call: captured on the first call with a given key
// (buffers, K's, stream), replayed afterwards.  Not used on the legacy
// default stream or while profiling.
bool use_graph(const lrdm_ctx* ctx, cudaStream_t st);
template <typename Body>
lrdm_status graph_call(lrdm_ctx* ctx, const std::vector<const void*>& key, cudaStream_t st, Body body) {
  if (ctx->graph_exec && key == ctx->graph_key) return from_cuda(cudaGraphLaunch(ctx->graph_exec, st));
  if (ctx->graph_exec) {
    cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
  }
  LRDM_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  lrdm_status rc = body();
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != LRDM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  LRDM_CU(e);
  e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
  cudaGraphDestroy(g);
  LRDM_CU(e);
  ctx->graph_key = key;
  return from_cuda(cudaGraphLaunch(ctx->graph_exec, st));
}

}  // namespace api
}  // namespace lrdm
