// Gram-Schmidt steps of the Krylov directions of the LRDM step (Eq.
// krylovOrtho, §II.B), in the w-weighted inner product <a, b> = w sum a b
// (summed over spin channels, Eq. innerproductDirectsumHilbertspace):
//   c_k = <t, u_k> (k < K),  u = t - sum_k c_k u_k,  u <- u / ||u||.
// FP64 accumulation throughout; per-block partial sums in a fixed order.
#include "lrdm_internal.h"

#include <math.h>

namespace lrdm {
namespace {

constexpr int KR_BLOCKS = 304;          // 2 x 152 SMs
constexpr int KR_THREADS = 256;

__device__ __forceinline__ double ld_io(const void* p, int io, long long i) {
  return io == LRDM_DTYPE_F64 ? static_cast<const double*>(p)[i]
                              : (double)static_cast<const float*>(p)[i];
}
__device__ __forceinline__ void st_io(void* p, int io, long long i, double x) {
  if (io == LRDM_DTYPE_F64) static_cast<double*>(p)[i] = x;
  else static_cast<float*>(p)[i] = (float)x;
}

__device__ __forceinline__ double block_sum(double x, double* sh) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  __syncthreads();
  return s;                             // valid in thread 0
}

// partial[b][k] = sum over this block's points of t u_k
__global__ void __launch_bounds__(KR_THREADS) k_dots(const void* __restrict__ U, int K,
                                                     const void* __restrict__ t, int io, long long n,
                                                     double* __restrict__ partial) {
  __shared__ double sh[32];
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x)
      acc += ld_io(t, io, r) * ld_io(U, io, (long long)k * n + r);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[(long long)blockIdx.x * K + k] = s;
  }
}

// out = t - sum_k c_k u_k with c_k = w sum_b partial[b][k]; npart[b] = this
// block's sum of out^2
__global__ void __launch_bounds__(KR_THREADS) k_gs_axpy(const void* __restrict__ U, int K,
                                                        const void* __restrict__ t, int io, long long n,
                                                        double w, const double* __restrict__ partial,
                                                        int nblk, void* __restrict__ out,
                                                        double* __restrict__ npart) {
  __shared__ double c[KMAX_LIMIT];
  __shared__ double sh[32];
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(long long)b * K + k];
    c[k] = w * s;
  }
  __syncthreads();
  double acc = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    double x = ld_io(t, io, r);
    for (int k = 0; k < K; ++k) x -= c[k] * ld_io(U, io, (long long)k * n + r);
    st_io(out, io, r, x);
    acc += x * x;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) npart[blockIdx.x] = s;
}

// out /= ||out||_w; norm_out[0] = ||out||_w before scaling (0 leaves out as is)
__global__ void __launch_bounds__(KR_THREADS) k_normalize(void* __restrict__ out, int io, long long n,
                                                          double w, const double* __restrict__ npart,
                                                          int nblk, double* __restrict__ norm_out) {
  __shared__ double nrm;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += npart[b];
    nrm = sqrt(w * s);
    if (blockIdx.x == 0 && norm_out) norm_out[0] = nrm;
  }
  __syncthreads();
  if (!(nrm > 0.0)) return;
  const double inv = 1.0 / nrm;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x)
    st_io(out, io, r, ld_io(out, io, r) * inv);
}

// norm_out[0] = sqrt(w sum_b partial[b])
__global__ void k_norm_finish(const double* __restrict__ partial, int nblk, double w,
                              double* __restrict__ norm_out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) norm_out[0] = sqrt(w * s);
}

}  // namespace

// Row-sharded systems: the per-block partial sums summed over the ranks
// (block by block, so every rank reduces the same values in the same order).
static bool sum_over_ranks(const AllReduce* ar, int* ar_failed, double* buf, long long count,
                           cudaStream_t st) {
  if (!ar || !ar->fn) return true;
  if (ar->fn(ar->user, buf, count, LRDM_DTYPE_F64, st) == 0) return true;
  if (ar_failed) *ar_failed = 1;
  return false;
}

cudaError_t launch_norm(const void* x, int io, long long n, double w, double* scratch,
                        double* norm_out, cudaStream_t st, const AllReduce* ar, int* ar_failed) {
  k_dots<<<KR_BLOCKS, KR_THREADS, 0, st>>>(x, 1, x, io, n, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!sum_over_ranks(ar, ar_failed, scratch, KR_BLOCKS, st)) return cudaSuccess;
  k_norm_finish<<<1, KR_THREADS, 0, st>>>(scratch, KR_BLOCKS, w, norm_out);
  return cudaGetLastError();
}

cudaError_t launch_gram_schmidt(const void* U, int K, const void* t, int io, long long n, double w,
                                void* out, double* scratch, double* norm_out, cudaStream_t st,
                                const AllReduce* ar, int* ar_failed) {
  double* partial = scratch;                            // [KR_BLOCKS][K]
  double* npart = scratch + (size_t)KR_BLOCKS * KMAX_LIMIT;   // [KR_BLOCKS]
  if (K > 0) {
    k_dots<<<KR_BLOCKS, KR_THREADS, 0, st>>>(U, K, t, io, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!sum_over_ranks(ar, ar_failed, partial, (long long)KR_BLOCKS * K, st)) return cudaSuccess;
  }
  k_gs_axpy<<<KR_BLOCKS, KR_THREADS, 0, st>>>(U, K, t, io, n, w, partial, KR_BLOCKS, out, npart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!sum_over_ranks(ar, ar_failed, npart, KR_BLOCKS, st)) return cudaSuccess;
  k_normalize<<<KR_BLOCKS, KR_THREADS, 0, st>>>(out, io, n, w, npart, KR_BLOCKS, norm_out);
  return cudaGetLastError();
}

size_t gram_schmidt_scratch() { return (size_t)KR_BLOCKS * (KMAX_LIMIT + 1); }

}  // namespace lrdm
