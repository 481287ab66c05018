// The low-rank least-squares step (Eqs. plowrank, relativeError, quasinewton):
//   S_kl = <f_k, f_l>, c_k = <f_k, R>, ||R||^2   (FP64 partial sums, fixed order)
//   S = Q diag(lambda) Q^T by parallel cyclic Jacobi rotations (FP64, one block)
//   a = Q diag(lambda^+) Q^T c  (lambda < rcond lambda_max dropped -> SINGULAR flag)
//   Delta = sum_k a_k v_k, rho <- rho - alpha Delta, s_rel = ||F a - R|| / ||R||
#include "lrdm_internal.h"

#include <math.h>

#include <atomic>

namespace lrdm {
namespace {

__device__ __forceinline__ double ldio(const void* p, int io, long long i) {
  return io == LRDM_DTYPE_F64 ? static_cast<const double*>(p)[i]
                              : (double)static_cast<const float*>(p)[i];
}

// values per block: K(K+1)/2 Gram entries (upper, row-major), K RHS, 1 ||R||^2
__global__ void __launch_bounds__(256) k_gram(const void* __restrict__ F,
                                              const void* __restrict__ R, int io, int K,
                                              long long n, double* __restrict__ partial) {
  __shared__ double Fs[KMAX_LIMIT][LS_CHUNK];
  __shared__ double Rs[LS_CHUNK];
  const int npair = K * (K + 1) / 2;
  const int nval = npair + K + 1;
  double acc[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t] = 0.0;
  for (long long base = (long long)blockIdx.x * LS_CHUNK; base < n;
       base += (long long)gridDim.x * LS_CHUNK) {
    for (int e = threadIdx.x; e < (K + 1) * LS_CHUNK; e += blockDim.x) {
      int k = e / LS_CHUNK, c = e % LS_CHUNK;
      long long r = base + c;
      double x = 0.0;
      if (r < n) x = k < K ? ldio(F, io, (long long)k * n + r) : ldio(R, io, r);
      if (k < K) Fs[k][c] = x;
      else Rs[c] = x;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      int idx = threadIdx.x + t * blockDim.x;
      if (idx < nval) {
        const double* x;
        const double* y;
        if (idx < npair) {
          // row-major upper triangle enumeration: idx -> (k, l), k <= l
          int k = 0, rem = idx;
          while (rem >= K - k) { rem -= K - k; ++k; }
          x = Fs[k];
          y = Fs[k + rem];
        } else if (idx < npair + K) {
          x = Fs[idx - npair];
          y = Rs;
        } else {
          x = Rs;
          y = Rs;
        }
        double s = 0.0;
        for (int c = 0; c < LS_CHUNK; ++c) s += x[c] * y[c];
        acc[t] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    int idx = threadIdx.x + t * blockDim.x;
    if (idx < nval) partial[(long long)blockIdx.x * nval + idx] = acc[t];
  }
}

// One block of LS_SOLVE_THREADS threads: reduce partials, Jacobi
// eigendecomposition, a = S^+ c.
constexpr int LS_SOLVE_THREADS = 256;
__global__ void __launch_bounds__(LS_SOLVE_THREADS, 1) k_ls_solve(const double* __restrict__ partial,
                                                         int nblk, int K, double w, double rcond,
                                                         double* __restrict__ coef,
                                                         double* __restrict__ coeff_out,
                                                         double* __restrict__ scal,
                                                         int* __restrict__ status) {
  // dynamic shared memory: A(K, K+1), Q(K, K+1) (FP64)
  extern __shared__ double dyn[];
  const int ldk = K + 1;
  double* Abuf = dyn;
  double* Qbuf = dyn + (size_t)K * ldk;
#define A(i, j) Abuf[(i) * ldk + (j)]
#define Q(i, j) Qbuf[(i) * ldk + (j)]
  __shared__ double c[KMAX_LIMIT];
  __shared__ double lam[KMAX_LIMIT];
  __shared__ double r2s;
  __shared__ int bad;
  const int npair = K * (K + 1) / 2;
  const int nval = npair + K + 1;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  // fixed-order reduction of the per-block partials: eight interleaved sums
  // (block b into sum b % 8, so eight loads are in flight), added pairwise
  for (int idx = t; idx < nval; idx += blockDim.x) {
    double a8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int b = 0;
    for (; b + 8 <= nblk; b += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) a8[u] += partial[(long long)(b + u) * nval + idx];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (b + u < nblk) a8[u] += partial[(long long)(b + u) * nval + idx];
    double s = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
    s *= w;
    if (idx < npair) {
      int k = 0, rem = idx;
      while (rem >= K - k) { rem -= K - k; ++k; }
      A(k, k + rem) = s;
      A(k + rem, k) = s;
    } else if (idx < npair + K) {
      c[idx - npair] = s;
    } else {
      r2s = s;
    }
  }
  __syncthreads();
  if (t < K) {
    for (int j = 0; j < K; ++j) Q(t, j) = (t == j) ? 1.0 : 0.0;
    for (int j = 0; j < K; ++j)
      if (!isfinite(A(t, j))) bad = 1;
    if (!isfinite(c[t])) bad = 1;
  }
  __syncthreads();
  if (bad) {
    if (t == 0) atomicOr(status, STATUS_NONFINITE);
    if (t < K) { coef[t] = 0.0; if (coeff_out) coeff_out[t] = 0.0; }
    if (t == 0) { scal[0] = r2s; }
    return;
  }
  // Parallel cyclic Jacobi sweeps (round-robin ordering): a sweep is n - 1
  // rounds (n = K rounded up to even; index K is a dummy when K is odd); a
  // round rotates the n / 2 disjoint pairs (p, q) at once, A <- J^T A J and
  // Q <- Q J, so every pair is rotated once per sweep.
  __shared__ double rc[KMAX_LIMIT / 2], rs[KMAX_LIMIT / 2], rt[KMAX_LIMIT / 2];
  __shared__ double rpq[KMAX_LIMIT / 2], rpp[KMAX_LIMIT / 2], rqq[KMAX_LIMIT / 2];
  __shared__ int rp[KMAX_LIMIT / 2], rq[KMAX_LIMIT / 2];
  __shared__ double red_o[LS_SOLVE_THREADS / 32], red_d[LS_SOLVE_THREADS / 32];
  const int n_rr = K + (K & 1);
  const int nrot = n_rr / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    // off-diagonal and diagonal Frobenius sums, fixed reduction order
    double o = 0.0, d = 0.0;
    if (t < K)
      for (int j = 0; j < K; ++j) {
        const double x = A(t, j);
        if (j == t) d += x * x;
        else o += x * x;
      }
    for (int s = 16; s > 0; s >>= 1) {
      o += __shfl_xor_sync(0xffffffffu, o, s);
      d += __shfl_xor_sync(0xffffffffu, d, s);
    }
    if ((t & 31) == 0) { red_o[t >> 5] = o; red_d[t >> 5] = d; }
    __syncthreads();
    o = 0.0;
    d = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) { o += red_o[wi]; d += red_d[wi]; }
    if (!(o > 1e-30 * d) || o == 0.0) break;
    for (int r = 0; r < n_rr - 1; ++r) {
      // the rotation of pair m (thread m)
      if (t < nrot) {
        int p, q;
        if (t == 0) { p = r; q = n_rr - 1; }
        else { p = (r + t) % (n_rr - 1); q = (r - t + n_rr - 1) % (n_rr - 1); }
        if (p > q) { const int x = p; p = q; q = x; }
        double cs = 1.0, sn = 0.0, tt = 0.0, apq = 0.0, app = 0.0, aqq = 0.0;
        if (q < K) {
          apq = A(p, q);
          app = A(p, p);
          aqq = A(q, q);
          if (apq != 0.0 && fabs(apq) >= 1e-300) {
            const double tau = (aqq - app) / (2.0 * apq);
            tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            cs = 1.0 / sqrt(1.0 + tt * tt);
            sn = tt * cs;
          }
        }
        rp[t] = p; rq[t] = q; rc[t] = cs; rs[t] = sn; rt[t] = tt;
        rpq[t] = apq; rpp[t] = app; rqq[t] = aqq;
      }
      __syncthreads();
      // columns: B = A J, Q <- Q J, one (row, pair) task per thread (each
      // task owns the entries (i, p) and (i, q): no two tasks share one)
      for (int task = t; task < K * nrot; task += blockDim.x) {
        const int i = task % K, m = task / K;
        const int p = rp[m], q = rq[m];
        if (q >= K || rt[m] == 0.0) continue;
        const double c = rc[m], s = rs[m];
        const double ap = A(i, p), aq = A(i, q);
        A(i, p) = c * ap - s * aq;
        A(i, q) = s * ap + c * aq;
        const double qp = Q(i, p), qq = Q(i, q);
        Q(i, p) = c * qp - s * qq;
        Q(i, q) = s * qp + c * qq;
      }
      __syncthreads();
      // rows: A <- J^T B, one (column, pair) task per thread
      for (int task = t; task < K * nrot; task += blockDim.x) {
        const int j = task % K, m = task / K;
        const int p = rp[m], q = rq[m];
        if (q >= K || rt[m] == 0.0) continue;
        const double c = rc[m], s = rs[m];
        const double bp = A(p, j), bq = A(q, j);
        A(p, j) = c * bp - s * bq;
        A(q, j) = s * bp + c * bq;
      }
      __syncthreads();
      // exact symmetry (the lower triangle mirrors the upper) and the closed
      // form of each rotated 2 x 2 block
      if (t < K)
        for (int j = t + 1; j < K; ++j) A(j, t) = A(t, j);
      __syncthreads();
      if (t < nrot && rq[t] < K && rt[t] != 0.0) {
        const int p = rp[t], q = rq[t];
        A(p, p) = rpp[t] - rt[t] * rpq[t];
        A(q, q) = rqq[t] + rt[t] * rpq[t];
        A(p, q) = 0.0;
        A(q, p) = 0.0;
      }
      __syncthreads();
    }
  }
  if (t < K) lam[t] = A(t, t);
  __syncthreads();
  __shared__ double lmax;
  __shared__ int dropped;
  if (t == 0) {
    double m = 0.0;
    for (int i = 0; i < K; ++i) m = fmax(m, lam[i]);
    lmax = m;
    dropped = 0;
  }
  __syncthreads();
  // y = diag(lambda^+) Q^T c
  __shared__ double y[KMAX_LIMIT];
  if (t < K) {
    double s = 0.0;
    for (int i = 0; i < K; ++i) s += Q(i, t) * c[i];
    if (lmax > 0.0 && lam[t] > rcond * lmax) {
      y[t] = s / lam[t];
    } else {
      y[t] = 0.0;
      atomicOr(&dropped, 1);
    }
  }
  __syncthreads();
  if (t < K) {
    double s = 0.0;
    for (int i = 0; i < K; ++i) s += Q(t, i) * y[i];
    coef[t] = s;
    if (coeff_out) coeff_out[t] = s;
  }
  if (t == 0) {
    scal[0] = r2s;
    if (dropped) atomicOr(status, STATUS_SINGULAR);
  }
#undef A
#undef Q
}

// Delta = sum_k a_k v_k; rho <- rho - alpha Delta (alpha != 0) or Delta;
// partial sums of (sum_k a_k f_k - R)^2.
__global__ void __launch_bounds__(256) k_update(const void* __restrict__ v,
                                                const void* __restrict__ f,
                                                const void* __restrict__ R, int io, int K,
                                                long long n, double alpha,
                                                const double* __restrict__ coef,
                                                void* __restrict__ rho,
                                                double* __restrict__ upd_partial) {
  __shared__ double a[KMAX_LIMIT];
  if (threadIdx.x < K) a[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  double acc = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    double d = 0.0, fa = 0.0;
    for (int k = 0; k < K; ++k) {
      d += a[k] * ldio(v, io, (long long)k * n + r);
      fa += a[k] * ldio(f, io, (long long)k * n + r);
    }
    double res = fa - ldio(R, io, r);
    acc += res * res;
    if (rho) {
      double out = alpha != 0.0 ? ldio(rho, io, r) - alpha * d : d;
      if (io == LRDM_DTYPE_F64) static_cast<double*>(rho)[r] = out;
      else static_cast<float*>(rho)[r] = (float)out;
    }
  }
  __shared__ double sw[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sw[i];
    upd_partial[blockIdx.x] = s;
  }
}

__global__ void k_srel(const double* __restrict__ upd_partial, int nblk, double w,
                       const double* __restrict__ scal, double* __restrict__ s_rel_out) {
  __shared__ double sw[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += upd_partial[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += sw[i];
    double r2 = scal[0];
    double val = r2 > 0.0 ? sqrt(w * tot / r2) : 0.0;
    if (s_rel_out) s_rel_out[0] = val;
    // scal layout: [0] = <R, R>, [1] = s_rel
    const_cast<double*>(scal)[1] = val;
  }
}

}  // namespace

cudaError_t launch_ls(const void* R, const void* v, const void* f, int io_dtype, int K,
                      long long n, double w, double alpha, double rcond, void* rho_inout,
                      double* coef, double* coeff_out, double* s_rel_out, double* partial,
                      double* scal, double* upd_partial, int* status, cudaStream_t st,
                      const AllReduce* ar, int* ar_failed) {
  k_gram<<<LS_BLOCKS, 256, 0, st>>>(f, R, io_dtype, K, n, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nval = K * (K + 1) / 2 + K + 1;
  // grid-row sharding: each rank's per-block sums, summed over the ranks
  // block by block, so that every rank reduces the same values in the same order
  if (ar && ar->fn && ar->fn(ar->user, partial, (long long)LS_BLOCKS * nval, LRDM_DTYPE_F64, st) != 0) {
    if (ar_failed) *ar_failed = 1;
    return cudaSuccess;
  }
  const size_t smem = 2 * (size_t)K * (K + 1) * sizeof(double);
  // the shared-memory limit is a per-device function attribute: one bit per
  // device ordinal records that it was raised (a racing first call from
  // another host thread sets the same value again)
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(k_ls_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * KMAX_LIMIT * (KMAX_LIMIT + 1) * (int)sizeof(double));
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit, std::memory_order_acq_rel);
  }
  k_ls_solve<<<1, LS_SOLVE_THREADS, smem, st>>>(partial, LS_BLOCKS, K, w, rcond, coef, coeff_out, scal,
                                          status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_update<<<UPD_BLOCKS, 256, 0, st>>>(v, f, R, io_dtype, K, n, alpha, coef, rho_inout,
                                       upd_partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ar && ar->fn && ar->fn(ar->user, upd_partial, (long long)UPD_BLOCKS, LRDM_DTYPE_F64, st) != 0) {
    if (ar_failed) *ar_failed = 1;
    return cudaSuccess;
  }
  k_srel<<<1, 256, 0, st>>>(upd_partial, UPD_BLOCKS, w, scal, s_rel_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free form of the least-squares step (lrdm_apply_static).
//
// Its scratch -- the per-block partial sums, the coefficients, <R, R> and
// s_rel, the per-block residual sums and the status word -- lives in one
// file-scope device array instead of a context's workspaces, so a call needs
// no lrdm_create and allocates nothing.  The array is sized for at most
// STATIC_K_MAX directions (about 370 KB) and is held by every GPU that loads
// this library until the process exits.  All calls share it: the partial sums
// are fully rewritten by every call and the status word is cleared at its
// start, but two calls that overlap on the GPU (different streams, or several
// host threads) race on it.
// ---------------------------------------------------------------------------

namespace {

constexpr int STATIC_K_MAX = 16;
constexpr int STATIC_NVAL = STATIC_K_MAX * (STATIC_K_MAX + 1) / 2 + STATIC_K_MAX + 1;
constexpr int SC_PARTIAL = 0;                                   // [LS_BLOCKS][STATIC_NVAL]
constexpr int SC_COEF = SC_PARTIAL + LS_BLOCKS * STATIC_NVAL;   // [STATIC_K_MAX]
constexpr int SC_SCAL = SC_COEF + STATIC_K_MAX;                 // [4]
constexpr int SC_UPD = SC_SCAL + 4;                             // [UPD_BLOCKS]
constexpr int SC_STATUS = SC_UPD + UPD_BLOCKS;                  // one double slot for the int status
constexpr int SC_TOTAL = SC_STATUS + 1;

static __device__ __align__(256) double g_ls_scratch[SC_TOTAL];

constexpr int MAX_DEVICES = 64;
// Device address of g_ls_scratch per device ordinal.  Host threads that race
// on a device's first call each look the address up and store the same value;
// the atomics make that race well defined.  The address belongs to the
// device's primary context: after cudaDeviceReset the process must reload
// the library before calling lrdm_apply_static again.
std::atomic<double*> g_scratch_addr[MAX_DEVICES];

// Device address of g_ls_scratch on the current device (looked up once per
// device with that device current; the host-side symbol is not a device
// address).
cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  double* a = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_ls_scratch);
    if (e != cudaSuccess) return e;
    a = static_cast<double*>(p);
    g_scratch_addr[dev].store(a, std::memory_order_release);
  }
  *out = a;
  return cudaSuccess;
}

}  // namespace

int static_k_max() { return STATIC_K_MAX; }

cudaError_t launch_ls_static(const void* R, const void* v, const void* f, int io_dtype, int K,
                             long long n, double w, double alpha, double rcond, void* rho_inout,
                             double* coeff_out, double* s_rel_out, int* status_out,
                             cudaStream_t st) {
  double* sc = nullptr;
  cudaError_t e = static_scratch(&sc);
  if (e != cudaSuccess) return e;
  int* status = reinterpret_cast<int*>(sc + SC_STATUS);
  e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  double* partial = sc + SC_PARTIAL;
  double* coef = sc + SC_COEF;
  double* scal = sc + SC_SCAL;
  double* upd = sc + SC_UPD;
  k_gram<<<LS_BLOCKS, 256, 0, st>>>(f, R, io_dtype, K, n, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = 2 * (size_t)K * (K + 1) * sizeof(double);   // <= 4352 bytes for K <= 16
  k_ls_solve<<<1, LS_SOLVE_THREADS, smem, st>>>(partial, LS_BLOCKS, K, w, rcond, coef, coeff_out, scal,
                                          status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_update<<<UPD_BLOCKS, 256, 0, st>>>(v, f, R, io_dtype, K, n, alpha, coef, rho_inout, upd);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_srel<<<1, 256, 0, st>>>(upd, UPD_BLOCKS, w, scal, s_rel_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (status_out)
    e = cudaMemcpyAsync(status_out, status, sizeof(int), cudaMemcpyDeviceToDevice, st);
  return e;
}

}  // namespace lrdm
