// CUDA-core (FP64 / FP32) forms of the two contractions.  These serve the
// FP64 and FP32 precisions; the tensor-core forms live in k_tc.cu.
//
// GEMM1: X_k = Psi^T diag(a_k) Psi   (H-breve' = Psi~^T H~' Psi~, §II.C),
//        upper-triangular 64x64 tiles, both triangles written.
// GEMM2: drho_k(r) = g sum_j sum_{i<=j} Psi_ri X''_k,ij Psi_rj with X'' the
//        Loewner-scaled matrix with doubled strict upper triangle (the
//        diagonal of Psi X' Psi^T, Eq. densityResponse, using X' = X'^T);
//        Psi X'' is held in registers, never written to memory.
#include "lrdm_internal.h"

namespace lrdm {
namespace {

constexpr int T = SIMT_TILE;  // 64
constexpr int BK = 16;

__device__ __forceinline__ void tri_index(int p, int& I, int& J) {
  int j = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while (j * (j + 1) / 2 > p) --j;
  while ((j + 1) * (j + 2) / 2 <= p) ++j;
  J = j;
  I = p - j * (j + 1) / 2;
}

template <typename Tc>
__global__ void __launch_bounds__(256) k_gemm1(const Tc* __restrict__ psi, int ns, long long Ng,
                                               const Tc* __restrict__ a, long long a_stride,
                                               int nq, Tc* __restrict__ Xpart, long long rows_per,
                                               int nsplit) {
  int I, J;
  tri_index(blockIdx.x, I, J);
  const int q = blockIdx.y, split = blockIdx.z;
  const int i0 = I * T, j0 = J * T;
  const Tc* aq = a + (long long)q * a_stride;
  const long long rb = (long long)split * rows_per;
  const long long re = min(Ng, rb + rows_per);
  // two stages in shared memory; the next stage's global values are loaded
  // into registers while the current one is multiplied (one barrier a stage)
  __shared__ __align__(16) Tc As[2][BK][T];
  __shared__ __align__(16) Tc Bs[2][BK][T];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  static_assert(BK * T == 4 * 256, "four elements of each operand per thread and stage");
  const int cc = threadIdx.x & (T - 1), rr0 = threadIdx.x / T;   // rows rr0 + 4 u of a stage
  Tc acc[4][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int n = 0; n < 4; ++n) acc[m][n] = Tc(0);
  Tc pa[4], pb[4];
  auto fetch = [&](long long r0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long r = r0 + rr0 + 4 * u;
      Tc av = Tc(0), bv = Tc(0);
      if (r < re) {
        const Tc sc = aq[r];
        if (i0 + cc < ns) av = psi[r * ns + i0 + cc] * sc;
        if (j0 + cc < ns) bv = psi[r * ns + j0 + cc];
      }
      pa[u] = av;
      pb[u] = bv;
    }
  };
  auto stash = [&](int b) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      As[b][rr0 + 4 * u][cc] = pa[u];
      Bs[b][rr0 + 4 * u][cc] = pb[u];
    }
  };
  if (rb < re) {
    fetch(rb);
    stash(0);
  }
  __syncthreads();
  int buf = 0;
  for (long long r0 = rb; r0 < re; r0 += BK) {
    const bool more = r0 + BK < re;
    if (more) fetch(r0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Tc ar[4], br[4];
      ld4(&As[buf][kk][4 * ty], ar);         // rows 4 ty .. 4 ty + 3
      ld4(&Bs[buf][kk][4 * tx], br);         // columns 4 tx .. 4 tx + 3
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n) acc[m][n] += ar[m] * br[n];
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  Tc* Xq = Xpart + ((long long)split * nq + q) * (long long)ns * ns;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int i = i0 + 4 * ty + m;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      int j = j0 + 4 * tx + n;
      if (i < ns && j < ns) {
        Xq[(long long)i * ns + j] = acc[m][n];
        if (I != J) Xq[(long long)j * ns + i] = acc[m][n];
      }
    }
  }
}

template <typename Tc>
__global__ void __launch_bounds__(256) k_gemm2(const Tc* __restrict__ psi, int ns, long long Ng,
                                               const Tc* __restrict__ Xpp, double factor,
                                               const void* __restrict__ v, long long v_stride,
                                               void* __restrict__ out, long long out_stride,
                                               int out_io, int out_is_io) {
  const int q = blockIdx.y;
  const long long r0 = (long long)blockIdx.x * T;
  const Tc* Xq = Xpp + (long long)q * ns * ns;
  __shared__ Tc Ps[T][BK + 1];
  __shared__ Tc Xs[BK][T];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  const int ntile = (ns + T - 1) / T;
  for (int Jt = 0; Jt < ntile; ++Jt) {
    const int j0 = Jt * T;
    const int iend = min(ns, j0 + T);
    Tc acc[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n) acc[m][n] = Tc(0);
    for (int i0 = 0; i0 < iend; i0 += BK) {
      for (int e = threadIdx.x; e < T * BK; e += 256) {
        int rr = e / BK, kk = e % BK;
        long long r = r0 + rr;
        int i = i0 + kk;
        Ps[rr][kk] = (r < Ng && i < iend) ? psi[r * ns + i] : Tc(0);
      }
      for (int e = threadIdx.x; e < BK * T; e += 256) {
        int kk = e / T, cc = e % T;
        int i = i0 + kk, j = j0 + cc;
        Xs[kk][cc] = (i < iend && j < ns) ? Xq[(long long)i * ns + j] : Tc(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        Tc ar[4], br[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) ar[m] = Ps[ty + 16 * m][kk];
#pragma unroll
        for (int n = 0; n < 4; ++n) br[n] = Xs[kk][tx + 16 * n];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int n = 0; n < 4; ++n) acc[m][n] += ar[m] * br[n];
      }
      __syncthreads();
    }
    // row-dot epilogue against the Psi(R, J) tile
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      long long r = r0 + ty + 16 * m;
      if (r < Ng) {
        Tc s = Tc(0);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          int j = j0 + tx + 16 * n;
          if (j < ns) s += acc[m][n] * psi[r * ns + j];
        }
        part[m] += (double)s;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    double p = part[m];
    for (int o = 8; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    long long r = r0 + ty + 16 * m;
    if (tx == 0 && r < Ng) {
      double d = factor * p;
      if (out_is_io) {
        double vv = out_io == LRDM_DTYPE_F64
                        ? static_cast<const double*>(v)[q * v_stride + r]
                        : (double)static_cast<const float*>(v)[q * v_stride + r];
        if (out_io == LRDM_DTYPE_F64) static_cast<double*>(out)[q * out_stride + r] = d - vv;
        else static_cast<float*>(out)[q * out_stride + r] = (float)(d - vv);
      } else {
        static_cast<Tc*>(out)[q * out_stride + r] = (Tc)d;
      }
    }
  }
}

}  // namespace

cudaError_t launch_gemm1_simt(int fp64, const void* psi, int ns, long long Ng, const void* a,
                              long long a_stride, int nq, void* Xpart, int nsplit,
                              cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  int nt = (ns + T - 1) / T;
  long long rows_per = (Ng + nsplit - 1) / nsplit;
  rows_per = (rows_per + BK - 1) / BK * BK;
  dim3 grid(nt * (nt + 1) / 2, nq, nsplit);
  if (fp64)
    k_gemm1<double><<<grid, 256, 0, st>>>(static_cast<const double*>(psi), ns, Ng,
                                          static_cast<const double*>(a), a_stride, nq,
                                          static_cast<double*>(Xpart), rows_per, nsplit);
  else
    k_gemm1<float><<<grid, 256, 0, st>>>(static_cast<const float*>(psi), ns, Ng,
                                         static_cast<const float*>(a), a_stride, nq,
                                         static_cast<float*>(Xpart), rows_per, nsplit);
  return cudaGetLastError();
}

cudaError_t launch_gemm2_simt(int fp64, const void* psi, int ns, long long Ng, const void* Xpp,
                              int nq, double factor, const void* v, long long v_stride,
                              void* out, long long out_stride, int out_io_dtype, int out_is_io,
                              cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  dim3 grid((unsigned)((Ng + T - 1) / T), nq);
  if (fp64)
    k_gemm2<double><<<grid, 256, 0, st>>>(static_cast<const double*>(psi), ns, Ng,
                                          static_cast<const double*>(Xpp), factor, v, v_stride,
                                          out, out_stride, out_io_dtype, out_is_io);
  else
    k_gemm2<float><<<grid, 256, 0, st>>>(static_cast<const float*>(psi), ns, Ng,
                                         static_cast<const float*>(Xpp), factor, v, v_stride, out,
                                         out_stride, out_io_dtype, out_is_io);
  return cudaGetLastError();
}

}  // namespace lrdm
