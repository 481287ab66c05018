// CUDA-core (FP64 / FP32) kernels of the Brillouin-zone-sampled response
// (§II.C, closing paragraphs; Eq. tracelessCondition).  Complex quantities
// are held as separate real and imaginary planes: psi = A + i B per k-point
// ([N_g][N_s] each), X = Xr + i Xi ([split][K][N_s][N_s]).
//
//   X_kappa = Psi^H diag(a_k) Psi:  Xr_ij = sum_r a (A_i A_j + B_i B_j),
//                                   Xi_ij = sum_r a (A_i B_j - B_i A_j),
//   upper-triangular 64 x 64 tiles, the lower triangle written as the
//   conjugate (X is Hermitian);
//   mu'_k = sum_kappa w_kappa sum_i L_ii Xr_ii / sum_kappa w_kappa sum_i L_ii;
//   X'' = c_ij L_ij conj(X_ij - delta_ij mu'), c = 2 / 1 / 0 above / on /
//   below the diagonal, so that Re sum_ij conj(psi_i) X''_ij psi_j equals
//   sum_ij psi_i Gamma_ij conj(psi_j), the diagonal of Psi Gamma Psi^H with
//   Gamma = L o (X - mu' I) Hermitian (the pair (i, j), (j, i) adds up to
//   twice the real part of one term);
//   drho_k(r) += g w_kappa Re sum_j T_j(r) psi_j(r), T_j = sum_i conj(psi_i) X''_ij
//   (T never leaves registers), accumulated over k-points in FP64.
//
// Tensor-core modes reuse the real contractions on the stacked operand
// C = [A B] (N_g x 2 N_s): P = C^T diag(a) C holds Re X = P11 + P22 and
// Im X = P12 - P21, and the density diag(Psi Gamma Psi^H) equals
// diag(C M C^T) with the symmetric M = [[Re G, Im G], [-Im G, Re G]]
// (G = Gamma), whose c-weighted upper triangle k_kp_scale_tc writes in the
// layout of the real GEMM2's X'' operand.
#include <cuda_bf16.h>

#include "lrdm_internal.h"

namespace lrdm {
namespace {

constexpr int T = 64;
constexpr int BK = 16;


// upper-triangular tile p -> (I, J), I <= J, column-major over J
__device__ __forceinline__ void kp_tri(int p, int& I, int& J) {
  int j = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while (j * (j + 1) / 2 > p) --j;
  while ((j + 1) * (j + 2) / 2 <= p) ++j;
  J = j;
  I = p - j * (j + 1) / 2;
}

// grid (tiles, K, row ranges), 256 threads, 4 x 4 outputs per thread
template <typename Tc>
__global__ void __launch_bounds__(256) k_kp_gemm1(const Tc* __restrict__ pr, const Tc* __restrict__ pi,
                                                  int ns, long long Ng, const Tc* __restrict__ a,
                                                  long long a_stride, int K, Tc* __restrict__ Xr,
                                                  Tc* __restrict__ Xi, long long rows_per) {
  int I, J;
  kp_tri(blockIdx.x, I, J);
  const int q = blockIdx.y, split = blockIdx.z;
  const int i0 = I * T, j0 = J * T;
  const Tc* aq = a + (long long)q * a_stride;
  const long long rb = (long long)split * rows_per;
  const long long re = min(Ng, rb + rows_per);
  __shared__ __align__(16) Tc Ar[BK][T];
  __shared__ __align__(16) Tc Ai[BK][T];
  __shared__ __align__(16) Tc Br[BK][T];
  __shared__ __align__(16) Tc Bi[BK][T];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  Tc sr[4][4], si[4][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int n = 0; n < 4; ++n) sr[m][n] = si[m][n] = Tc(0);
  for (long long r0 = rb; r0 < re; r0 += BK) {
    for (int e = threadIdx.x; e < BK * T; e += 256) {
      const int rr = e / T, cc = e % T;
      const long long r = r0 + rr;
      Tc ar = 0, ai = 0, br = 0, bi = 0;
      if (r < re) {
        const Tc sc = aq[r];
        if (i0 + cc < ns) {
          ar = pr[r * ns + i0 + cc] * sc;
          ai = pi[r * ns + i0 + cc] * sc;
        }
        if (j0 + cc < ns) {
          br = pr[r * ns + j0 + cc];
          bi = pi[r * ns + j0 + cc];
        }
      }
      Ar[rr][cc] = ar;
      Ai[rr][cc] = ai;
      Br[rr][cc] = br;
      Bi[rr][cc] = bi;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Tc xr[4], xi[4], yr[4], yi[4];
      ld4(&Ar[kk][4 * ty], xr);              // rows 4 ty .. 4 ty + 3
      ld4(&Ai[kk][4 * ty], xi);
      ld4(&Br[kk][4 * tx], yr);              // columns 4 tx .. 4 tx + 3
      ld4(&Bi[kk][4 * tx], yi);
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          // conj(x) y = (xr yr + xi yi) + i (xr yi - xi yr)
          sr[m][n] += xr[m] * yr[n] + xi[m] * yi[n];
          si[m][n] += xr[m] * yi[n] - xi[m] * yr[n];
        }
    }
    __syncthreads();
  }
  const long long mat = (long long)ns * ns;
  Tc* Xrq = Xr + ((long long)split * K + q) * mat;
  Tc* Xiq = Xi + ((long long)split * K + q) * mat;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int i = i0 + 4 * ty + m;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int j = j0 + 4 * tx + n;
      if (i < ns && j < ns) {
        Xrq[(long long)i * ns + j] = sr[m][n];
        Xiq[(long long)i * ns + j] = si[m][n];
        if (I != J) {
          Xrq[(long long)j * ns + i] = sr[m][n];
          Xiq[(long long)j * ns + i] = -si[m][n];
        }
      }
    }
  }
}

// mu'_k over all k-points (one block of 256 threads per direction; row-range
// partials summed in order).
__global__ void __launch_bounds__(256) k_kp_dmu(KpDmuArgs A, double* __restrict__ dmu,
                                                double* __restrict__ dmu_out) {
  const int k = blockIdx.x;
  double num = 0.0, den = 0.0;
  const long long mat = (long long)A.ld * A.ld;
  for (int kp = 0; kp < A.nk; ++kp) {
    const double wk = A.kw[kp];
    for (int i = threadIdx.x; i < A.ns; i += blockDim.x) {
      double x = 0.0;
      for (int p = 0; p < A.nsplit; ++p) {
        const long long o = ((long long)p * A.K + k) * mat + (long long)i * A.ld + i;
        x += A.fp64 ? static_cast<const double*>(A.Xr[kp])[o] : (double)static_cast<const float*>(A.Xr[kp])[o];
        if (A.stacked) {
          const long long o2 = o + (long long)A.ns * A.ld + A.ns;
          x += A.fp64 ? static_cast<const double*>(A.Xr[kp])[o2]
                      : (double)static_cast<const float*>(A.Xr[kp])[o2];
        }
      }
      const double l = A.L[kp][(long long)i * A.ns + i];
      num += wk * l * x;
      den += wk * l;
    }
  }
  __shared__ double sn[8], sd[8];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sn[threadIdx.x >> 5] = num;
    sd[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += sn[w];
      b += sd[w];
    }
    const double v = b != 0.0 ? a / b : 0.0;
    dmu[k] = v;
    if (dmu_out) dmu_out[k] = v;
  }
}

// X'' = c_ij L_ij conj(X_ij - delta_ij mu'_k), splits summed; upper part only.
template <typename Tc>
__global__ void k_kp_scale(const Tc* __restrict__ Xr, const Tc* __restrict__ Xi, int nsplit, int K,
                           int ns, const double* __restrict__ L, const double* __restrict__ dmu,
                           Tc* __restrict__ Yr, Tc* __restrict__ Yi) {
  const long long mat = (long long)ns * ns;
  const long long tot = (long long)K * mat;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / mat);
    const long long rem = e - (long long)k * mat;
    const int i = (int)(rem / ns), j = (int)(rem - (long long)i * ns);
    double yr = 0.0, yi = 0.0;
    if (i <= j) {
      double xr = 0.0, xi = 0.0;
      for (int p = 0; p < nsplit; ++p) {
        xr += (double)Xr[(long long)p * tot + e];
        xi += (double)Xi[(long long)p * tot + e];
      }
      const double l = L[(long long)i * ns + j];
      if (i == j) {
        yr = l * (xr - dmu[k]);
      } else {
        yr = 2.0 * l * xr;
        yi = -2.0 * l * xi;
      }
    }
    Yr[e] = (Tc)yr;
    Yi[e] = (Tc)yi;
  }
}

// drho[k][r] += factor * Re sum_j T_j(r) psi_j(r), T_j = sum_{i<=j} conj(psi_i(r)) X''_ij.
// grid (row blocks of 64, K), 256 threads.
template <typename Tc>
__global__ void __launch_bounds__(256) k_kp_gemm2(const Tc* __restrict__ pr, const Tc* __restrict__ pi,
                                                  int ns, long long Ng, const Tc* __restrict__ Yr,
                                                  const Tc* __restrict__ Yi, double factor,
                                                  double* __restrict__ drho) {
  const int q = blockIdx.y;
  const long long r0 = (long long)blockIdx.x * T;
  const long long mat = (long long)ns * ns;
  const Tc* Yrq = Yr + (long long)q * mat;
  const Tc* Yiq = Yi + (long long)q * mat;
  __shared__ Tc Pr[T][BK + 1], Pi[T][BK + 1];
  __shared__ Tc Sr[BK][T], Si[BK][T];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  const int ntile = (ns + T - 1) / T;
  for (int Jt = 0; Jt < ntile; ++Jt) {
    const int j0 = Jt * T;
    const int iend = min(ns, j0 + T);
    Tc tr[4][4], ti[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int n = 0; n < 4; ++n) tr[m][n] = ti[m][n] = Tc(0);
    for (int i0 = 0; i0 < iend; i0 += BK) {
      for (int e = threadIdx.x; e < T * BK; e += 256) {
        const int rr = e / BK, kk = e % BK;
        const long long r = r0 + rr;
        const int i = i0 + kk;
        const bool in = r < Ng && i < iend;
        Pr[rr][kk] = in ? pr[r * ns + i] : Tc(0);
        Pi[rr][kk] = in ? pi[r * ns + i] : Tc(0);
      }
      for (int e = threadIdx.x; e < BK * T; e += 256) {
        const int kk = e / T, cc = e % T;
        const int i = i0 + kk, j = j0 + cc;
        const bool in = i < iend && j < ns;
        Sr[kk][cc] = in ? Yrq[(long long)i * ns + j] : Tc(0);
        Si[kk][cc] = in ? Yiq[(long long)i * ns + j] : Tc(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        Tc ar[4], ai[4], br[4], bi[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          ar[m] = Pr[ty + 16 * m][kk];
          ai[m] = Pi[ty + 16 * m][kk];
        }
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          br[n] = Sr[kk][tx + 16 * n];
          bi[n] = Si[kk][tx + 16 * n];
        }
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int n = 0; n < 4; ++n) {
            // conj(psi_i) X''_ij = (ar - i ai)(br + i bi)
            tr[m][n] += ar[m] * br[n] + ai[m] * bi[n];
            ti[m][n] += ar[m] * bi[n] - ai[m] * br[n];
          }
      }
      __syncthreads();
    }
    // row-dot epilogue: Re T_j psi_j = tr A_j - ti B_j
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const long long r = r0 + ty + 16 * m;
      if (r < Ng) {
        Tc sacc = Tc(0);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          const int j = j0 + tx + 16 * n;
          if (j < ns) sacc += tr[m][n] * pr[r * ns + j] - ti[m][n] * pi[r * ns + j];
        }
        part[m] += (double)sacc;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    double p = part[m];
    for (int o = 8; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    const long long r = r0 + ty + 16 * m;
    if (tx == 0 && r < Ng) drho[(long long)q * Ng + r] += factor * p;
  }
}

// f = drho - v in the io dtype
__global__ void k_kp_finish(const double* __restrict__ drho, const void* __restrict__ v, int io,
                            long long n, void* __restrict__ f) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    if (io == LRDM_DTYPE_F64)
      static_cast<double*>(f)[e] = drho[e] - static_cast<const double*>(v)[e];
    else
      static_cast<float*>(f)[e] = (float)(drho[e] - (double)static_cast<const float*>(v)[e]);
  }
}

// rho = (first ? floor : rho) + g w sum_i f_i (A_i^2 + B_i^2), one warp per grid
// point; A, B rows of leading dimension ld
template <typename Tc>
__global__ void k_kp_density(const Tc* __restrict__ pr, const Tc* __restrict__ pi, int ns, int ld,
                             long long Ng, const double* __restrict__ occ, double gw, int first,
                             double floor, double* __restrict__ rho) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < Ng; r += nwarps) {
    double acc = 0.0;
    for (int i = lane; i < ns; i += 32) {
      const double a = pr[r * ld + i], b = pi[r * ld + i];
      acc += occ[i] * (a * a + b * b);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rho[r] = (first ? floor : rho[r]) + gw * acc;
  }
}

// one plane of the caller's Psi (io dtype, leading dimension ld) into the
// compute type, [N_g][N_s]
template <typename Tc>
__global__ void k_kp_copy(const void* __restrict__ src, int io, int ld, long long Ng, int ns,
                          Tc* __restrict__ dst, int ldd, int col0) {
  const long long tot = Ng * ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ns;
    const int i = (int)(e - r * ns);
    const double x = io == LRDM_DTYPE_F64 ? static_cast<const double*>(src)[r * ld + i]
                                          : (double)static_cast<const float*>(src)[r * ld + i];
    dst[r * ldd + col0 + i] = (Tc)x;
  }
}

// M'' at [k][j][i] (i fastest) for i <= j < 2 ns: c_ij M_ij with c = 2 off the
// diagonal; zero elsewhere (padding included).  One thread per four columns.
// P (both triangles written by GEMM1) and L are symmetric, so every read
// takes the entry whose column follows i: consecutive threads read
// consecutive addresses.
__global__ void k_kp_scale_tc(const float* __restrict__ P, int nsplit, int K, int ns, int ld,
                              const double* __restrict__ L, const double* __restrict__ dmu, int layout,
                              void* __restrict__ out, __nv_bfloat16* __restrict__ out_lo) {
  const int c0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y;
  const int k = blockIdx.z;
  if (c0 >= ld) return;
  const long long mat = (long long)ld * ld;
  const long long tot = (long long)K * mat;
  const float* Pk = P + (long long)k * mat;
  auto Pat = [&](int r, int c) {               // P[r][c] summed over the row ranges
    double x = 0.0;
    for (int p = 0; p < nsplit; ++p) x += (double)Pk[(long long)p * tot + (long long)r * ld + c];
    return x;
  };
  const int n2 = 2 * ns;
  float v[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = c0 + e;
    double m = 0.0;
    if (i <= j && j < n2) {
      const int a = i < ns ? i : i - ns, b = j < ns ? j : j - ns;
      const double l = L[(long long)b * ns + a];
      if ((i < ns) == (j < ns)) {              // diagonal blocks: Re Gamma_ab = L_ab (P11 + P22 - mu')
        const double xr = Pat(b, a) + Pat(ns + b, ns + a);
        m = l * (xr - (a == b ? dmu[k] : 0.0));
      } else {                                 // i in block 0, j in block 1: Im Gamma_ab = L_ab (P12 - P21)
        const double xi = Pat(ns + b, a) - Pat(b, ns + a);
        m = l * xi;
      }
      if (i < j) m *= 2.0;
    }
    v[e] = (float)m;
  }
  const long long o = ((long long)k * ld + j) * ld + c0;
  if (layout == 1) {
    float4 t;
    t.x = tf32_rna(v[0]);
    t.y = tf32_rna(v[1]);
    t.z = tf32_rna(v[2]);
    t.w = tf32_rna(v[3]);
    *reinterpret_cast<float4*>(static_cast<float*>(out) + o) = t;
  } else {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 h23 = __floats2bfloat162_rn(v[2], v[3]);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(v[0] - f01.x, v[1] - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(v[2] - f23.x, v[3] - f23.y);
    uint2 hw, lw;
    hw.x = *reinterpret_cast<const uint32_t*>(&h01);
    hw.y = *reinterpret_cast<const uint32_t*>(&h23);
    lw.x = *reinterpret_cast<const uint32_t*>(&l01);
    lw.y = *reinterpret_cast<const uint32_t*>(&l23);
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(out) + o) = hw;
    *reinterpret_cast<uint2*>(out_lo + o) = lw;
  }
}

// f = sum_kappa part_kappa - v, FP64 sum of the FP32 contributions
__global__ void k_kp_sum(KpSumArgs A, const void* __restrict__ v, int io, long long n,
                         void* __restrict__ f) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int q = 0; q < A.nk; ++q) d += (double)A.part[q][e];
    if (io == LRDM_DTYPE_F64)
      static_cast<double*>(f)[e] = d - static_cast<const double*>(v)[e];
    else
      static_cast<float*>(f)[e] = (float)(d - (double)static_cast<const float*>(v)[e]);
  }
}

// out[k][r] (compute type, row stride ld) = sum_kappa part_kappa[k][r]
// (A given: FP32 contributions) or drho[k][r] (FP64 accumulator); zero for
// N_g <= r < ld.
__global__ void k_kp_collect(KpSumArgs A, int use_parts, const double* __restrict__ drho, long long Ng,
                             long long ld, long long tot, void* __restrict__ out, int fp64) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / ld, r = e - k * ld;
    double d = 0.0;
    if (r < Ng) {
      const long long o = k * Ng + r;
      if (use_parts)
        for (int q = 0; q < A.nk; ++q) d += (double)A.part[q][o];
      else
        d = drho[o];
    }
    if (fp64) static_cast<double*>(out)[e] = d;
    else static_cast<float*>(out)[e] = (float)d;
  }
}

inline unsigned kp_grid(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_kp_gemm1(int fp64, const void* pr, const void* pi, int ns, long long Ng,
                            const void* a, long long a_stride, int K, void* Xr, void* Xi, int nsplit,
                            cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  const int nt = (ns + T - 1) / T;
  long long rows_per = (Ng + nsplit - 1) / nsplit;
  rows_per = (rows_per + BK - 1) / BK * BK;
  dim3 grid(nt * (nt + 1) / 2, K, nsplit);
  if (fp64)
    k_kp_gemm1<double><<<grid, 256, 0, st>>>(static_cast<const double*>(pr), static_cast<const double*>(pi),
                                             ns, Ng, static_cast<const double*>(a), a_stride, K,
                                             static_cast<double*>(Xr), static_cast<double*>(Xi), rows_per);
  else
    k_kp_gemm1<float><<<grid, 256, 0, st>>>(static_cast<const float*>(pr), static_cast<const float*>(pi),
                                            ns, Ng, static_cast<const float*>(a), a_stride, K,
                                            static_cast<float*>(Xr), static_cast<float*>(Xi), rows_per);
  return cudaGetLastError();
}

cudaError_t launch_kp_dmu(const KpDmuArgs& A, double* dmu, double* dmu_out, cudaStream_t st) {
  if (A.K == 0) return cudaSuccess;
  k_kp_dmu<<<A.K, 256, 0, st>>>(A, dmu, dmu_out);
  return cudaGetLastError();
}

cudaError_t launch_kp_scale(int fp64, const void* Xr, const void* Xi, int nsplit, int K, int ns,
                            const double* L, const double* dmu, void* Yr, void* Yi, cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  const unsigned g = kp_grid((long long)K * ns * ns, 256);
  if (fp64)
    k_kp_scale<double><<<g, 256, 0, st>>>(static_cast<const double*>(Xr), static_cast<const double*>(Xi),
                                          nsplit, K, ns, L, dmu, static_cast<double*>(Yr),
                                          static_cast<double*>(Yi));
  else
    k_kp_scale<float><<<g, 256, 0, st>>>(static_cast<const float*>(Xr), static_cast<const float*>(Xi),
                                         nsplit, K, ns, L, dmu, static_cast<float*>(Yr),
                                         static_cast<float*>(Yi));
  return cudaGetLastError();
}

cudaError_t launch_kp_gemm2(int fp64, const void* pr, const void* pi, int ns, long long Ng,
                            const void* Yr, const void* Yi, int K, double factor, double* drho,
                            cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  dim3 grid((unsigned)((Ng + T - 1) / T), K);
  if (fp64)
    k_kp_gemm2<double><<<grid, 256, 0, st>>>(static_cast<const double*>(pr), static_cast<const double*>(pi),
                                             ns, Ng, static_cast<const double*>(Yr),
                                             static_cast<const double*>(Yi), factor, drho);
  else
    k_kp_gemm2<float><<<grid, 256, 0, st>>>(static_cast<const float*>(pr), static_cast<const float*>(pi),
                                            ns, Ng, static_cast<const float*>(Yr),
                                            static_cast<const float*>(Yi), factor, drho);
  return cudaGetLastError();
}

cudaError_t launch_kp_finish(const double* drho, const void* v, int io, long long n, void* f,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_kp_finish<<<kp_grid(n, 256), 256, 0, st>>>(drho, v, io, n, f);
  return cudaGetLastError();
}

cudaError_t launch_kp_density(int fp64, const void* pr, const void* pi, int ns, int ld, long long Ng,
                              const double* occ, double gw, int first, double floor, double* rho,
                              cudaStream_t st) {
  const unsigned g = kp_grid(Ng * 32, 256);
  if (fp64)
    k_kp_density<double><<<g, 256, 0, st>>>(static_cast<const double*>(pr), static_cast<const double*>(pi),
                                            ns, ld, Ng, occ, gw, first, floor, rho);
  else
    k_kp_density<float><<<g, 256, 0, st>>>(static_cast<const float*>(pr), static_cast<const float*>(pi),
                                           ns, ld, Ng, occ, gw, first, floor, rho);
  return cudaGetLastError();
}

cudaError_t launch_kp_copy(int fp64, const void* src, int io, int ld, long long Ng, int ns, void* dst,
                           int ldd, int col0, cudaStream_t st) {
  const unsigned g = kp_grid(Ng * ns, 256);
  if (fp64) k_kp_copy<double><<<g, 256, 0, st>>>(src, io, ld, Ng, ns, static_cast<double*>(dst), ldd, col0);
  else k_kp_copy<float><<<g, 256, 0, st>>>(src, io, ld, Ng, ns, static_cast<float*>(dst), ldd, col0);
  return cudaGetLastError();
}

cudaError_t launch_kp_scale_tc(const float* P, int nsplit, int K, int ns, int ld, const double* L,
                               const double* dmu, int layout, void* out, void* out_lo, cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  dim3 grid((unsigned)((ld / 4 + 127) / 128), (unsigned)ld, (unsigned)K);
  k_kp_scale_tc<<<grid, 128, 0, st>>>(P, nsplit, K, ns, ld, L, dmu, layout, out,
                                      static_cast<__nv_bfloat16*>(out_lo));
  return cudaGetLastError();
}

cudaError_t launch_kp_collect(const KpSumArgs* A, const double* drho, int K, long long Ng, long long ld,
                              void* out, int fp64, cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  const long long tot = (long long)K * ld;
  KpSumArgs a{};
  if (A) a = *A;
  k_kp_collect<<<kp_grid(tot, 256), 256, 0, st>>>(a, A ? 1 : 0, drho, Ng, ld, tot, out, fp64);
  return cudaGetLastError();
}

cudaError_t launch_kp_sum(const KpSumArgs& A, const void* v, int io, long long n, void* f,
                          cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_kp_sum<<<kp_grid(n, 256), 256, 0, st>>>(A, v, io, n, f);
  return cudaGetLastError();
}

}  // namespace lrdm
