// Set-up kernels run once by lrdm_create: operand copies of Psi, the density
// and the LDA exchange kernel, and the Loewner matrix of the Fermi function.
#include "lrdm_internal.h"

#include <math.h>

namespace lrdm {
namespace {

// round-to-nearest into the TF32 format (the tensor cores read 10 mantissa bits)
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ double load_io(const void* p, int io_dtype, long long i) {
  return io_dtype == LRDM_DTYPE_F64 ? static_cast<const double*>(p)[i]
                                    : (double)static_cast<const float*>(p)[i];
}

// Row-major copies: psi64 / psi32 [Ng][ns]
__global__ void k_copy_rowmajor(const void* __restrict__ src, int io_dtype, int ld, long long Ng,
                                int ns, double* __restrict__ d64, float* __restrict__ d32) {
  long long total = Ng * ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e / ns;
    int i = (int)(e - r * ns);
    double x = load_io(src, io_dtype, r * ld + i);
    if (d64) d64[e] = x;
    if (d32) d32[e] = (float)x;
  }
}

// Padded row-major [Ng_pad][ns_pad] and transposed (tile-major, see below)
// copies for the tensor-core paths; split into bf16 hi/lo (x = hi + lo,
// lo = bf16(x - hi)) or rounded to TF32.  Tiled transpose through shared memory.
__global__ void k_copy_tc(const void* __restrict__ src, int io_dtype, int ld, long long Ng, int ns,
                          long long Ng_pad, int ns_pad, float* __restrict__ R32,
                          float* __restrict__ T32, __nv_bfloat16* __restrict__ Rhi,
                          __nv_bfloat16* __restrict__ Rlo, __nv_bfloat16* __restrict__ Thi,
                          __nv_bfloat16* __restrict__ Tlo, float* __restrict__ Tf) {
  __shared__ float tile[32][33];
  long long r0 = (long long)blockIdx.x * 32;
  int i0 = blockIdx.y * 32;
  int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    long long r = r0 + yy;
    int i = i0 + tx;
    float x = 0.f;
    if (r < Ng && i < ns) x = (float)load_io(src, io_dtype, r * ld + i);
    tile[yy][tx] = x;
    if (r < Ng_pad && i < ns_pad) {
      long long o = r * ns_pad + i;
      if (R32) R32[o] = to_tf32(x);
      if (Rhi) {
        __nv_bfloat16 hi = __float2bfloat16_rn(x);
        Rhi[o] = hi;
        Rlo[o] = __float2bfloat16_rn(x - __bfloat162float(hi));
      }
    }
  }
  __syncthreads();
  // transposed copies are tile-major: [i / 128][r / RB][i % 128][r % RB] with
  // RB = 64 bytes of the operand type (16 TF32, 32 bf16; the exact FP32 copy
  // of the split mode shares the bf16 RB = 32), so that one (128 states x RB
  // rows) tensor-core operand tile is a contiguous block
  for (int yy = ty; yy < 32; yy += 8) {
    int i = i0 + yy;
    long long r = r0 + tx;
    if (i < ns_pad && r < Ng_pad) {
      float x = tile[tx][yy];
      const int RB = T32 ? 16 : 32;
      long long o = (((long long)(i >> 7) * (Ng_pad / RB) + r / RB) * 128 + (i & 127)) * RB + r % RB;
      if (T32) T32[o] = to_tf32(x);
      if (Thi) {
        __nv_bfloat16 hi = __float2bfloat16_rn(x);
        Thi[o] = hi;
        Tlo[o] = __float2bfloat16_rn(x - __bfloat162float(hi));
      }
      if (Tf) Tf[o] = x;
    }
  }
}

// rho(r) = g sum_i f_i psi_i(r)^2 + floor, one warp per grid point (Eq. densityChFSI)
__global__ void k_density(const void* __restrict__ psi, int io_dtype, int ld, long long Ng, int ns,
                          const double* __restrict__ occ, double g, double floor,
                          double* __restrict__ rho) {
  int lane = threadIdx.x & 31;
  long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < Ng; r += nwarps) {
    double acc = 0.0;
    for (int i = lane; i < ns; i += 32) {
      double p = load_io(psi, io_dtype, r * ld + i);
      acc += occ[i] * p * p;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rho[r] = g * acc + floor;
  }
}

__global__ void k_copy_rho(const void* __restrict__ src, int io_dtype, long long Ng,
                           double* __restrict__ rho) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < Ng;
       r += (long long)gridDim.x * blockDim.x)
    rho[r] = load_io(src, io_dtype, r);
}

// LDA exchange kernel dV_x/drho = -(1/3) c rho^(-2/3), c = (3/pi)^(1/3)
// (restricted) or (6/pi)^(1/3) (one spin channel); density floored at 1e-12.
__global__ void k_fx(const double* __restrict__ rho, long long Ng, int spin_polarized,
                     double* __restrict__ fx) {
  const double c = spin_polarized ? 1.2407009817988002 /* (6/pi)^(1/3) */
                                  : 0.98474502184269654 /* (3/pi)^(1/3) */;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < Ng;
       r += (long long)gridDim.x * blockDim.x) {
    double x = fmax(rho[r], 1e-12);
    double t = rcbrt(x);
    fx[r] = -(c / 3.0) * t * t;
  }
}

__device__ __forceinline__ double log_cosh(double y) {
  double a = fabs(y);
  return a + log1p(exp(-2.0 * a)) - 0.69314718055994531;
}

// log(sinh(u)/u), even in u
__device__ __forceinline__ double log_sinhc(double u) {
  double a = fabs(u);
  if (a == 0.0) return 0.0;
  if (a < 0.5) return log1p(sinh(a) / a - 1.0);
  return a + log1p(-exp(-2.0 * a)) - 0.69314718055994531 - log(a);
}

// Loewner matrix of the Fermi function at eps:
//   L_ij = -sinhc((x_i - x_j)/2) / (4 kT cosh(x_i/2) cosh(x_j/2)), x = (eps - mu)/kT,
// equal to (f_i - f_j)/(eps_i - eps_j) and to -f(1-f)/kT on the diagonal, with no
// cancellation for near-degenerate pairs.  Log domain where a factor could overflow.
// occ_mode: divided differences of the given occupations, midpoint derivative
// for |eps_i - eps_j| <= degen_tol kT.
__global__ void k_loewner_f32(const double* __restrict__ L, int ns, int ns_pad,
                              float* __restrict__ Lf) {
  const long long total = (long long)ns_pad * ns_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ns_pad), j = (int)(e - (long long)i * ns_pad);
    Lf[e] = (i < ns && j < ns) ? (float)L[(long long)i * ns + j] : 0.f;
  }
}

// artanh(w) / w, even in w, |w| < 1
__device__ __forceinline__ double artanhc(double w) {
  const double a = fabs(w);
  if (a < 1e-4) return 1.0 + a * a / 3.0;
  return atanh(a) / a;
}

// Loewner matrix of f_T(e) = 1 / (1 + exp(g(e))), g = c artanh(u), c = 2^(T+1),
// u = (e - mu) / (c kT), |u| < 1: with
//   f_i - f_j = -sinh((g_i - g_j)/2) / (2 cosh(g_i/2) cosh(g_j/2)) and
//   g_i - g_j = c artanh(w), w = (u_i - u_j) / (1 - u_i u_j),  u_i - u_j = (e_i - e_j)/(c kT),
//   L_ij = -sinhc((g_i - g_j)/2) artanhc(w) / (4 kT (1 - u_i u_j) cosh(g_i/2) cosh(g_j/2)),
// free of cancellation for close e_i, e_j; in the log domain where a factor
// would overflow.  The diagonal (w = 0) is f_T'.
__device__ double loewner_T(double ei, double ej, double mu, double kT, int T) {
  const double c = ldexp(1.0, T + 1);
  const double ui = (ei - mu) / (c * kT), uj = (ej - mu) / (c * kT);
  const double gi = c * atanh(ui), gj = c * atanh(uj);
  const double den = 1.0 - ui * uj;
  const double w = (ui - uj) / den;
  const double hd = 0.5 * (gi - gj);
  if (fabs(gi) < 1400.0 && fabs(gj) < 1400.0 && fabs(hd) < 700.0) {
    const double sc = hd == 0.0 ? 1.0 : sinh(hd) / hd;
    return -sc * artanhc(w) / (4.0 * kT * den * cosh(0.5 * gi) * cosh(0.5 * gj));
  }
  const double lm = log_sinhc(hd) + log(artanhc(w)) - log(4.0 * kT * den) - log_cosh(0.5 * gi) -
                    log_cosh(0.5 * gj);
  return -exp(lm);
}

__global__ void k_loewner(const double* __restrict__ eps, const double* __restrict__ occ, int ns,
                          double mu, double kT, int occ_mode, double degen_tol, int fermi_T,
                          double* __restrict__ L) {
  long long total = (long long)ns * ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / ns), j = (int)(e - (long long)i * ns);
    double val;
    if (fermi_T > 0) {
      val = loewner_T(eps[i], eps[j], mu, kT, fermi_T);
    } else if (occ_mode) {
      double de = eps[i] - eps[j];
      if (fabs(de) <= degen_tol * kT) {
        double fb = 0.5 * (occ[i] + occ[j]);
        val = -fb * (1.0 - fb) / kT;
      } else {
        val = (occ[i] - occ[j]) / de;
      }
    } else {
      double xi = (eps[i] - mu) / kT, xj = (eps[j] - mu) / kT;
      double u = 0.5 * (xi - xj);
      if (fabs(xi) < 700.0 && fabs(xj) < 700.0 && fabs(u) < 700.0) {
        double sc = (u == 0.0) ? 1.0 : sinh(u) / u;
        val = -sc / (4.0 * kT * cosh(0.5 * xi) * cosh(0.5 * xj));
      } else {
        double lm = log_sinhc(u) - log(4.0 * kT) - log_cosh(0.5 * xi) - log_cosh(0.5 * xj);
        val = -exp(lm);
      }
    }
    L[e] = val;
  }
}

__global__ void k_to_io(const double* __restrict__ src, long long n, void* __restrict__ dst,
                        int io_dtype) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    if (io_dtype == LRDM_DTYPE_F64) static_cast<double*>(dst)[r] = src[r];
    else static_cast<float*>(dst)[r] = (float)src[r];
  }
}

inline int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  if (b > 152LL * 64) b = 152LL * 64;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_convert_psi(const void* src, int io_dtype, int ld, long long Ng, int ns,
                               Channel& c, int prec, long long Ng_pad, cudaStream_t st) {
  if (prec == LRDM_FP64 || prec == LRDM_FP32) {
    k_copy_rowmajor<<<grid_for(Ng * ns, 256), 256, 0, st>>>(src, io_dtype, ld, Ng, ns, c.psi64,
                                                             c.psi32);
    return cudaGetLastError();
  }
  dim3 blk(32, 8);
  dim3 grd((unsigned)((Ng_pad + 31) / 32), (unsigned)((c.ns_pad + 31) / 32));
  k_copy_tc<<<grd, blk, 0, st>>>(src, io_dtype, ld, Ng, ns, Ng_pad, c.ns_pad, c.psiR32, c.psiT32,
                                 c.psiR_hi, c.psiR_lo, c.psiT_hi, c.psiT_lo, c.psiTf);
  return cudaGetLastError();
}

cudaError_t launch_density(const void* psi_src, int io_dtype, int ld, long long Ng, int ns,
                           const double* occ, double g, double floor, double* rho,
                           cudaStream_t st) {
  k_density<<<grid_for(Ng * 32, 256), 256, 0, st>>>(psi_src, io_dtype, ld, Ng, ns, occ, g, floor,
                                                     rho);
  return cudaGetLastError();
}

cudaError_t launch_copy_rho(const void* src, int io_dtype, long long Ng, double* rho,
                            cudaStream_t st) {
  k_copy_rho<<<grid_for(Ng, 256), 256, 0, st>>>(src, io_dtype, Ng, rho);
  return cudaGetLastError();
}

cudaError_t launch_fx(const double* rho, long long Ng, int spin_polarized, double* fx,
                      cudaStream_t st) {
  k_fx<<<grid_for(Ng, 256), 256, 0, st>>>(rho, Ng, spin_polarized, fx);
  return cudaGetLastError();
}

cudaError_t launch_loewner(const double* eps, const double* occ, int ns, double mu, double kT,
                           int occ_mode, double degen_tol, int fermi_T, double* L,
                           cudaStream_t st) {
  k_loewner<<<grid_for((long long)ns * ns, 256), 256, 0, st>>>(eps, occ, ns, mu, kT, occ_mode,
                                                                degen_tol, fermi_T, L);
  return cudaGetLastError();
}

cudaError_t launch_loewner_f32(const double* L, int ns, int ns_pad, float* Lf, cudaStream_t st) {
  k_loewner_f32<<<grid_for((long long)ns_pad * ns_pad, 256), 256, 0, st>>>(L, ns, ns_pad, Lf);
  return cudaGetLastError();
}

cudaError_t launch_to_io(const double* src, long long n, void* dst, int io_dtype,
                         cudaStream_t st) {
  k_to_io<<<grid_for(n, 256), 256, 0, st>>>(src, n, dst, io_dtype);
  return cudaGetLastError();
}

}  // namespace lrdm
