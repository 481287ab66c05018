// Element-wise and reduction kernels of the hot path: the perturbation
// potential (Hartree symbol, LDA kernel, quadrature weight), the chemical-
// potential shift mu' and the Loewner scaling of the projected matrices, and
// the backward-only reductions.  All FP64 arithmetic where the result feeds an
// FP64 quantity (mu', L, eps_bar, occ_bar).
#include "lrdm_internal.h"

#include <math.h>

namespace lrdm {
namespace {

__device__ __forceinline__ double ld_c(const void* p, int fp64, long long i) {
  return fp64 ? static_cast<const double*>(p)[i] : (double)static_cast<const float*>(p)[i];
}
__device__ __forceinline__ void st_c(void* p, int fp64, long long i, double x) {
  if (fp64) static_cast<double*>(p)[i] = x;
  else static_cast<float*>(p)[i] = (float)x;
}

inline int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

#define GRID_STRIDE(e, n)                                                          \
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (n); \
       e += (long long)gridDim.x * blockDim.x)

// Grid-length element-wise kernels: one thread per four consecutive grid
// points r0 .. r0 + 3, looping over the directions k (and spins s) so that
// the per-point factors (f_x, the symbol) are read and converted once; every
// row access of a warp is contiguous, 16-byte vector loads and stores when
// `vec` (all row starts 16-byte aligned).  Arithmetic in the compute type C
// (float in the FP32 / TF32 / BF16x3 modes, double in FP64 mode).
template <typename T>
__device__ __forceinline__ void ld4(const T* __restrict__ p, int n, bool vec, T (&o)[4]) {
  if (vec && n == 4) {
    if constexpr (sizeof(T) == 4) {
      const float4 t = *reinterpret_cast<const float4*>(p);
      o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
      const double2 a = reinterpret_cast<const double2*>(p)[0];
      const double2 b = reinterpret_cast<const double2*>(p)[1];
      o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] = e < n ? p[e] : T(0);
  }
}
template <typename T>
__device__ __forceinline__ void st4(T* __restrict__ p, int n, bool vec, const T (&v)[4]) {
  if (vec && n == 4) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
      reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < n) p[e] = v[e];
  }
}
__device__ __forceinline__ int quad_count(long long len, long long r0) {
  const long long n = len - r0;
  return n <= 0 ? 0 : (n >= 4 ? 4 : (int)n);
}

// out[k * ostride + r] = sum_s v[k][s][r]
template <typename Ti, typename C>
__global__ void k_spin_sum(const Ti* __restrict__ v, int K, int nspin, long long Ng,
                           C* __restrict__ out, long long ostride, int vec) {
  const long long r0 = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  const int n = quad_count(Ng, r0);
  if (n == 0) return;
  for (int k = 0; k < K; ++k) {
    C acc[4] = {C(0), C(0), C(0), C(0)};
    for (int s = 0; s < nspin; ++s) {
      Ti x[4];
      ld4(v + ((long long)k * nspin + s) * Ng + r0, n, vec, x);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] += (C)x[e];
    }
    st4(out + (long long)k * ostride + r0, n, vec, acc);
  }
}

// Multiplies the half-spectrum (R2C layout [K][n0][n1][n2/2+1]) by
// 4 pi / |G|^2 / N_g (G = 0 -> 0); kind 1 replaces |G|^2 by the second-order
// finite-difference symbol sum_d (4/h_d^2) sin^2(G_d h_d / 2).
__global__ void k_poisson_table(int n0, int n1, int n2, double h0, double h1, double h2, int kind,
                                double* __restrict__ sym) {
  const int m2n = n2 / 2 + 1;
  const long long per = (long long)n0 * n1 * m2n;
  const double inv_ng = 1.0 / ((double)n0 * n1 * n2);
  const double two_pi = 6.283185307179586;
  GRID_STRIDE(e, per) {
    int m2 = (int)(e % m2n);
    long long t = e / m2n;
    int m1 = (int)(t % n1);
    int m0 = (int)(t / n1);
    int f0 = m0 <= n0 / 2 ? m0 : m0 - n0;
    int f1 = m1 <= n1 / 2 ? m1 : m1 - n1;
    int f2 = m2;
    double g0 = two_pi * f0 / (n0 * h0), g1 = two_pi * f1 / (n1 * h1), g2 = two_pi * f2 / (n2 * h2);
    double q;
    if (kind == 1) {
      double s0 = sin(0.5 * g0 * h0), s1 = sin(0.5 * g1 * h1), s2 = sin(0.5 * g2 * h2);
      q = 4.0 * (s0 * s0 / (h0 * h0) + s1 * s1 / (h1 * h1) + s2 * s2 / (h2 * h2));
    } else {
      q = g0 * g0 + g1 * g1 + g2 * g2;
    }
    sym[e] = (f0 == 0 && f1 == 0 && f2 == 0) || q <= 0.0 ? 0.0 : 12.566370614359172 / q * inv_ng;
  }
}

// Applies the symbol table to all K transformed fields: one thread per
// half-complex point, looping over the fields (the symbol is read once).
__global__ void k_poisson(void* __restrict__ cplx, int K, long long per,
                          const double* __restrict__ sym, int fp64) {
  GRID_STRIDE(m, per) {
    const double sm = sym[m];
    if (fp64) {
      double2* z = static_cast<double2*>(cplx);
      for (int k = 0; k < K; ++k) {
        double2 v = z[(long long)k * per + m];
        v.x *= sm;
        v.y *= sm;
        z[(long long)k * per + m] = v;
      }
    } else {
      float2* z = static_cast<float2*>(cplx);
      const float sf = (float)sm;
      for (int k = 0; k < K; ++k) {
        float2 v = z[(long long)k * per + m];
        v.x *= sf;
        v.y *= sf;
        z[(long long)k * per + m] = v;
      }
    }
  }
}

// a[k][s][r] = scale (V_H[k][r] + f_xs[r] v[k][s][r]) for r < Ng; rows
// Ng <= r < Ng_pad are zero
template <typename Ti, typename C>
__global__ void k_dv_weights(const Ti* __restrict__ v, const C* __restrict__ VH,
                             const double* __restrict__ fx0, const double* __restrict__ fx1, int K,
                             int nspin, long long Ng, long long Ng_pad, C scale,
                             C* __restrict__ a, long long vstride, int vec) {
  const long long r0 = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  const int n_out = quad_count(Ng_pad, r0);
  if (n_out == 0) return;
  const int n = quad_count(Ng, r0);
  C fx[2][4];                            // nspin <= 2; unrolled so that fx stays in registers
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const double* f = s == 0 ? fx0 : fx1;
#pragma unroll
    for (int e = 0; e < 4; ++e) fx[s][e] = e < n ? (C)f[r0 + e] : C(0);
  }
  for (int k = 0; k < K; ++k) {
    C vh[4];
    ld4(VH + (long long)k * vstride + r0, n, vec, vh);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (s >= nspin) break;
      const long long q = (long long)k * nspin + s;
      Ti x[4];
      ld4(v + q * Ng + r0, n, vec, x);
      C o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = e < n ? scale * (vh[e] + fx[s][e] * (C)x[e]) : C(0);
      st4(a + q * Ng_pad + r0, n_out, vec, o);
    }
  }
}

// vbar[k][s][r] = V_H[sum_s dVbar][k][r] + f_xs[r] dVbar[k][s][r] - fbar[k][s][r]
template <typename Ti, typename C>
__global__ void k_adjoint_potential(const C* __restrict__ dvbar, const C* __restrict__ VH,
                                    const double* __restrict__ fx0, const double* __restrict__ fx1,
                                    const Ti* __restrict__ fbar, int K, int nspin, long long Ng,
                                    long long Ng_pad, Ti* __restrict__ vbar, long long vstride,
                                    int vec) {
  const long long r0 = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  const int n = quad_count(Ng, r0);
  if (n == 0) return;
  C fx[2][4];                            // nspin <= 2; unrolled so that fx stays in registers
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const double* f = s == 0 ? fx0 : fx1;
#pragma unroll
    for (int e = 0; e < 4; ++e) fx[s][e] = e < n ? (C)f[r0 + e] : C(0);
  }
  for (int k = 0; k < K; ++k) {
    C vh[4];
    ld4(VH + (long long)k * vstride + r0, n, vec, vh);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (s >= nspin) break;
      const long long q = (long long)k * nspin + s;
      C d[4];
      Ti fb[4], o[4];
      ld4(dvbar + q * Ng_pad + r0, n, vec, d);
      ld4(fbar + q * Ng + r0, n, vec, fb);
#pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = (Ti)(vh[e] + fx[s][e] * d[e] - (C)fb[e]);
      st4(vbar + q * Ng + r0, n, vec, o);
    }
  }
}

// spin sum of the (padded) adjoint potential for the Hartree transform
template <typename C>
__global__ void k_spin_sum_padded(const C* __restrict__ d, int K, int nspin, long long Ng,
                                  long long Ng_pad, C* __restrict__ out, long long ostride, int vec) {
  const long long r0 = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  const int n = quad_count(Ng, r0);
  if (n == 0) return;
  for (int k = 0; k < K; ++k) {
    C acc[4] = {C(0), C(0), C(0), C(0)};
    for (int s = 0; s < nspin; ++s) {
      C x[4];
      ld4(d + ((long long)k * nspin + s) * Ng_pad + r0, n, vec, x);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] += x[e];
    }
    st4(out + (long long)k * ostride + r0, n, vec, acc);
  }
}

// a[k][s][r] = scale fbar[k][s][r] for r < Ng, zero for Ng <= r < Ng_pad
template <typename Ti, typename C>
__global__ void k_scale_weights(const Ti* __restrict__ fbar, int K, int nspin, long long Ng,
                                long long Ng_pad, C scale, C* __restrict__ a, int vec) {
  const long long r0 = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  const int n_out = quad_count(Ng_pad, r0);
  if (n_out == 0) return;
  const int n = quad_count(Ng, r0);
  for (int q = 0; q < K * nspin; ++q) {
    Ti x[4];
    ld4(fbar + (long long)q * Ng + r0, n, vec, x);
    C o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] = e < n ? scale * (C)x[e] : C(0);
    st4(a + (long long)q * Ng_pad + r0, n_out, vec, o);
  }
}

// One block per direction k.  mu'_k = sum_s sum_i L_ii X_ii / sum_s sum_i L_ii
// with X summed over the grid splits.  Also flags non-finite X.
struct DmuArgs {
  const void* X[2];
  const double* L[2];
  int ns[2];
  int ldx[2];
  int nsplit;
  int nspin;
  int K;
};
__global__ void k_dmu(DmuArgs A, int acc64, double* __restrict__ dmu, double* __restrict__ dmu_out,
                      int* __restrict__ status) {
  int k = blockIdx.x;
  double num = 0.0, den = 0.0;
  for (int s = 0; s < A.nspin; ++s) {
    long long mat = (long long)A.ldx[s] * A.ldx[s];
    for (int i = threadIdx.x; i < A.ns[s]; i += blockDim.x) {
      double x = 0.0;
      for (int p = 0; p < A.nsplit; ++p)
        x += ld_c(A.X[s], acc64, ((long long)p * A.K + k) * mat + (long long)i * A.ldx[s] + i);
      double l = A.L[s][(long long)i * A.ns[s] + i];
      num += l * x;
      den += l;
    }
  }
  __shared__ double sn[32], sd[32];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sn[wid] = num; sd[wid] = den; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sn[w]; b += sd[w]; }
    double m = b != 0.0 ? a / b : 0.0;
    if (!isfinite(m)) { atomicOr(status, STATUS_NONFINITE); }
    dmu[k] = m;
    if (dmu_out) dmu_out[k] = m;
  }
}

// X'' in one of three layouts:
//   layout 0: out[k][i][j] (ld = ns)        -- CUDA-core GEMM2, compute type
//   layout 1: out[k][j][i] (ld = ns_pad) fp32 -- TF32 GEMM2 B operand (K-major)
//   layout 2: out_hi/out_lo[k][j][i] bf16     -- BF16X3 GEMM2 B operand (K-major)
// value c_ij * (L_ij (X_ij - delta_ij shift_k)) with c = 2, 1, 0 for i <, =, > j.
// Adjoint form (adjoint = 1): L_ij G_ij - delta_ij L_ii shift_k * inv_trace.
// X is the full symmetric matrix (GEMM1 writes both triangles), summed over splits.
__global__ void k_loewner_scale(const void* __restrict__ X, int acc64, int nsplit, int K, int ns,
                                int ldx, const double* __restrict__ L,
                                const double* __restrict__ shift, int adjoint, double inv_trace,
                                int layout, int ldo, void* __restrict__ out,
                                __nv_bfloat16* __restrict__ out_lo) {
  long long mat_x = (long long)ldx * ldx;
  long long mat_o = (long long)ldo * ldo;
  GRID_STRIDE(e, (long long)K * mat_o) {
    long long k = e / mat_o, rem = e - k * mat_o;
    int row = (int)(rem / ldo), col = (int)(rem - (long long)row * ldo);
    // layout 0: (row, col) = (i, j);  layouts 1, 2: (row, col) = (j, i)
    int i = layout == 0 ? row : col;
    int j = layout == 0 ? col : row;
    double val = 0.0;
    if (i < ns && j < ns && i <= j) {
      double x = 0.0;
      // read the (row, col) entry: X and L are symmetric
      for (int p = 0; p < nsplit; ++p)
        x += ld_c(X, acc64, ((long long)p * K + k) * mat_x + (long long)row * ldx + col);
      double l = L[(long long)row * ns + col];
      double xp;
      if (adjoint) xp = l * x - (i == j ? l * shift[k] * inv_trace : 0.0);
      else xp = l * (x - (i == j ? shift[k] : 0.0));
      val = (i == j ? 1.0 : 2.0) * xp;
    }
    if (layout == 0) {
      st_c(out, acc64, e, val);
    } else if (layout == 1) {
      uint32_t t;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"((float)val));
      static_cast<float*>(out)[e] = __uint_as_float(t);
    } else {
      float v32 = (float)val;
      __nv_bfloat16 hi = __float2bfloat16_rn(v32);
      static_cast<__nv_bfloat16*>(out)[e] = hi;
      out_lo[e] = __float2bfloat16_rn(v32 - __bfloat162float(hi));
    }
  }
}

// X'' for the tensor-core response GEMM: entry (k, row = j, col = i) =
// c_ij L_ij (X_ij - delta_ij shift_k) (adjoint: c_ij (L_ij X_ij - delta_ij
// L_ii shift_k inv_trace)), c = 2 / 1 / 0 for i < j / i = j / i > j, rounded to
// TF32 (layout 1) or split into bf16 hi / lo (layout 2).  Off-diagonal products
// in FP32 with the FP32 copy of L (the result is stored with at most 16
// significant bits); the diagonal (mu' shift) in FP64.  One thread per four
// consecutive columns of one row, looping over the K directions so that the
// row's L entries are read once: grid (column quads, rows).
__global__ void k_loewner_scale_tc(const float* __restrict__ X, int nsplit, int K, int ns, int ld,
                                   const float* __restrict__ Lf, const double* __restrict__ L,
                                   const double* __restrict__ shift, int adjoint,
                                   double inv_trace, int layout, void* __restrict__ out,
                                   __nv_bfloat16* __restrict__ out_lo) {
  const int c0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int row = blockIdx.y;
  if (c0 >= ld) return;
  const long long mat = (long long)ld * ld;
  const long long base = (long long)row * ld + c0;
  const float4 l4 = *reinterpret_cast<const float4*>(Lf + base);
  const float ls[4] = {l4.x, l4.y, l4.z, l4.w};
  // column c0 + dg is the diagonal of this row when 0 <= dg < 4
  const int dg = row - c0;
  const double ldiag = (dg >= 0 && dg < 4 && row < ns) ? L[(long long)row * ns + row] : 0.0;
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    const long long o = (long long)k * mat + base;
    // X: [nsplit][K][ld][ld] partial sums over grid-row ranges, added in order
    float4 x4 = *reinterpret_cast<const float4*>(X + o);
    for (int p = 1; p < nsplit; ++p) {
      const float4 y = *reinterpret_cast<const float4*>(X + o + (long long)p * K * mat);
      x4.x += y.x;
      x4.y += y.y;
      x4.z += y.z;
      x4.w += y.w;
    }
    const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = c0 + e, j = row;
      if (i < j && j < ns) {
        v[e] = 2.f * ls[e] * xs[e];
      } else if (i == j && j < ns) {
        v[e] = (float)(adjoint ? ldiag * (double)xs[e] - ldiag * shift[k] * inv_trace
                               : ldiag * ((double)xs[e] - shift[k]));
      } else {
        v[e] = 0.f;
      }
    }
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
}

// Backward trace terms T_k = sum_s sum_m L_mm Gbar_k,mm (the adjoint of the
// mu' constraint) -- same reduction as k_dmu without the division.
__global__ void k_trace_bar(DmuArgs A, int acc64, double* __restrict__ tbar) {
  int k = blockIdx.x;
  double num = 0.0;
  for (int s = 0; s < A.nspin; ++s) {
    long long mat = (long long)A.ldx[s] * A.ldx[s];
    for (int i = threadIdx.x; i < A.ns[s]; i += blockDim.x) {
      double x = 0.0;
      for (int p = 0; p < A.nsplit; ++p)
        x += ld_c(A.X[s], acc64, ((long long)p * A.K + k) * mat + (long long)i * A.ldx[s] + i);
      num += A.L[s][(long long)i * A.ns[s] + i] * x;
    }
  }
  __shared__ double sn[32];
  for (int o = 16; o > 0; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
  if ((threadIdx.x & 31) == 0) sn[threadIdx.x >> 5] = num;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sn[w];
    tbar[k] = a;
  }
}

// One block per state i of channel s:
//   Lbar_ij = sum_k G_k,ij (X_k,ij - delta_ij mu'_k) - delta_ij sum_k tbar_k/s (X_k,ii - mu'_k)
//   eps_bar_i = sum_{j != i, |de| > tau} 2 Lbar_ij (-L_ij / (eps_i - eps_j))
//   occ_bar_i = sum_{j != i, |de| > tau} 2 Lbar_ij / (eps_i - eps_j)
//             + sum_{j != i, |de| <= tau} 2 Lbar_ij (-(1 - 2 fbar)/(2 kT)) + Lbar_ii (-(1 - 2 f_i)/kT)
//
// With FP32 partials (the tensor-core and FP32 modes) Lbar_ij (j != i) is
// summed over the directions in FP32, four consecutive j per thread with
// 16-byte loads when the leading dimension allows; where the FP32 copy of L
// exists (Lf, leading dimension ldf: the tensor-core modes) the terms of a gap
// above tau are formed in FP32 from the FP64 gap, summed per thread in FP32
// and added to the FP64 sums once (Lbar itself carries FP32 rounding there).
struct EobArgs {
  const double* L;
  const float* Lf;
  int ldf;
  const double* eps;
  const double* occ;
  double kT, tau;
};

__device__ __forceinline__ void eob_term(const EobArgs& a, int i, int j, double eps_i, double lb,
                                         int ns, double& eb, double& ob, float& ebf, float& obf) {
  const double de = eps_i - a.eps[j];
  if (i == j) {
    ob += lb * (-(1.0 - 2.0 * a.occ[i]) / a.kT);
  } else if (fabs(de) > a.tau && a.Lf) {
    const float t = 2.f * (float)lb / (float)de;
    ebf = fmaf(-t, a.Lf[(long long)i * a.ldf + j], ebf);
    obf += t;
  } else if (fabs(de) > a.tau) {
    const double rde = 1.0 / de;
    eb += 2.0 * lb * (-a.L[(long long)i * ns + j] * rde);
    ob += 2.0 * lb * rde;
  } else {
    const double fb = 0.5 * (a.occ[i] + a.occ[j]);
    ob += 2.0 * lb * (-(1.0 - 2.0 * fb) / (2.0 * a.kT));
  }
}

// Lbar_ij in FP64 (the FP64 mode, and the diagonal in every mode)
__device__ __forceinline__ double eob_lbar64(const void* X, const void* G, int acc64, int nsplit,
                                             int K, long long mat, long long row, int i, int j,
                                             const double* dmu, const double* tbar,
                                             double inv_trace) {
  double lb = 0.0;
  for (int k = 0; k < K; ++k) {
    double x = 0.0, gg = 0.0;
    for (int p = 0; p < nsplit; ++p) {
      const long long o = ((long long)p * K + k) * mat + row + j;
      x += ld_c(X, acc64, o);
      gg += ld_c(G, acc64, o);
    }
    if (i == j) lb += gg * (x - dmu[k]) - tbar[k] * inv_trace * (x - dmu[k]);
    else lb += gg * x;
  }
  return lb;
}

__global__ void k_eps_occ_bar(const void* __restrict__ X, const void* __restrict__ G, int acc64,
                              int nsplit, int K, int ns, int ldx, EobArgs a,
                              const double* __restrict__ dmu, const double* __restrict__ tbar,
                              double inv_trace, double* __restrict__ eps_bar,
                              double* __restrict__ occ_bar) {
  const int i = blockIdx.x;
  const long long mat = (long long)ldx * ldx;
  const long long row = (long long)i * ldx;
  double eb = 0.0, ob = 0.0;
  float ebf = 0.f, obf = 0.f;
  const double eps_i = a.eps[i];
  if (!acc64 && ldx % 4 == 0) {
    // FP32 partials: rows of 16-byte quads (ldx is a multiple of 4, so a quad
    // starting below ns stays inside the padded row)
    const float* Xf = static_cast<const float*>(X);
    const float* Gf = static_cast<const float*>(G);
    for (int j0 = 4 * threadIdx.x; j0 < ns; j0 += 4 * blockDim.x) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      if (nsplit == 1) {
        // one partial: unrolled so that several directions' loads are in flight
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
          const long long o = (long long)k * mat + row + j0;
          const float4 x = *reinterpret_cast<const float4*>(Xf + o);
          const float4 g = *reinterpret_cast<const float4*>(Gf + o);
          acc[0] = fmaf(g.x, x.x, acc[0]);
          acc[1] = fmaf(g.y, x.y, acc[1]);
          acc[2] = fmaf(g.z, x.z, acc[2]);
          acc[3] = fmaf(g.w, x.w, acc[3]);
        }
      } else {
        for (int k = 0; k < K; ++k) {
          float4 x = make_float4(0.f, 0.f, 0.f, 0.f), g = x;
          for (int p = 0; p < nsplit; ++p) {
            const long long o = ((long long)p * K + k) * mat + row + j0;
            const float4 xv = *reinterpret_cast<const float4*>(Xf + o);
            const float4 gv = *reinterpret_cast<const float4*>(Gf + o);
            x.x += xv.x; x.y += xv.y; x.z += xv.z; x.w += xv.w;
            g.x += gv.x; g.y += gv.y; g.z += gv.z; g.w += gv.w;
          }
          acc[0] = fmaf(g.x, x.x, acc[0]);
          acc[1] = fmaf(g.y, x.y, acc[1]);
          acc[2] = fmaf(g.z, x.z, acc[2]);
          acc[3] = fmaf(g.w, x.w, acc[3]);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = j0 + e;
        if (j >= ns) break;
        const double lb = j == i ? eob_lbar64(X, G, 0, nsplit, K, mat, row, i, j, dmu, tbar, inv_trace)
                                 : (double)acc[e];
        eob_term(a, i, j, eps_i, lb, ns, eb, ob, ebf, obf);
      }
    }
  } else {
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
      double lb;
      if (acc64 || i == j) {
        lb = eob_lbar64(X, G, acc64, nsplit, K, mat, row, i, j, dmu, tbar, inv_trace);
      } else {
        // FP32 partials with an unaligned leading dimension
        const float* Xf = static_cast<const float*>(X);
        const float* Gf = static_cast<const float*>(G);
        float acc = 0.f;
        for (int k = 0; k < K; ++k) {
          float x = 0.f, gg = 0.f;
          for (int p = 0; p < nsplit; ++p) {
            const long long o = ((long long)p * K + k) * mat + row + j;
            x += Xf[o];
            gg += Gf[o];
          }
          acc = fmaf(gg, x, acc);
        }
        lb = (double)acc;
      }
      eob_term(a, i, j, eps_i, lb, ns, eb, ob, ebf, obf);
    }
  }
  eb += (double)ebf;
  ob += (double)obf;
  __shared__ double se[32], so[32];
  for (int o = 16; o > 0; o >>= 1) {
    eb += __shfl_xor_sync(0xffffffffu, eb, o);
    ob += __shfl_xor_sync(0xffffffffu, ob, o);
  }
  if ((threadIdx.x & 31) == 0) { se[threadIdx.x >> 5] = eb; so[threadIdx.x >> 5] = ob; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += se[w]; s1 += so[w]; }
    if (eps_bar) eps_bar[i] = s0;
    if (occ_bar) occ_bar[i] = s1;
  }
}

// out[i][j] = sum over splits of X[p][k][i][j] (FP64, ld = ns)
__global__ void k_get_projection(const void* __restrict__ X, int acc64, int nsplit, int K, int k,
                                 int ns, int ldx, double* __restrict__ out) {
  const long long mat = (long long)ldx * ldx;
  GRID_STRIDE(e, (long long)ns * ns) {
    const int i = (int)(e / ns), j = (int)(e - (long long)i * ns);
    double x = 0.0;
    for (int p = 0; p < nsplit; ++p) x += ld_c(X, acc64, ((long long)p * K + k) * mat + (long long)i * ldx + j);
    out[e] = x;
  }
}

}  // namespace

cudaError_t launch_get_projection(const SysState& S, int s, int k, int acc_fp64, double* out,
                                  cudaStream_t st) {
  const Channel& c = S.ch[s];
  const int tc = (c.psiR_hi || c.psiR32) ? 1 : 0;
  k_get_projection<<<grid_for((long long)c.ns * c.ns, 256), 256, 0, st>>>(
      c.Xpart, acc_fp64, S.nsplit, S.last_K, k, c.ns, tc ? c.ns_pad : c.ns, out);
  return cudaGetLastError();
}

// grid of the quad kernels: one thread per four consecutive points of `len`
inline unsigned quad_grid(long long len) {
  const long long quads = (len + 3) / 4;
  return (unsigned)((quads + 255) / 256);
}
inline bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Instantiates kernel<Ti, C> for the io dtype (Ti) and compute precision (C).
#define IO_C_DISPATCH(io, fp64, CALL)                              \
  do {                                                             \
    if (io == LRDM_DTYPE_F64) {                                    \
      if (fp64) { using Ti = double; using C = double; CALL; }     \
      else { using Ti = double; using C = float; CALL; }           \
    } else {                                                       \
      if (fp64) { using Ti = float; using C = double; CALL; }      \
      else { using Ti = float; using C = float; CALL; }            \
    }                                                              \
  } while (0)

cudaError_t launch_spin_sum(const void* v, int io_dtype, int K, int nspin, long long Ng,
                            void* fft_real, int fp64, cudaStream_t st, long long out_stride) {
  if (K == 0 || Ng == 0) return cudaSuccess;
  const int vec = Ng % 4 == 0 && out_stride % 4 == 0 && al16(v) && al16(fft_real);
  IO_C_DISPATCH(io_dtype, fp64,
                (k_spin_sum<Ti, C><<<quad_grid(Ng), 256, 0, st>>>(
                    static_cast<const Ti*>(v), K, nspin, Ng, static_cast<C*>(fft_real), out_stride,
                    vec)));
  return cudaGetLastError();
}

cudaError_t launch_poisson_table(const int* n, const double* h, int kind, double* sym,
                                 cudaStream_t st) {
  const long long per = (long long)n[0] * n[1] * (n[2] / 2 + 1);
  k_poisson_table<<<grid_for(per, 256), 256, 0, st>>>(n[0], n[1], n[2], h[0], h[1], h[2], kind, sym);
  return cudaGetLastError();
}

cudaError_t launch_poisson_symbol(void* cplx, int K, long long per, const double* sym, int fp64,
                                  cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  k_poisson<<<grid_for(per, 256), 256, 0, st>>>(cplx, K, per, sym, fp64);
  return cudaGetLastError();
}

cudaError_t launch_dv_weights(const void* v, int io_dtype, const void* VH, const double* fx0,
                              const double* fx1, int K, int nspin, long long Ng, long long Ng_pad,
                              double scale, void* a, int fp64, cudaStream_t st, long long vh_stride) {
  if (K == 0 || Ng_pad == 0) return cudaSuccess;
  const int vec = Ng % 4 == 0 && Ng_pad % 4 == 0 && vh_stride % 4 == 0 && al16(v) && al16(VH) &&
                  al16(a);
  IO_C_DISPATCH(io_dtype, fp64,
                (k_dv_weights<Ti, C><<<quad_grid(Ng_pad), 256, 0, st>>>(
                    static_cast<const Ti*>(v), static_cast<const C*>(VH), fx0, fx1, K, nspin, Ng,
                    Ng_pad, (C)scale, static_cast<C*>(a), vh_stride, vec)));
  return cudaGetLastError();
}

cudaError_t launch_adjoint_potential(const void* dvbar, const void* VH, const double* fx0,
                                     const double* fx1, const void* fbar, int io_dtype, int K,
                                     int nspin, long long Ng, long long Ng_pad, void* vbar,
                                     int fp64, cudaStream_t st, long long vh_stride) {
  if (K == 0 || Ng == 0) return cudaSuccess;
  const int vec = Ng % 4 == 0 && Ng_pad % 4 == 0 && vh_stride % 4 == 0 && al16(dvbar) && al16(VH) &&
                  al16(fbar) && al16(vbar);
  IO_C_DISPATCH(io_dtype, fp64,
                (k_adjoint_potential<Ti, C><<<quad_grid(Ng), 256, 0, st>>>(
                    static_cast<const C*>(dvbar), static_cast<const C*>(VH), fx0, fx1,
                    static_cast<const Ti*>(fbar), K, nspin, Ng, Ng_pad, static_cast<Ti*>(vbar),
                    vh_stride, vec)));
  return cudaGetLastError();
}

cudaError_t launch_spin_sum_padded(const void* d, int K, int nspin, long long Ng,
                                   long long Ng_pad, void* out, int fp64, cudaStream_t st,
                                   long long out_stride) {
  if (K == 0 || Ng == 0) return cudaSuccess;
  const int vec = Ng % 4 == 0 && Ng_pad % 4 == 0 && out_stride % 4 == 0 && al16(d) && al16(out);
  if (fp64)
    k_spin_sum_padded<double><<<quad_grid(Ng), 256, 0, st>>>(
        static_cast<const double*>(d), K, nspin, Ng, Ng_pad, static_cast<double*>(out), out_stride,
        vec);
  else
    k_spin_sum_padded<float><<<quad_grid(Ng), 256, 0, st>>>(
        static_cast<const float*>(d), K, nspin, Ng, Ng_pad, static_cast<float*>(out), out_stride,
        vec);
  return cudaGetLastError();
}

cudaError_t launch_scale_weights(const void* fbar, int io_dtype, int K, int nspin, long long Ng,
                                 long long Ng_pad, double scale, void* a, int fp64,
                                 cudaStream_t st) {
  if (K == 0 || Ng_pad == 0) return cudaSuccess;
  const int vec = Ng % 4 == 0 && Ng_pad % 4 == 0 && al16(fbar) && al16(a);
  IO_C_DISPATCH(io_dtype, fp64,
                (k_scale_weights<Ti, C><<<quad_grid(Ng_pad), 256, 0, st>>>(
                    static_cast<const Ti*>(fbar), K, nspin, Ng, Ng_pad, (C)scale,
                    static_cast<C*>(a), vec)));
  return cudaGetLastError();
}

static DmuArgs dmu_args(const SysState& S, const void* const* X, int K) {
  DmuArgs A{};
  int tc = (S.ch[0].psiR_hi || S.ch[0].psiR32) ? 1 : 0;
  for (int s = 0; s < S.nspin; ++s) {
    A.X[s] = X[s];
    A.L[s] = S.ch[s].L;
    A.ns[s] = S.ch[s].ns;
    A.ldx[s] = tc ? S.ch[s].ns_pad : S.ch[s].ns;
  }
  A.nsplit = S.nsplit;
  A.nspin = S.nspin;
  A.K = K;
  return A;
}

cudaError_t launch_dmu(const SysState& S, const void* const* Xparts, int K, int acc_fp64,
                       double* dmu, double* dmu_out, int* status, cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  k_dmu<<<K, 256, 0, st>>>(dmu_args(S, Xparts, K), acc_fp64, dmu, dmu_out, status);
  return cudaGetLastError();
}

cudaError_t launch_trace_bar(const SysState& S, const void* const* Gparts, int K, int acc_fp64,
                             double* tbar, cudaStream_t st) {
  if (K == 0) return cudaSuccess;
  k_trace_bar<<<K, 256, 0, st>>>(dmu_args(S, Gparts, K), acc_fp64, tbar);
  return cudaGetLastError();
}

cudaError_t launch_loewner_scale(const SysState& S, int s, const void* Xpart, int K, int acc_fp64,
                                 const double* shift, int adjoint, double inv_trace_L, int prec,
                                 cudaStream_t st) {
  const Channel& c = S.ch[s];
  int layout = prec == LRDM_BF16X3 ? 2 : (prec == LRDM_TF32 ? 1 : 0);
  if (K == 0) return cudaSuccess;
  if (layout != 0) {
    const int ld = c.ns_pad;                     // multiple of 128
    dim3 grid((ld / 4 + 127) / 128, ld);
    k_loewner_scale_tc<<<grid, 128, 0, st>>>(static_cast<const float*>(Xpart), S.nsplit, K, c.ns, ld,
                                              c.Lf, c.L,
                                              shift, adjoint, inv_trace_L, layout, c.Xpp,
                                              static_cast<__nv_bfloat16*>(c.Xpp_lo));
    return cudaGetLastError();
  }
  int ldx = c.ns;
  int ldo = c.ns;
  long long tot = (long long)K * ldo * ldo;
  k_loewner_scale<<<grid_for(tot, 256), 256, 0, st>>>(
      Xpart, acc_fp64, S.nsplit, K, c.ns, ldx, c.L, shift, adjoint, inv_trace_L, layout, ldo,
      c.Xpp, static_cast<__nv_bfloat16*>(c.Xpp_lo));
  return cudaGetLastError();
}

cudaError_t launch_eps_occ_bar(const SysState& S, int s, int K, int acc_fp64, double inv_trace_L,
                               double degen_tol, double* eps_bar, double* occ_bar,
                               cudaStream_t st) {
  const Channel& c = S.ch[s];
  int tc = (c.psiR_hi || c.psiR32) ? 1 : 0;
  int ldx = tc ? c.ns_pad : c.ns;
  // the FP32 copy of L exists in the tensor-core modes (leading dimension ns_pad)
  EobArgs a{c.L, acc_fp64 ? nullptr : c.Lf, c.ns_pad, c.eps, c.occ, S.kT, degen_tol * S.kT};
  k_eps_occ_bar<<<c.ns, 256, 0, st>>>(c.Xpart, c.Gpart, acc_fp64, S.nsplit, K, c.ns, ldx, a, S.dmu,
                                      S.tbar, inv_trace_L, eps_bar, occ_bar);
  return cudaGetLastError();
}

}  // namespace lrdm
