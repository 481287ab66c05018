// Host side of the C ABI declared in include/lrdm.h: argument validation,
// set-up (chemical potential, occupations, Loewner matrix, xc kernel, operand
// copies, cuFFT plans, workspaces) and the launch sequences of the forward,
// least-squares and adjoint calls.  The accumulated driver (LRDMA) and the
// Brillouin-zone-sampled systems have files of their own.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "api_common.h"

using namespace lrdm;
using namespace lrdm::api;

namespace lrdm {
namespace api {

lrdm_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LRDM_OK;
  // LRDM_DEBUG=1 in the environment prints the CUDA error behind a failure
  static const bool debug = getenv("LRDM_DEBUG") != nullptr;
  if (debug) fprintf(stderr, "liblrdm: CUDA error %d (%s): %s\n", (int)e, cudaGetErrorName(e),
                     cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LRDM_ERR_OOM : LRDM_ERR_CUDA;
}
lrdm_status from_cufft(cufftResult r) {
  if (r == CUFFT_SUCCESS) return LRDM_OK;
  return r == CUFFT_ALLOC_FAILED ? LRDM_ERR_OOM : LRDM_ERR_CUDA;
}

// Numerically stable Fermi function f = 1/(1 + exp(x)).
double fermi_host(double x) {
  if (x > 0) {
    double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

// mu with g sum_s sum_i f((eps - mu)/kT) = N_e by bisection (Eq. kseqcont).
lrdm_status solve_mu_host(const std::vector<std::vector<double>>& eps, double ne, double kT,
                          double g, double* mu_out) {
  size_t nstates = 0;
  double lo = 1e300, hi = -1e300;
  for (auto& e : eps) {
    nstates += e.size();
    for (double x : e) {
      lo = fmin(lo, x);
      hi = fmax(hi, x);
    }
  }
  if (!(ne > 0.0 && ne < g * (double)nstates)) return LRDM_ERR_MU_NOT_CONVERGED;
  lo -= 800.0 * kT;
  hi += 800.0 * kT;
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    double cnt = 0.0;
    for (auto& e : eps)
      for (double x : e) cnt += fermi_host((x - mid) / kT);
    cnt *= g;
    if (cnt < ne) lo = mid;
    else hi = mid;
  }
  double mu = 0.5 * (lo + hi);
  if (!isfinite(mu)) return LRDM_ERR_MU_NOT_CONVERGED;
  *mu_out = mu;
  return LRDM_OK;
}


constexpr int PROF_MAX = 4096;

// Records the start event of a timed contraction; returns the pair index or -1.
int prof_begin(lrdm_ctx* ctx, int kind, cudaStream_t st) {
  if (!ctx->prof_on || ctx->prof_n >= PROF_MAX) return -1;
  int i = ctx->prof_n++;
  ctx->prof_kind[i] = kind;
  cudaEventRecord(ctx->prof_ev[2 * i], st);
  return i;
}
void prof_end(lrdm_ctx* ctx, int i, cudaStream_t st) {
  if (i >= 0) cudaEventRecord(ctx->prof_ev[2 * i + 1], st);
}
void count(lrdm_ctx* ctx, int n) {
  if (ctx->prof_on) ctx->launches += n;
}

lrdm_status validate_system(const lrdm_system& s, const lrdm_options& o) {
  for (int d = 0; d < 3; ++d) {
    if (s.n[d] < 1) return LRDM_ERR_SHAPE;
    if (!(s.h[d] > 0.0)) return LRDM_ERR_INVALID_ARG;
  }
  if (s.nspin != 1 && s.nspin != 2) return LRDM_ERR_INVALID_ARG;
  if (!(s.kT > 0.0)) return LRDM_ERR_INVALID_ARG;
  int km = s.k_max > 0 ? s.k_max : o.k_max;
  if (km < 1 || km > KMAX_LIMIT) return LRDM_ERR_INVALID_ARG;
  for (int c = 0; c < s.nspin; ++c) {
    if (s.ns[c] < 1) return LRDM_ERR_SHAPE;
    if (s.ld_psi[c] < s.ns[c]) return LRDM_ERR_SHAPE;
    if (!s.psi[c] || !s.eps[c]) return LRDM_ERR_INVALID_ARG;
    long long ng = (long long)s.n[0] * s.n[1] * s.n[2];
    if (s.ns[c] > ng) return LRDM_ERR_SHAPE;
  }
  return LRDM_OK;
}

// Poisson: batched real <-> half-complex transforms over k_max fields, the
// symbol table and the transform buffers of system S.
lrdm_status setup_poisson(lrdm_ctx* ctx, SysState& S, cudaStream_t st) {
  const lrdm_options& o = ctx->opt;
  const int fp64 = o.prec == LRDM_FP64;
  const size_t csz = fp64 ? sizeof(double) : sizeof(float);
  const long long nc = (long long)S.n[0] * S.n[1] * (S.n[2] / 2 + 1);
  LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&S.fft_real), (size_t)S.kmax * S.Ngrid * csz));
  LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&S.fft_cplx), (size_t)S.kmax * nc * 2 * csz));
  int nn[3] = {S.n[0], S.n[1], S.n[2]};
  LRDM_FFT(cufftPlanMany(&S.plan_r2c, 3, nn, nullptr, 1, (int)S.Ngrid, nullptr, 1, (int)nc,
                         fp64 ? CUFFT_D2Z : CUFFT_R2C, S.kmax));
  S.plans = true;
  LRDM_FFT(cufftPlanMany(&S.plan_c2r, 3, nn, nullptr, 1, (int)nc, nullptr, 1, (int)S.Ngrid,
                         fp64 ? CUFFT_Z2D : CUFFT_C2R, S.kmax));
  LRDM_CK(dalloc(ctx, &S.sym, (size_t)nc, false));
  LRDM_CU(launch_poisson_table(S.n, S.h, o.poisson_symbol, S.sym, st));
  return LRDM_OK;
}

lrdm_status setup_system(lrdm_ctx* ctx, int idx, const lrdm_system& in, cudaStream_t st) {
  const lrdm_options& o = ctx->opt;
  SysState& S = ctx->sys[idx];
  const int prec = o.prec;
  const int fp64 = prec == LRDM_FP64;
  const size_t csz = fp64 ? sizeof(double) : sizeof(float);
  for (int d = 0; d < 3; ++d) {
    S.n[d] = in.n[d];
    S.h[d] = in.h[d];
  }
  S.Ngrid = (long long)in.n[0] * in.n[1] * in.n[2];
  // a row-sharded context holds rows [r0, r0 + Ng) of the grid; every
  // row-wise array (Psi copies, rho, f_x, weights, directions) has Ng rows
  S.Ng = ctx->rows ? ctx->rows_n : S.Ngrid;
  S.r0 = ctx->rows ? ctx->rows_begin : 0;
  S.Ng_pad = is_tc(prec) ? (S.Ng + TC_PAD_GRID - 1) / TC_PAD_GRID * TC_PAD_GRID : S.Ng;
  S.nspin = in.nspin;
  S.kmax = in.k_max > 0 ? in.k_max : o.k_max;
  S.w = in.h[0] * in.h[1] * in.h[2];
  S.g = in.occ_factor != 0.0 ? in.occ_factor : (in.nspin == 1 ? 2.0 : 1.0);
  S.kT = in.kT;
  S.ne = in.n_electrons;
  S.occ_given = in.occ[0] != nullptr;

  // eigenvalues (and given occupations) to the host for mu
  std::vector<std::vector<double>> eps(in.nspin), occ(in.nspin);
  for (int c = 0; c < in.nspin; ++c) {
    eps[c].resize(in.ns[c]);
    LRDM_CU(cudaMemcpy(eps[c].data(), in.eps[c], in.ns[c] * sizeof(double),
                       cudaMemcpyDeviceToHost));
    if (S.occ_given) {
      if (!in.occ[c]) return LRDM_ERR_INVALID_ARG;
      occ[c].resize(in.ns[c]);
      LRDM_CU(cudaMemcpy(occ[c].data(), in.occ[c], in.ns[c] * sizeof(double),
                         cudaMemcpyDeviceToHost));
    }
  }
  lrdm_status ms = solve_mu_host(eps, S.ne, S.kT, S.g, &S.mu);
  if (ms != LRDM_OK) {
    if (!S.occ_given) return ms;
    S.mu = 0.0;
  }
  if (!S.occ_given)
    for (int c = 0; c < in.nspin; ++c) {
      occ[c].resize(in.ns[c]);
      for (int i = 0; i < in.ns[c]; ++i) occ[c][i] = fermi_host((eps[c][i] - S.mu) / S.kT);
    }

  for (int c = 0; c < in.nspin; ++c) {
    Channel& ch = S.ch[c];
    const int ns = in.ns[c];
    ch.ns = ns;
    ch.ns_pad = is_tc(prec) ? (ns + TC_PAD_STATES - 1) / TC_PAD_STATES * TC_PAD_STATES : ns;
    LRDM_CK(dalloc(ctx, &ch.eps, ns));
    LRDM_CK(dalloc(ctx, &ch.occ, ns));
    LRDM_CU(cudaMemcpyAsync(ch.eps, eps[c].data(), ns * sizeof(double), cudaMemcpyHostToDevice, st));
    LRDM_CU(cudaMemcpyAsync(ch.occ, occ[c].data(), ns * sizeof(double), cudaMemcpyHostToDevice, st));
    LRDM_CK(dalloc(ctx, &ch.L, (size_t)ns * ns, false));
    if (o.fermi_T > 0)
      for (int i = 0; i < ns; ++i)
        if (!(fabs(eps[c][i] - S.mu) < S.kT * std::ldexp(1.0, o.fermi_T + 1)))
          return LRDM_ERR_INVALID_ARG;     // outside the recursion's monotone window
    LRDM_CU(launch_loewner(ch.eps, ch.occ, ns, S.mu, S.kT, S.occ_given ? 1 : 0, o.degen_tol,
                           o.fermi_T, ch.L, st));
    if (is_tc(prec)) {
      LRDM_CK(dalloc(ctx, &ch.Lf, (size_t)ch.ns_pad * ch.ns_pad, false));
      LRDM_CU(launch_loewner_f32(ch.L, ns, ch.ns_pad, ch.Lf, st));
    }
    // density and xc kernel
    LRDM_CK(dalloc(ctx, &ch.rho, S.Ng, false));
    if (in.rho[c]) {
      LRDM_CU(launch_copy_rho(in.rho[c], o.io_dtype, S.Ng, ch.rho, st));
    } else {
      LRDM_CU(launch_density(in.psi[c], o.io_dtype, in.ld_psi[c], S.Ng, ns, ch.occ, S.g,
                             in.rho_floor, ch.rho, st));
    }
    LRDM_CK(dalloc(ctx, &ch.fx, S.Ng, false));
    LRDM_CU(launch_fx(ch.rho, S.Ng, in.nspin == 2, ch.fx, st));
    // operand copies of Psi
    const size_t npsi = (size_t)S.Ng * ns;
    if (prec == LRDM_FP64) {
      LRDM_CK(dalloc(ctx, &ch.psi64, npsi, false));
    } else if (prec == LRDM_FP32) {
      LRDM_CK(dalloc(ctx, &ch.psi32, npsi, false));
    } else {
      const size_t npad = (size_t)S.Ng_pad * ch.ns_pad;
      if (prec == LRDM_TF32) {
        LRDM_CK(dalloc(ctx, &ch.psiR32, npad, false));
        LRDM_CK(dalloc(ctx, &ch.psiT32, npad, false));
      } else {
        LRDM_CK(dalloc(ctx, &ch.psiR_hi, npad, false));
        LRDM_CK(dalloc(ctx, &ch.psiR_lo, npad, false));
        LRDM_CK(dalloc(ctx, &ch.psiT_hi, npad, false));
        LRDM_CK(dalloc(ctx, &ch.psiT_lo, npad, false));
        LRDM_CK(dalloc(ctx, &ch.psiTf, npad, false));
      }
    }
    LRDM_CU(launch_convert_psi(in.psi[c], o.io_dtype, in.ld_psi[c], S.Ng, ns, ch, prec, S.Ng_pad, st));
  }

  // split of the grid reduction for the CUDA-core GEMM1 (enough blocks to fill
  // 152 SMs twice); the tensor-core GEMM1 reduces the whole grid per tile.
  if (!is_tc(prec)) {
    int nt = (S.ch[0].ns + SIMT_TILE - 1) / SIMT_TILE;
    long long blocks = (long long)nt * (nt + 1) / 2 * S.kmax;
    long long want = (2LL * 152 * 2 + blocks - 1) / blocks;
    long long maxsplit = S.Ng / 256 > 0 ? S.Ng / 256 : 1;
    if (want > maxsplit) want = maxsplit;
    if (want > 64) want = 64;
    // row-sharded: one partial X per rank, summed over the ranks as it is
    S.nsplit = ctx->rows ? 1 : (int)(want < 1 ? 1 : want);
  } else {
    S.nsplit = 1;
  }

  // workspaces
  const int accsz = fp64 ? 8 : 4;
  // tensor cores: the X / G buffers hold up to 8 grid-row partials of a
  // k_max-direction call while they stay within 512 MB per channel, so that
  // small subspaces (few tiles) can split their grid reduction at any K
  S.xslots = S.kmax;
  if (is_tc(prec)) {
    size_t ldmax = 0;
    for (int c = 0; c < in.nspin; ++c) ldmax = std::max(ldmax, (size_t)S.ch[c].ns_pad);
    const size_t per = (size_t)S.kmax * ldmax * ldmax * accsz;
    const size_t cap = std::min<size_t>(8, std::max<size_t>(1, (512ull << 20) / per));
    S.xslots = (int)(cap * S.kmax);
  }
  for (int c = 0; c < in.nspin; ++c) {
    Channel& ch = S.ch[c];
    const size_t ldx = is_tc(prec) ? ch.ns_pad : ch.ns;
    const size_t xcount = (size_t)S.nsplit * (is_tc(prec) ? S.xslots : S.kmax) * ldx * ldx;
    LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ch.Xpart), xcount * accsz));
    LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ch.Gpart), xcount * accsz));
    const size_t pcount = (size_t)S.kmax * ldx * ldx;
    if (prec == LRDM_BF16X3) {
      LRDM_CK(dalloc(ctx, reinterpret_cast<__nv_bfloat16**>(&ch.Xpp), pcount));
      LRDM_CK(dalloc(ctx, reinterpret_cast<__nv_bfloat16**>(&ch.Xpp_lo), pcount));
    } else {
      LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ch.Xpp), pcount * csz));
    }
  }
  LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&S.a), (size_t)S.kmax * S.nspin * S.Ng_pad * csz));
  LRDM_CK(dalloc(ctx, &S.dmu, S.kmax));
  LRDM_CK(dalloc(ctx, &S.tbar, S.kmax));

  return setup_poisson(ctx, S, st);
}

// V_H = F^-1[4 pi F[fft_real] / |G|^2] in place in S.fft_real (all k_max slots).
lrdm_status hartree_body(lrdm_ctx* ctx, SysState& S, int K, cudaStream_t st) {
  const int fp64 = ctx->opt.prec == LRDM_FP64;
  LRDM_FFT(cufftSetStream(S.plan_r2c, st));
  LRDM_FFT(cufftSetStream(S.plan_c2r, st));
  if (fp64) {
    LRDM_FFT(cufftExecD2Z(S.plan_r2c, static_cast<cufftDoubleReal*>(S.fft_real),
                          static_cast<cufftDoubleComplex*>(S.fft_cplx)));
  } else {
    LRDM_FFT(cufftExecR2C(S.plan_r2c, static_cast<cufftReal*>(S.fft_real),
                          static_cast<cufftComplex*>(S.fft_cplx)));
  }
  LRDM_CU(launch_poisson_symbol(S.fft_cplx, K, (long long)S.n[0] * S.n[1] * (S.n[2] / 2 + 1),
                                S.sym, fp64, st));
  if (fp64) {
    LRDM_FFT(cufftExecZ2D(S.plan_c2r, static_cast<cufftDoubleComplex*>(S.fft_cplx),
                          static_cast<cufftDoubleReal*>(S.fft_real)));
  } else {
    LRDM_FFT(cufftExecC2R(S.plan_c2r, static_cast<cufftComplex*>(S.fft_cplx),
                          static_cast<cufftReal*>(S.fft_real)));
  }
  return LRDM_OK;
}

lrdm_status hartree(lrdm_ctx* ctx, SysState& S, int K, cudaStream_t st) {
  NvtxRange nvtx_("poisson");
  int pi = prof_begin(ctx, 3, st);
  lrdm_status rc = hartree_body(ctx, S, K, st);
  prof_end(ctx, pi, st);
  return rc;
}

size_t io_size(int io) { return io == LRDM_DTYPE_F64 ? 8 : 4; }

// CUDA-core GEMM1 of channel c with weights S.a -> Xdst (split partials)
lrdm_status gemm1_simt(lrdm_ctx* ctx, SysState& S, int c, int K, void* Xdst, cudaStream_t st) {
  const int prec = ctx->opt.prec;
  Channel& ch = S.ch[c];
  const size_t csz = prec == LRDM_FP64 ? 8 : 4;
  const char* a = static_cast<const char*>(S.a) + (size_t)c * S.Ng_pad * csz;
  int pi = prof_begin(ctx, 1, st);
  count(ctx, 1);
  const void* psi = prec == LRDM_FP64 ? static_cast<const void*>(ch.psi64)
                                      : static_cast<const void*>(ch.psi32);
  cudaError_t e = launch_gemm1_simt(prec == LRDM_FP64, psi, ch.ns, S.Ng, a,
                                    (long long)S.nspin * S.Ng_pad, K, Xdst, S.nsplit, st);
  prof_end(ctx, pi, st);
  return from_cuda(e);
}

// CUDA-core GEMM2 of channel c: out = factor * diag(Psi X'' Psi^T) (- v)
lrdm_status gemm2_simt(lrdm_ctx* ctx, SysState& S, int c, int K, double factor, const void* v,
                       long long v_stride, void* out, long long out_stride, int out_is_io,
                       cudaStream_t st) {
  const int prec = ctx->opt.prec;
  Channel& ch = S.ch[c];
  int pi = prof_begin(ctx, 2, st);
  count(ctx, 1);
  const void* psi = prec == LRDM_FP64 ? static_cast<const void*>(ch.psi64)
                                      : static_cast<const void*>(ch.psi32);
  cudaError_t e = launch_gemm2_simt(prec == LRDM_FP64, psi, ch.ns, S.Ng, ch.Xpp, K, factor, v,
                                    v_stride, out, out_stride, ctx->opt.io_dtype, out_is_io, st);
  prof_end(ctx, pi, st);
  return from_cuda(e);
}

// One grouped tensor-core launch over the entries collected in ctx->tc_entries.
lrdm_status tc_group(lrdm_ctx* ctx, int gemm, int out_is_io, cudaStream_t st) {
  NvtxRange nvtx_("contraction (tensor cores)");
  const int n = (int)ctx->tc_entries.size();
  if (n == 0) return LRDM_OK;
  int pi = prof_begin(ctx, gemm, st);
  // test-only fault injection, once: the next projection launch times out
  const int stall = gemm == 1 && (ctx->opt.debug_flags & LRDM_DEBUG_STALL_PROJECTION) ? 1 : 0;
  if (stall) ctx->opt.debug_flags &= ~LRDM_DEBUG_STALL_PROJECTION;
  int launches = (n + TC_MAX_SLOTS - 1) / TC_MAX_SLOTS;
  cudaError_t e;
  if (gemm == 1) {
    e = launch_gemm1_tc_group(ctx->opt.prec, ctx->tc_entries.data(), n, ctx->d_status, st, ctx->tune,
                              0, stall, ctx->d_round);
  } else {
    launches = 0;
    e = launch_gemm2_tc_group(ctx->opt.prec, ctx->tc_entries.data(), n, ctx->opt.io_dtype, out_is_io,
                              ctx->d_status, st, ctx->tune, 0, &launches, ctx->d_round);
  }
  count(ctx, launches);
  prof_end(ctx, pi, st);
  return from_cuda(e);
}

// Grid-row ranges of the tensor-core GEMM1 for K directions of system s.
// The work items (tiles x directions x ranges) are of equal size, so the
// launch time follows the number of waves over the SMs: the count that fills
// the last wave best (by more than half a percent over a smaller count), with
// at most 8 ranges, nsplit * K <= the X buffer's direction slots (k_max, or
// up to 8 k_max for small subspaces) and at least 64 stages of the reduction
// per range.  1 at the
// benchmark's K = 16 (4352 items, 0.987 of 29 waves); 5 at K = 1 there
// (1360 items, 0.994 of 9 waves, against 0.895 for 1-4 ranges).
int choose_split(lrdm_ctx* ctx, int s, int K) {
  const SysState& S = ctx->sys[s];
  if (!is_tc(ctx->opt.prec) || K <= 0 || ctx->tc_pid.empty() || ctx->rows) return 1;
  const TcProblem& pr = ctx->tc_host[ctx->tc_pid[2 * s]];
  const bool pair = ctx->tune.g1_nb == G1_PAIR;
  const bool wide = ctx->tune.g1_nb == 256;
  const int dpt = wide || pair ? 1 : ctx->tune.g1_dpt;
  const long long items =
      (long long)(pair ? pr.ntiles_p : wide ? pr.ntiles_w : pr.ntiles) * ((K + dpt - 1) / dpt);
  // work units of the persistent grid: SMs, or CTA pairs for the pair tiles
  const long long sms = pair ? tc_pair_units(ctx->opt.prec) : ctx->sm_count > 0 ? ctx->sm_count : 148;
  int smax = S.xslots / K;
  if (smax > 8) smax = 8;
  if (smax > pr.nch / 64) smax = pr.nch / 64;
  int best = 1;
  double best_fill = 0.0;
  for (int sp = 1; sp <= smax; ++sp) {
    const long long n = items * sp;
    const double fill = (double)n / (double)(((n + sms - 1) / sms) * sms);
    if (fill > best_fill + 0.005) {
      best_fill = fill;
      best = sp;
    }
  }
  return best;
}

TcEntry tc_entry(lrdm_ctx* ctx, int s, int c, int K) {
  TcEntry x;
  const int pid = ctx->tc_pid[2 * s + c];
  x.dev_base = ctx->tc_dev;
  x.host = &ctx->tc_host[pid];
  x.pid = pid;
  x.K = K;
  return x;
}

// ---------------------------------------------------------------------------
// autotuner: launch shape of the tensor-core contractions
// ---------------------------------------------------------------------------

// Identifies the problem set (device, precision, every (N_g, N_s padded, k_max)).
std::string tune_key(lrdm_ctx* ctx) {
  int dev = 0, sms = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  std::string k = "sm" + std::to_string(major) + std::to_string(minor) + "x" + std::to_string(sms) +
                  ";prec" + std::to_string(ctx->opt.prec);
  if (ctx->kp) {                      // one stacked problem per k-point
    for (const Channel& c : ctx->kp_ch)
      k += ";kp" + std::to_string(ctx->sys[0].Ng) + "," + std::to_string(c.ns_pad) + "," +
           std::to_string(ctx->sys[0].kmax);
    return k;
  }
  for (int s = 0; s < ctx->nsys; ++s)
    for (int c = 0; c < ctx->sys[s].nspin; ++c)
      k += ";" + std::to_string(ctx->sys[s].Ng) + "," + std::to_string(ctx->sys[s].ch[c].ns_pad) +
           "," + std::to_string(ctx->sys[s].kmax);
  return k;
}

// Cache file: one JSON object per line,
//   {"key": "...", "g1_nb": 256, "g1_dpt": 1, "g2_bn": 256, "g2_kgroup": 4}
bool tune_cache_read(const char* path, const std::string& key, TcTune& t) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[4096];
  const std::string want = "\"key\": \"" + key + "\"";
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    if (!strstr(line, want.c_str())) continue;
    const char* z = strstr(line, "\"g1_nb\":");
    const char* a = strstr(line, "\"g1_dpt\":");
    const char* b = strstr(line, "\"g2_bn\":");
    const char* c = strstr(line, "\"g2_kgroup\":");
    TcTune u;
    if (z && a && b && c && sscanf(z, "\"g1_nb\": %d", &u.g1_nb) == 1 &&
        (u.g1_nb == 128 || u.g1_nb == 256 || u.g1_nb == G1_PAIR) &&
        sscanf(a, "\"g1_dpt\": %d", &u.g1_dpt) == 1 &&
        sscanf(b, "\"g2_bn\": %d", &u.g2_bn) == 1 &&
        sscanf(c, "\"g2_kgroup\": %d", &u.g2_kgroup) == 1 && (u.g1_dpt == 1 || u.g1_dpt == 2) &&
        (u.g2_bn == 128 || u.g2_bn == 256 || u.g2_bn == G2_PAIR) &&
        (u.g2_kgroup == 1 || u.g2_kgroup == 2 || u.g2_kgroup == 4)) {
      t = u;
      found = true;                  // the last matching line wins
    }
  }
  fclose(f);
  return found;
}

void tune_cache_append(const char* path, const std::string& key, const TcTune& t) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"g1_nb\": %d, \"g1_dpt\": %d, \"g2_bn\": %d, \"g2_kgroup\": %d}\n",
          key.c_str(), t.g1_nb, t.g1_dpt, t.g2_bn, t.g2_kgroup);
  fclose(f);
}

// Minimum over `reps` timed launches (after one untimed) of a launch function.
template <typename F>
float time_launch(F&& launch, cudaStream_t st, int reps, cudaError_t& err) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  err = launch();
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    cudaEventRecord(e0, st);
    err = launch();
    cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// Times the candidate launch shapes on this context's own problems (K = each
// system's k_max, reductions capped so that the whole search takes about a
// second at the largest sizes) and keeps the fastest.  The buffers written
// (X, the GEMM1 weights scratch) are overwritten by every later call.
lrdm_status autotune(lrdm_ctx* ctx, cudaStream_t st) {
  constexpr int G1_NCH_CAP = 256, G2_NR_CAP = 608, REPS = 3;
  const char* cache = getenv("LRDM_TUNE_CACHE");
  const std::string key = tune_key(ctx);
  if (cache && *cache && tune_cache_read(cache, key, ctx->tune)) return LRDM_OK;
  std::vector<TcEntry> g1, g2;
  std::vector<int> g1_sys;                             // system of each projection entry (-1: k-point)
  for (size_t q = 0; q < ctx->kp_ch.size(); ++q) {     // k-point context: the stacked problems
    SysState& S = ctx->sys[0];
    TcEntry x;
    x.dev_base = ctx->tc_dev;
    x.pid = ctx->kp_pid[q];
    x.host = &ctx->tc_host[x.pid];
    x.K = S.kmax;
    x.X = ctx->kp_ch[q].Xpart;
    g1.push_back(x);
    g1_sys.push_back(-1);
    x.X = nullptr;
    x.factor = 1.0;
    x.out = ctx->kp_out[q];
    x.out_stride = S.Ng;
    g2.push_back(x);
  }
  for (int s = 0; s < ctx->nsys && !ctx->kp; ++s) {
    SysState& S = ctx->sys[s];
    for (int c = 0; c < S.nspin; ++c) {
      TcEntry x = tc_entry(ctx, s, c, S.kmax);
      x.X = S.ch[c].Xpart;
      g1.push_back(x);
      g1_sys.push_back(s);
      TcEntry y = tc_entry(ctx, s, c, S.kmax);
      y.factor = 1.0;
      y.out = static_cast<float*>(S.a) + (size_t)c * S.Ng_pad;
      y.out_stride = (long long)S.nspin * S.Ng_pad;
      g2.push_back(y);
    }
  }
  cudaError_t err = cudaSuccess;
  TcTune best = ctx->tune;
  float tbest = 1e30f;
  const int g1_cand[4][2] = {{G1_PAIR, 1}, {256, 1}, {128, 1}, {128, 2}};   // (MMA width, directions per tile)
  const TcTune start = ctx->tune;
  for (const auto& c : g1_cand) {
    TcTune t = start;
    t.g1_nb = c[0];
    t.g1_dpt = c[1];
    // each candidate runs with the row-range split a call of k_max directions
    // would take in that shape (the split fills the last wave differently
    // for each tile shape)
    ctx->tune = t;
    for (size_t e = 0; e < g1.size(); ++e)
      if (g1_sys[e] >= 0) g1[e].split = choose_split(ctx, g1_sys[e], g1[e].K);
    ctx->tune = start;
    const float ms = time_launch([&] { return launch_gemm1_tc_group(ctx->opt.prec, g1.data(), (int)g1.size(),
                                                                    ctx->d_status, st, t, G1_NCH_CAP, 0,
                                                                    ctx->d_round); },
                                 st, REPS, err);
    if (err != cudaSuccess) return from_cuda(err);
    if (ms < tbest) { tbest = ms; best.g1_nb = c[0]; best.g1_dpt = c[1]; }
  }
  tbest = 1e30f;
  for (int bn = 128; bn <= G2_PAIR; bn *= 2)          // 128, 256, and 256 on CTA pairs
    for (int kg = 1; kg <= 4; kg *= 2) {
      TcTune t = ctx->tune;
      t.g2_bn = bn;
      t.g2_kgroup = kg;
      const float ms = time_launch([&] { return launch_gemm2_tc_group(ctx->opt.prec, g2.data(), (int)g2.size(),
                                                                      LRDM_DTYPE_F32, 0, ctx->d_status, st, t,
                                                                      G2_NR_CAP, nullptr, ctx->d_round); },
                                   st, REPS, err);
      if (err != cudaSuccess) return from_cuda(err);
      if (ms < tbest) { tbest = ms; best.g2_bn = bn; best.g2_kgroup = kg; }
    }
  ctx->tune = best;
  if (cache && *cache) tune_cache_append(cache, key, best);
  return LRDM_OK;
}

// The forward path of all systems: potentials and weights per system, then
// one projection contraction over every (system, channel), mu' and the
// Loewner scaling, then one response contraction over every (system, channel).
// The caller's sum over the ranks of a row-sharded context (a no-op otherwise).
lrdm_status allreduce(lrdm_ctx* ctx, void* buf, long long count, int dtype, cudaStream_t st) {
  if (!ctx->rows || count == 0) return LRDM_OK;
  return ctx->ar.fn(ctx->ar.user, buf, count, dtype, st) == 0 ? LRDM_OK : LRDM_ERR_COLLECTIVE;
}

// The K full-grid Poisson inputs of system S: `write(at, stride)` writes this
// context's rows of field k at at + k * stride.  A row-sharded context writes
// its rows into the zeroed full-grid buffer and sums it over the ranks.
template <typename W>
lrdm_status gather_fields(lrdm_ctx* ctx, SysState& S, int K, cudaStream_t st, W&& write) {
  const int fp64 = ctx->opt.prec == LRDM_FP64;
  const size_t csz = fp64 ? sizeof(double) : sizeof(float);
  if (ctx->rows) LRDM_CU(cudaMemsetAsync(S.fft_real, 0, (size_t)K * S.Ngrid * csz, st));
  LRDM_CU(write(static_cast<char*>(S.fft_real) + S.r0 * csz, S.Ngrid));
  return allreduce(ctx, S.fft_real, (long long)K * S.Ngrid, fp64 ? LRDM_DTYPE_F64 : LRDM_DTYPE_F32, st);
}

// Row-sharded context: the projections of the slabs (X, or Gbar in the
// adjoint) summed over the ranks; the buffers hold nsplit = 1 partials.
lrdm_status reduce_projections(lrdm_ctx* ctx, const int* K, bool adjoint, cudaStream_t st) {
  if (!ctx->rows) return LRDM_OK;
  const int fp64 = ctx->opt.prec == LRDM_FP64;
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    if (K[s] == 0) continue;
    for (int c = 0; c < S.nspin; ++c) {
      const long long ld = is_tc(ctx->opt.prec) ? S.ch[c].ns_pad : S.ch[c].ns;
      void* buf = adjoint ? S.ch[c].Gpart : S.ch[c].Xpart;
      LRDM_CK(allreduce(ctx, buf, (long long)S.nsplit * K[s] * ld * ld,
                        fp64 ? LRDM_DTYPE_F64 : LRDM_DTYPE_F32, st));
    }
  }
  return LRDM_OK;
}

lrdm_status forward_all(lrdm_ctx* ctx, const void* const* v, const int* K, void* const* f,
                        double* dmu_out, cudaStream_t st) {
  const int prec = ctx->opt.prec;
  const int fp64 = prec == LRDM_FP64;
  const int io = ctx->opt.io_dtype;
  const size_t isz = io_size(io);
  const bool tc = is_tc(prec);
  const size_t csz = fp64 ? sizeof(double) : sizeof(float);
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    S.last_K = K[s];
    if (K[s] == 0) continue;
    LRDM_CK(gather_fields(ctx, S, K[s], st, [&](void* at, long long stride) {
      return launch_spin_sum(v[s], io, K[s], S.nspin, S.Ng, at, fp64, st, stride);
    }));
    LRDM_CK(hartree(ctx, S, K[s], st));
    LRDM_CU(launch_dv_weights(v[s], io, static_cast<char*>(S.fft_real) + S.r0 * csz, S.ch[0].fx,
                              S.ch[S.nspin - 1].fx, K[s], S.nspin, S.Ng, S.Ng_pad, S.w, S.a, fp64, st,
                              S.Ngrid));
    count(ctx, 3);
  }
  // projection X_k = Psi^T diag(w dV_k) Psi
  if (tc) {
    ctx->tc_entries.clear();
    for (int s = 0; s < ctx->nsys; ++s) {
      if (K[s] > 0) ctx->sys[s].nsplit = choose_split(ctx, s, K[s]);
      for (int c = 0; c < ctx->sys[s].nspin && K[s] > 0; ++c) {
        TcEntry x = tc_entry(ctx, s, c, K[s]);
        x.X = ctx->sys[s].ch[c].Xpart;
        x.split = ctx->sys[s].nsplit;
        ctx->tc_entries.push_back(x);
      }
    }
    LRDM_CK(tc_group(ctx, 1, 0, st));
  } else {
    for (int s = 0; s < ctx->nsys; ++s)
      for (int c = 0; c < ctx->sys[s].nspin && K[s] > 0; ++c)
        LRDM_CK(gemm1_simt(ctx, ctx->sys[s], c, K[s], ctx->sys[s].ch[c].Xpart, st));
  }
  LRDM_CK(reduce_projections(ctx, K, false, st));
  // mu' and the Loewner scaling
  int off = 0;
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    if (K[s] > 0) {
      const void* X[2] = {S.ch[0].Xpart, S.ch[S.nspin - 1].Xpart};
      LRDM_CU(launch_dmu(S, X, K[s], fp64, S.dmu, dmu_out ? dmu_out + off : nullptr, ctx->d_status, st));
      for (int c = 0; c < S.nspin; ++c)
        LRDM_CU(launch_loewner_scale(S, c, S.ch[c].Xpart, K[s], fp64, S.dmu, 0, 0.0, prec, st));
      count(ctx, 1 + S.nspin);
    }
    off += K[s];
  }
  // response drho_k and f_k = drho_k - v_k
  if (tc) ctx->tc_entries.clear();
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    for (int c = 0; c < S.nspin && K[s] > 0; ++c) {
      const void* vc = static_cast<const char*>(v[s]) + (size_t)c * S.Ng * isz;
      void* fc = static_cast<char*>(f[s]) + (size_t)c * S.Ng * isz;
      const long long stride = (long long)S.nspin * S.Ng;
      if (tc) {
        TcEntry x = tc_entry(ctx, s, c, K[s]);
        x.factor = S.g;
        x.v = vc;
        x.v_stride = stride;
        x.out = fc;
        x.out_stride = stride;
        ctx->tc_entries.push_back(x);
      } else {
        LRDM_CK(gemm2_simt(ctx, S, c, K[s], S.g, vc, stride, fc, stride, 1, st));
      }
    }
  }
  if (tc) LRDM_CK(tc_group(ctx, 2, 1, st));
  return LRDM_OK;
}

// CUDA graph of a forward call: captured on the first call with a given key
// (buffers, K's, stream), replayed afterwards.  Not used on the legacy
// default stream or while profiling.
bool use_graph(const lrdm_ctx* ctx, cudaStream_t st) {
  return ctx->opt.use_graph && st != nullptr && !ctx->prof_on && !ctx->rows;
}

// One forward call of the direction drivers (Krylov step, LRDMA): system sys
// gets K[sys] directions, the others none; a Brillouin-zone-sampled context
// runs its own forward (one system, one channel).
lrdm_status forward_one(lrdm_ctx* ctx, int sys, const void* const* v, const int* K, void* const* f,
                        cudaStream_t st) {
  if (ctx->kp) {
    ctx->sys[0].last_K = K[sys];
    return K[sys] > 0 ? kp_forward(ctx, v[sys], K[sys], f[sys], nullptr, st) : LRDM_OK;
  }
  return forward_all(ctx, v, K, f, nullptr, st);
}

void free_ctx(lrdm_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    if (S.plan_r2c) cufftDestroy(S.plan_r2c);
    if (S.plan_c2r) cufftDestroy(S.plan_c2r);
  }
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  for (void* p : ctx->allocs) cudaFree(p);
  delete[] ctx->sys;
  delete ctx;
}

}  // namespace api
}  // namespace lrdm

extern "C" {

void lrdm_default_options(lrdm_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->prec = LRDM_BF16X3;
  o->io_dtype = LRDM_DTYPE_F32;
  o->k_max = 16;
  o->pinv_rcond = 1e-12;
  o->degen_tol = 1e-5;
  o->poisson_symbol = 0;
  o->use_graph = 0;
  o->autotune = 0;
  o->debug_flags = 0;
}

const char* lrdm_status_string(lrdm_status s) {
  switch (s) {
    case LRDM_OK: return "ok";
    case LRDM_ERR_INVALID_ARG: return "invalid argument";
    case LRDM_ERR_SHAPE: return "inconsistent shape";
    case LRDM_ERR_OOM: return "out of device memory";
    case LRDM_ERR_CUDA: return "CUDA error";
    case LRDM_ERR_MU_NOT_CONVERGED: return "chemical potential not found";
    case LRDM_ERR_SINGULAR: return "singular least-squares matrix (pseudo-inverse used)";
    case LRDM_ERR_TIMEOUT: return "bounded device wait expired";
    case LRDM_ERR_NONFINITE: return "non-finite value on the device";
    case LRDM_ERR_UNSUPPORTED: return "unsupported precision or feature";
  }
  return "unknown status";
}

namespace {
lrdm_status create_ctx(lrdm_ctx** out, const lrdm_system* sys, int nsys, const lrdm_options* opt,
                       void* stream, const lrdm_rows* rows) {
  if (!out) return LRDM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!sys || nsys < 1) return LRDM_ERR_INVALID_ARG;
  lrdm_options o;
  if (opt) o = *opt;
  else lrdm_default_options(&o);
  if (o.prec < LRDM_FP64 || o.prec > LRDM_BF16X3) return LRDM_ERR_INVALID_ARG;
  if (o.io_dtype != LRDM_DTYPE_F64 && o.io_dtype != LRDM_DTYPE_F32) return LRDM_ERR_INVALID_ARG;
  if (o.k_max < 1 || o.k_max > KMAX_LIMIT) return LRDM_ERR_INVALID_ARG;
  if (!(o.pinv_rcond >= 0.0)) return LRDM_ERR_INVALID_ARG;
  if (!(o.degen_tol >= 0.0)) return LRDM_ERR_INVALID_ARG;
  if (o.poisson_symbol != 0 && o.poisson_symbol != 1) return LRDM_ERR_INVALID_ARG;
  if (o.fermi_T < 0 || o.fermi_T > 30) return LRDM_ERR_INVALID_ARG;
  if (o.fermi_T > 0)
    for (int s = 0; s < nsys; ++s)
      if (sys[s].occ[0]) return LRDM_ERR_INVALID_ARG;
  for (int s = 0; s < nsys; ++s) LRDM_CK(validate_system(sys[s], o));
  if (is_tc(o.prec) && !tc_supported()) return LRDM_ERR_UNSUPPORTED;

  lrdm_ctx* ctx = new (std::nothrow) lrdm_ctx();
  if (!ctx) return LRDM_ERR_OOM;
  ctx->nsys = nsys;
  ctx->opt = o;
  if (rows) {
    ctx->rows = true;
    ctx->rows_begin = rows->row_begin;
    ctx->rows_n = rows->n_rows;
    ctx->ar.fn = rows->allreduce;
    ctx->ar.user = rows->user;
  }
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  ctx->sys = new (std::nothrow) SysState[nsys];
  if (!ctx->sys) {
    delete ctx;
    return LRDM_ERR_OOM;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lrdm_status rc = LRDM_OK;
  do {
    if ((rc = dalloc(ctx, &ctx->d_status, 1)) != LRDM_OK) break;
    if ((rc = dalloc(ctx, &ctx->d_round, 1)) != LRDM_OK) break;
    const int maxval = KMAX_LIMIT * (KMAX_LIMIT + 1) / 2 + KMAX_LIMIT + 1;
    if ((rc = dalloc(ctx, &ctx->ls_partial, (size_t)LS_BLOCKS * maxval)) != LRDM_OK) break;
    if ((rc = dalloc(ctx, &ctx->ls_coef, KMAX_LIMIT)) != LRDM_OK) break;
    if ((rc = dalloc(ctx, &ctx->ls_scal, 4)) != LRDM_OK) break;
    if ((rc = dalloc(ctx, &ctx->upd_partial, UPD_BLOCKS)) != LRDM_OK) break;
    if ((rc = dalloc(ctx, &ctx->gs_scratch, gram_schmidt_scratch())) != LRDM_OK) break;
    if ((rc = dalloc(ctx, &ctx->gs_norm, 1)) != LRDM_OK) break;
    ctx->inv_trace.resize(nsys);
    for (int s = 0; s < nsys && rc == LRDM_OK; ++s) {
      rc = setup_system(ctx, s, sys[s], st);
      if (rc != LRDM_OK) break;
      // 1 / sum_s sum_i L_ii with L_ii = -f_i (1 - f_i)/kT
      double tr = 0.0;
      SysState& S = ctx->sys[s];
      // sum of the diagonal of L as the device holds it (the same entries the
      // forward's mu' uses), whichever Fermi operator L describes
      for (int c = 0; c < S.nspin; ++c) {
        const int ns = S.ch[c].ns;
        std::vector<double> diag(ns);
        if (cudaMemcpy2DAsync(diag.data(), sizeof(double), S.ch[c].L, (size_t)(ns + 1) * sizeof(double),
                              sizeof(double), ns, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          rc = LRDM_ERR_CUDA;
          break;
        }
        for (double l : diag) tr += l;
      }
      ctx->inv_trace[s] = tr != 0.0 ? 1.0 / tr : 0.0;
    }
    if (rc != LRDM_OK) break;
    if (is_tc(o.prec)) {
      ctx->tc_pid.assign(2 * nsys, -1);
      for (int s = 0; s < nsys && rc == LRDM_OK; ++s)
        for (int c = 0; c < ctx->sys[s].nspin; ++c) {
          TcProblem pr;
          if (!build_tc_problem(o.prec, ctx->sys[s].ch[c], ctx->sys[s], c, pr)) {
            rc = LRDM_ERR_CUDA;
            break;
          }
          if ((rc = dalloc(ctx, &pr.part, (size_t)G2_MAX_SPLIT * ctx->sys[s].Ng)) != LRDM_OK) break;
          ctx->tc_pid[2 * s + c] = (int)ctx->tc_host.size();
          ctx->tc_host.push_back(pr);
        }
      if (rc != LRDM_OK) break;
      if ((rc = dalloc(ctx, reinterpret_cast<char**>(&ctx->tc_dev),
                       ctx->tc_host.size() * sizeof(TcProblem), false)) != LRDM_OK)
        break;
      if (cudaMemcpy(ctx->tc_dev, ctx->tc_host.data(), ctx->tc_host.size() * sizeof(TcProblem),
                     cudaMemcpyHostToDevice) != cudaSuccess) {
        rc = LRDM_ERR_CUDA;
        break;
      }
      ctx->tc_entries.reserve(2 * nsys);
      if (o.autotune && (rc = autotune(ctx, st)) != LRDM_OK) break;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = LRDM_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) rc = LRDM_ERR_CUDA;
  } while (0);
  if (rc != LRDM_OK) {
    free_ctx(ctx);
    return rc;
  }
  *out = ctx;
  return LRDM_OK;
}
}  // namespace

lrdm_status lrdm_create(lrdm_ctx** out, const lrdm_system* sys, int nsys,
                        const lrdm_options* opt, void* stream) {
  NvtxRange nvtx_("lrdm_create");
  return create_ctx(out, sys, nsys, opt, stream, nullptr);
}

lrdm_status lrdm_create_rows(lrdm_ctx** out, const lrdm_system* sys, const lrdm_rows* rows,
                             const lrdm_options* opt, void* stream) {
  NvtxRange nvtx_("lrdm_create_rows");
  if (!out) return LRDM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!sys || !rows || !rows->allreduce) return LRDM_ERR_INVALID_ARG;
  const long long ng = (long long)sys->n[0] * sys->n[1] * sys->n[2];
  if (rows->row_begin < 0 || rows->n_rows < 1 || rows->row_begin + rows->n_rows > ng)
    return LRDM_ERR_SHAPE;
  return create_ctx(out, sys, 1, opt, stream, rows);
}

lrdm_status lrdm_gateaux_batch(lrdm_ctx* ctx, const void* const* v, const int* K,
                               void* const* f_out, double* dmu_out, void* stream) {
  NvtxRange nvtx_("lrdm_gateaux_batch");
  if (ctx && ctx->kp) return LRDM_ERR_UNSUPPORTED;
  if (!ctx || !v || !K || !f_out) return LRDM_ERR_INVALID_ARG;
  for (int s = 0; s < ctx->nsys; ++s) {
    if (K[s] < 0 || K[s] > ctx->sys[s].kmax) return LRDM_ERR_INVALID_ARG;
    if (K[s] > 0 && (!v[s] || !f_out[s])) return LRDM_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (use_graph(ctx, st)) {
    std::vector<const void*> key;
    key.reserve(3 * ctx->nsys + 2);
    for (int s = 0; s < ctx->nsys; ++s) {
      key.push_back(v[s]);
      key.push_back(f_out[s]);
      key.push_back(reinterpret_cast<const void*>((intptr_t)K[s]));
      ctx->sys[s].last_K = K[s];
    }
    key.push_back(dmu_out);
    key.push_back(st);
    return graph_call(ctx, key, st, [&] { return forward_all(ctx, v, K, f_out, dmu_out, st); });
  }
  return forward_all(ctx, v, K, f_out, dmu_out, st);
}

lrdm_status lrdm_apply(lrdm_ctx* ctx, int sys, const void* R, const void* v, const void* f, int K,
                       double alpha, void* rho_inout, double* coeff_out, double* s_rel_out,
                       void* stream) {
  NvtxRange nvtx_("lrdm_apply");
  if (!ctx || sys < 0 || sys >= ctx->nsys || !R || !v || !f) return LRDM_ERR_INVALID_ARG;
  if (K < 1 || K > KMAX_LIMIT) return LRDM_ERR_INVALID_ARG;
  if (!isfinite(alpha)) return LRDM_ERR_INVALID_ARG;
  SysState& S = ctx->sys[sys];
  long long n = (long long)S.nspin * S.Ng;
  count(ctx, 4);
  int ar_failed = 0;
  const lrdm_status rc = from_cuda(launch_ls(R, v, f, ctx->opt.io_dtype, K, n, S.w, alpha,
                                             ctx->opt.pinv_rcond, rho_inout, ctx->ls_coef, coeff_out,
                                             s_rel_out, ctx->ls_partial, ctx->ls_scal, ctx->upd_partial,
                                             ctx->d_status, static_cast<cudaStream_t>(stream),
                                             ctx->rows ? &ctx->ar : nullptr, &ar_failed));
  return ar_failed ? LRDM_ERR_COLLECTIVE : rc;
}

lrdm_status lrdm_krylov_step(lrdm_ctx* ctx, int sys, const void* R, double s_tol, int r_max,
                             double alpha, void* rho_inout, void* U, void* T, double* coeff_out,
                             double* s_rel_out, int* rank_out, double* r_norm_out, void* stream) {
  NvtxRange nvtx_("lrdm_krylov_step");
  if (!ctx || sys < 0 || sys >= ctx->nsys || !R || !U || !T) return LRDM_ERR_INVALID_ARG;
  if (r_max < 1 || r_max > KMAX_LIMIT || !(s_tol >= 0.0) || !isfinite(alpha)) return LRDM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SysState& S = ctx->sys[sys];
  const int io = ctx->opt.io_dtype;
  const long long n = (long long)S.nspin * S.Ng;
  const size_t vb = (size_t)n * io_size(io);
  // row-sharded: every grid sum of the step is summed over the ranks
  const AllReduce* ar = ctx->rows ? &ctx->ar : nullptr;
  int ar_failed = 0;
  // u_1 = R / ||R||
  LRDM_CU(launch_gram_schmidt(nullptr, 0, R, io, n, S.w, U, ctx->gs_scratch, ctx->gs_norm, st, ar,
                              &ar_failed));
  if (ar_failed) return LRDM_ERR_COLLECTIVE;
  count(ctx, 2);
  double r_norm = 0.0;
  LRDM_CU(cudaMemcpyAsync(&r_norm, ctx->gs_norm, sizeof(double), cudaMemcpyDeviceToHost, st));
  LRDM_CU(cudaStreamSynchronize(st));
  if (!(r_norm > 0.0) || !isfinite(r_norm)) return LRDM_ERR_INVALID_ARG;
  if (r_norm_out) *r_norm_out = r_norm;
  std::vector<const void*> v(ctx->nsys, nullptr);
  std::vector<void*> f(ctx->nsys, nullptr);
  std::vector<int> K(ctx->nsys, 0);
  int rank = 0;
  for (int i = 0; i < r_max; ++i) {
    // t_i = d/dlam R[rho + lam u_i]
    v[sys] = static_cast<const char*>(U) + i * vb;
    f[sys] = static_cast<char*>(T) + i * vb;
    K[sys] = 1;
    LRDM_CK(forward_one(ctx, sys, v.data(), K.data(), f.data(), st));
    rank = i + 1;
    // least squares on the first i + 1 directions (no update yet) -> s_rel
    LRDM_CU(launch_ls(R, U, T, io, rank, n, S.w, 0.0, ctx->opt.pinv_rcond, nullptr, ctx->ls_coef,
                      coeff_out, nullptr, ctx->ls_partial, ctx->ls_scal, ctx->upd_partial,
                      ctx->d_status, st, ar, &ar_failed));
    if (ar_failed) return LRDM_ERR_COLLECTIVE;
    count(ctx, 4);
    double s_rel = 0.0;
    LRDM_CU(cudaMemcpyAsync(&s_rel, ctx->ls_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    LRDM_CU(cudaStreamSynchronize(st));
    if (s_rel_out) s_rel_out[i] = s_rel;
    if (s_rel < s_tol || rank == r_max) break;
    // u_{i+1} = t_i - sum_k <t_i, u_k> u_k, normalised
    LRDM_CU(launch_gram_schmidt(U, rank, static_cast<const char*>(T) + i * vb, io, n, S.w,
                                static_cast<char*>(U) + rank * vb, ctx->gs_scratch, ctx->gs_norm, st,
                                ar, &ar_failed));
    if (ar_failed) return LRDM_ERR_COLLECTIVE;
    count(ctx, 3);
  }
  if (rank_out) *rank_out = rank;
  if (rho_inout) {
    const double a = alpha < 0.0 ? (r_norm < 2.0 ? 0.5 : 0.1) : alpha;
    LRDM_CU(launch_ls(R, U, T, io, rank, n, S.w, a, ctx->opt.pinv_rcond, rho_inout, ctx->ls_coef,
                      coeff_out, nullptr, ctx->ls_partial, ctx->ls_scal, ctx->upd_partial,
                      ctx->d_status, st, ar, &ar_failed));
    if (ar_failed) return LRDM_ERR_COLLECTIVE;
    count(ctx, 4);
  }
  return LRDM_OK;
}

lrdm_status lrdm_apply_static(const void* R, const void* v, const void* f, int io_dtype, int K,
                              long long n, double w, double alpha, double pinv_rcond,
                              void* rho_inout, double* coeff_out, double* s_rel_out,
                              int* status_out, void* stream) {
  if (!R || !v || !f) return LRDM_ERR_INVALID_ARG;
  if (io_dtype != LRDM_DTYPE_F64 && io_dtype != LRDM_DTYPE_F32) return LRDM_ERR_INVALID_ARG;
  if (K < 1 || K > static_k_max()) return LRDM_ERR_INVALID_ARG;
  if (n < 1 || !(w > 0.0) || !isfinite(alpha) || !(pinv_rcond >= 0.0)) return LRDM_ERR_INVALID_ARG;
  return from_cuda(launch_ls_static(R, v, f, io_dtype, K, n, w, alpha, pinv_rcond, rho_inout,
                                    coeff_out, s_rel_out, status_out,
                                    static_cast<cudaStream_t>(stream)));
}

lrdm_status lrdm_backward(lrdm_ctx* ctx, const void* const* f_bar, void* const* v_bar,
                          double* const* eps_bar, double* const* occ_bar, void* stream) {
  NvtxRange nvtx_("lrdm_backward");
  if (!ctx || !f_bar || !v_bar) return LRDM_ERR_INVALID_ARG;
  if (ctx->kp) return kp_backward(ctx, f_bar, v_bar, eps_bar, occ_bar, static_cast<cudaStream_t>(stream));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int prec = ctx->opt.prec;
  const int fp64 = prec == LRDM_FP64;
  const int io = ctx->opt.io_dtype;
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    if (S.last_K < 0) return LRDM_ERR_INVALID_ARG;   // no forward call yet
    if (S.last_K > 0 && (!f_bar[s] || !v_bar[s])) return LRDM_ERR_INVALID_ARG;
    if (ctx->opt.fermi_T > 0)
      for (int c = 0; c < S.nspin; ++c)
        if ((eps_bar && eps_bar[2 * s + c]) || (occ_bar && occ_bar[2 * s + c]))
          return LRDM_ERR_UNSUPPORTED;
  }
  const bool tc = is_tc(prec);
  const size_t csz = fp64 ? 8 : 4;
  // Gbar_k = g Psi^T diag(fbar_k) Psi
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    if (S.last_K > 0) {
      LRDM_CU(launch_scale_weights(f_bar[s], io, S.last_K, S.nspin, S.Ng, S.Ng_pad, S.g, S.a, fp64, st));
      count(ctx, 1);
    }
  }
  if (tc) {
    ctx->tc_entries.clear();
    for (int s = 0; s < ctx->nsys; ++s) {
      // the same ranges as the forward call (the adjoint reduction reads X and Gbar together)
      if (ctx->sys[s].last_K > 0) ctx->sys[s].nsplit = choose_split(ctx, s, ctx->sys[s].last_K);
      for (int c = 0; c < ctx->sys[s].nspin && ctx->sys[s].last_K > 0; ++c) {
        TcEntry x = tc_entry(ctx, s, c, ctx->sys[s].last_K);
        x.X = ctx->sys[s].ch[c].Gpart;
        x.split = ctx->sys[s].nsplit;
        ctx->tc_entries.push_back(x);
      }
    }
    LRDM_CK(tc_group(ctx, 1, 0, st));
  } else {
    for (int s = 0; s < ctx->nsys; ++s)
      for (int c = 0; c < ctx->sys[s].nspin && ctx->sys[s].last_K > 0; ++c)
        LRDM_CK(gemm1_simt(ctx, ctx->sys[s], c, ctx->sys[s].last_K, ctx->sys[s].ch[c].Gpart, st));
  }
  if (ctx->rows) {
    std::vector<int> Ks(ctx->nsys);
    for (int s = 0; s < ctx->nsys; ++s) Ks[s] = ctx->sys[s].last_K;
    LRDM_CK(reduce_projections(ctx, Ks.data(), true, st));
  }
  // Ybar = L o Gbar - diag(L) T / sum L;  dVbar = w diag(Psi Ybar Psi^T) into S.a
  if (tc) ctx->tc_entries.clear();
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    const int K = S.last_K;
    if (K == 0) continue;
    const double inv_tr = ctx->inv_trace[s];
    const void* G[2] = {S.ch[0].Gpart, S.ch[S.nspin - 1].Gpart};
    LRDM_CU(launch_trace_bar(S, G, K, fp64, S.tbar, st));
    count(ctx, 1 + S.nspin);
    for (int c = 0; c < S.nspin; ++c) {
      LRDM_CU(launch_loewner_scale(S, c, S.ch[c].Gpart, K, fp64, S.tbar, 1, inv_tr, prec, st));
      void* out = static_cast<char*>(S.a) + (size_t)c * S.Ng_pad * csz;
      const long long stride = (long long)S.nspin * S.Ng_pad;
      if (tc) {
        TcEntry x = tc_entry(ctx, s, c, K);
        x.factor = S.w;
        x.out = out;
        x.out_stride = stride;
        ctx->tc_entries.push_back(x);
      } else {
        LRDM_CK(gemm2_simt(ctx, S, c, K, S.w, nullptr, 0, out, stride, 0, st));
      }
    }
  }
  if (tc) LRDM_CK(tc_group(ctx, 2, 0, st));
  // vbar = V_H[sum_s dVbar] + f_x dVbar - fbar;  eps_bar, occ_bar
  for (int s = 0; s < ctx->nsys; ++s) {
    SysState& S = ctx->sys[s];
    const int K = S.last_K;
    const double inv_tr = ctx->inv_trace[s];
    if (K > 0) {
      LRDM_CK(gather_fields(ctx, S, K, st, [&](void* at, long long stride) {
        return launch_spin_sum_padded(S.a, K, S.nspin, S.Ng, S.Ng_pad, at, fp64, st, stride);
      }));
      LRDM_CK(hartree(ctx, S, K, st));
      LRDM_CU(launch_adjoint_potential(S.a, static_cast<char*>(S.fft_real) + S.r0 * csz, S.ch[0].fx,
                                       S.ch[S.nspin - 1].fx, f_bar[s], io, K, S.nspin, S.Ng,
                                       S.Ng_pad, v_bar[s], fp64, st, S.Ngrid));
      count(ctx, 3);
    }
    for (int c = 0; c < S.nspin; ++c) {
      double* eb = eps_bar ? eps_bar[2 * s + c] : nullptr;
      double* ob = occ_bar ? occ_bar[2 * s + c] : nullptr;
      if (!eb && !ob) continue;
      if (K == 0) {
        if (eb) LRDM_CU(cudaMemsetAsync(eb, 0, S.ch[c].ns * sizeof(double), st));
        if (ob) LRDM_CU(cudaMemsetAsync(ob, 0, S.ch[c].ns * sizeof(double), st));
        continue;
      }
      LRDM_CU(launch_eps_occ_bar(S, c, K, fp64, inv_tr, ctx->opt.degen_tol, eb, ob, st));
      count(ctx, 1);
    }
  }
  return LRDM_OK;
}

lrdm_status lrdm_status_query(lrdm_ctx* ctx, int synchronize) {
  if (!ctx) return LRDM_ERR_INVALID_ARG;
  if (synchronize && cudaDeviceSynchronize() != cudaSuccess) return LRDM_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LRDM_ERR_CUDA;
  if (cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) return LRDM_ERR_CUDA;
  if (h & STATUS_TIMEOUT) return LRDM_ERR_TIMEOUT;
  if (h & STATUS_NONFINITE) return LRDM_ERR_NONFINITE;
  if (h & STATUS_SINGULAR) return LRDM_ERR_SINGULAR;
  return LRDM_OK;
}

lrdm_status lrdm_get_mu(lrdm_ctx* ctx, int sys, double* mu_host) {
  if (!ctx || !mu_host || sys < 0 || sys >= ctx->nsys) return LRDM_ERR_INVALID_ARG;
  *mu_host = ctx->sys[sys].mu;
  return LRDM_OK;
}

lrdm_status lrdm_get_density(lrdm_ctx* ctx, int sys, int spin, void* out, void* stream) {
  if (!ctx || !out || sys < 0 || sys >= ctx->nsys) return LRDM_ERR_INVALID_ARG;
  SysState& S = ctx->sys[sys];
  if (spin < 0 || spin >= S.nspin) return LRDM_ERR_INVALID_ARG;
  return from_cuda(launch_to_io(S.ch[spin].rho, S.Ng, out, ctx->opt.io_dtype,
                                static_cast<cudaStream_t>(stream)));
}

lrdm_status lrdm_get_projection(lrdm_ctx* ctx, int sys, int spin, int k, double* out,
                                void* stream) {
  if (ctx && ctx->kp) return LRDM_ERR_UNSUPPORTED;
  if (!ctx || !out || sys < 0 || sys >= ctx->nsys) return LRDM_ERR_INVALID_ARG;
  SysState& S = ctx->sys[sys];
  if (spin < 0 || spin >= S.nspin || k < 0 || k >= S.last_K) return LRDM_ERR_INVALID_ARG;
  return from_cuda(launch_get_projection(S, spin, k, ctx->opt.prec == LRDM_FP64, out,
                                         static_cast<cudaStream_t>(stream)));
}

lrdm_status lrdm_get_tuning(lrdm_ctx* ctx, int* g1_nb, int* g1_dpt, int* g2_bn, int* g2_kgroup) {
  if (!ctx) return LRDM_ERR_INVALID_ARG;
  if (g1_nb) *g1_nb = ctx->tune.g1_nb;
  if (g1_dpt) *g1_dpt = ctx->tune.g1_dpt;
  if (g2_bn) *g2_bn = ctx->tune.g2_bn;
  if (g2_kgroup) *g2_kgroup = ctx->tune.g2_kgroup;
  return LRDM_OK;
}

lrdm_status lrdm_set_tuning(lrdm_ctx* ctx, int g1_nb, int g1_dpt, int g2_bn, int g2_kgroup) {
  if (!ctx) return LRDM_ERR_INVALID_ARG;
  if (!is_tc(ctx->opt.prec)) return LRDM_ERR_UNSUPPORTED;
  const bool nb_ok = g1_nb == 128 || g1_nb == 256 || g1_nb == G1_PAIR;
  const bool dpt_ok = g1_dpt == 1 || (g1_dpt == 2 && g1_nb == 128);
  const bool bn_ok = g2_bn == 128 || g2_bn == 256 || g2_bn == G2_PAIR;
  const bool kg_ok = g2_kgroup == 1 || g2_kgroup == 2 || g2_kgroup == 4;
  if (!nb_ok || !dpt_ok || !bn_ok || !kg_ok) return LRDM_ERR_INVALID_ARG;
  ctx->tune.g1_nb = g1_nb;
  ctx->tune.g1_dpt = g1_dpt;
  ctx->tune.g2_bn = g2_bn;
  ctx->tune.g2_kgroup = g2_kgroup;
  if (ctx->graph_exec) {            // captured with the old shape (freed once it has run)
    cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
    ctx->graph_key.clear();
  }
  return LRDM_OK;
}

lrdm_status lrdm_profile_enable(lrdm_ctx* ctx, int on) {
  if (!ctx) return LRDM_ERR_INVALID_ARG;
  if (on && ctx->prof_ev.empty()) {
    ctx->prof_ev.resize(2 * PROF_MAX);
    ctx->prof_kind.resize(PROF_MAX);
    for (auto& e : ctx->prof_ev)
      if (cudaEventCreate(&e) != cudaSuccess) return LRDM_ERR_CUDA;
  }
  ctx->prof_on = on != 0;
  return LRDM_OK;
}

lrdm_status lrdm_profile_read(lrdm_ctx* ctx, double* gemm1_ms, long long* gemm1_launches,
                              double* gemm2_ms, long long* gemm2_launches, double* poisson_ms,
                              long long* poisson_calls, long long* kernel_launches, int reset) {
  if (!ctx) return LRDM_ERR_INVALID_ARG;
  double t[4] = {0, 0, 0, 0};
  long long n[4] = {0, 0, 0, 0};
  for (int i = 0; i < ctx->prof_n; ++i) {
    if (cudaEventSynchronize(ctx->prof_ev[2 * i + 1]) != cudaSuccess) return LRDM_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]) != cudaSuccess)
      return LRDM_ERR_CUDA;
    t[ctx->prof_kind[i]] += ms;
    n[ctx->prof_kind[i]] += 1;
  }
  if (gemm1_ms) *gemm1_ms = t[1];
  if (gemm1_launches) *gemm1_launches = n[1];
  if (gemm2_ms) *gemm2_ms = t[2];
  if (gemm2_launches) *gemm2_launches = n[2];
  if (poisson_ms) *poisson_ms = t[3];
  if (poisson_calls) *poisson_calls = n[3];
  if (kernel_launches) *kernel_launches = ctx->launches;
  if (reset) {
    ctx->prof_n = 0;
    ctx->launches = 0;
  }
  return LRDM_OK;
}

void lrdm_destroy(lrdm_ctx* ctx) { free_ctx(ctx); }

}  // extern "C"
