// Brillouin-zone-sampled systems (§II.C closing paragraphs, Eq.
// tracelessCondition) behind lrdm_kp_create / lrdm_kp_gateaux: set-up of the
// k-point subspaces, the BZ-averaged response (CUDA cores in FP64 / FP32, the
// real tensor-core contractions on the stacked operand [Re Psi, Im Psi] in
// TF32 / BF16x3) and its adjoint.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "api_common.h"

using namespace lrdm;
using namespace lrdm::api;

// ---------------------------------------------------------------------------
// Brillouin-zone-sampled systems (lrdm_kp_create / lrdm_kp_gateaux)
// ---------------------------------------------------------------------------

namespace {

// mu with g sum_kappa w_kappa sum_i f((eps_i,kappa - mu)/kT) = N_e, bisection
lrdm_status solve_mu_kp_host(const std::vector<std::vector<double>>& eps, const std::vector<double>& kw,
                             double ne, double kT, double g, double* mu) {
  auto electrons = [&](double m) {
    double c = 0.0;
    for (size_t q = 0; q < eps.size(); ++q) {
      double cq = 0.0;
      for (double e : eps[q]) cq += fermi_host((e - m) / kT);
      c += kw[q] * cq;
    }
    return g * c;
  };
  double lo = 1e300, hi = -1e300;
  for (const auto& e : eps)
    for (double x : e) {
      lo = fmin(lo, x);
      hi = fmax(hi, x);
    }
  lo -= 800.0 * kT;
  hi += 800.0 * kT;
  if (!(electrons(lo) < ne && ne < electrons(hi))) return LRDM_ERR_MU_NOT_CONVERGED;
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (electrons(mid) < ne) lo = mid;
    else hi = mid;
  }
  *mu = 0.5 * (lo + hi);
  return LRDM_OK;
}

// The k-point response of the weights in S.a ([K][N_g,pad], compute type):
// per point P = Psi^H diag(a_k) Psi, mu'_k from the BZ-averaged traceless
// condition (into S.dmu, and dmu_out when given), Gamma = L o (P - mu' I),
// and factor * w_kappa diag(Psi Gamma Psi^H) into the per-point FP32
// contributions (tensor cores) or the FP64 accumulator (CUDA cores).  The
// forward passes a = w dV and factor g; the adjoint a = fbar and factor w g
// (the map is self-adjoint, the same traceless projection applies).
// Grid-row ranges of the tensor-core projection for K directions over all
// k-points: the fewest ranges (up to the P buffers' capacity, at least 64
// stages each) whose work items fill the persistent grid's waves to 90 %,
// else the best fill.
int kp_choose_split(lrdm_ctx* ctx, int K) {
  const bool pair = ctx->tune.g1_nb == G1_PAIR;
  // work units of the persistent grid: SMs, or CTA pairs for the pair tiles
  const int sms = pair ? tc_pair_units(ctx->opt.prec) : ctx->sm_count > 0 ? ctx->sm_count : 152;
  long long per = 0;                                // items of one range over all points
  int nch = 1 << 30;
  for (int q = 0; q < ctx->kp_nk; ++q) {
    const TcProblem& pr = ctx->tc_host[ctx->kp_pid[q]];
    const bool wide = ctx->tune.g1_nb == 256;
    const int dpt = wide || pair ? 1 : ctx->tune.g1_dpt;
    per += (long long)(pair ? pr.ntiles_p : wide ? pr.ntiles_w : pr.ntiles) * ((K + dpt - 1) / dpt);
    nch = std::min(nch, pr.nch);
  }
  int best = 1;
  double best_fill = 0.0;
  for (int s = 1; s <= ctx->kp_split_cap && nch / s >= 64; ++s) {
    const long long items = per * s;
    const long long waves = (items + sms - 1) / sms;
    const double fill = (double)items / (double)(waves * sms);
    if (fill > best_fill + 1e-9) {
      best_fill = fill;
      best = s;
    }
    if (fill >= 0.9) break;
  }
  return best;
}

lrdm_status kp_response(lrdm_ctx* ctx, int K, double factor, double* dmu_out, cudaStream_t st) {
  NvtxRange nvtx_("k-point response");
  SysState& S = ctx->sys[0];
  const int prec = ctx->opt.prec;
  const int fp64 = prec == LRDM_FP64;
  const bool tc = is_tc(prec);
  const int ns = ctx->kp_ns, nk = ctx->kp_nk;
  const int split = tc ? kp_choose_split(ctx, K) : ctx->kp_nsplit;
  if (tc) {
    ctx->tc_entries.clear();
    for (int q = 0; q < nk; ++q) {
      TcEntry x;
      x.dev_base = ctx->tc_dev;
      x.pid = ctx->kp_pid[q];
      x.host = &ctx->tc_host[x.pid];
      x.K = K;
      x.X = ctx->kp_ch[q].Xpart;
      x.split = split;
      ctx->tc_entries.push_back(x);
    }
    LRDM_CK(tc_group(ctx, 1, 0, st));
  } else {
    int pi = prof_begin(ctx, 1, st);
    for (int q = 0; q < nk; ++q)
      LRDM_CU(launch_kp_gemm1(fp64, ctx->kp_pr[q], ctx->kp_pi[q], ns, S.Ng, S.a, S.Ng_pad, K, ctx->kp_Xr[q],
                              ctx->kp_Xi[q], ctx->kp_nsplit, st));
    prof_end(ctx, pi, st);
    count(ctx, nk);
  }
  KpDmuArgs A{};
  for (int q = 0; q < nk; ++q) {
    A.Xr[q] = tc ? ctx->kp_ch[q].Xpart : ctx->kp_Xr[q];
    A.L[q] = ctx->kp_L[q];
    A.kw[q] = ctx->kp_w[q];
  }
  A.nk = nk;
  A.ns = ns;
  A.K = K;
  A.nsplit = split;
  A.fp64 = fp64;
  A.ld = tc ? ctx->kp_ch[0].ns_pad : ns;
  A.stacked = tc ? 1 : 0;
  LRDM_CU(launch_kp_dmu(A, S.dmu, dmu_out, st));
  count(ctx, 1);
  if (tc) {
    const int layout = prec == LRDM_BF16X3 ? 2 : 1;
    ctx->tc_entries.clear();
    for (int q = 0; q < nk; ++q) {
      const Channel& c = ctx->kp_ch[q];
      LRDM_CU(launch_kp_scale_tc(static_cast<const float*>(c.Xpart), split, K, ns, c.ns_pad, ctx->kp_L[q],
                                 S.dmu, layout, c.Xpp, c.Xpp_lo, st));
      TcEntry x;
      x.dev_base = ctx->tc_dev;
      x.pid = ctx->kp_pid[q];
      x.host = &ctx->tc_host[x.pid];
      x.K = K;
      x.factor = factor * ctx->kp_w[q];
      x.out = ctx->kp_out[q];
      x.out_stride = S.Ng;
      ctx->tc_entries.push_back(x);
    }
    count(ctx, nk);
    LRDM_CK(tc_group(ctx, 2, 0, st));
  } else {
    LRDM_CU(cudaMemsetAsync(ctx->kp_drho, 0, (size_t)K * S.Ng * sizeof(double), st));
    for (int q = 0; q < nk; ++q)
      LRDM_CU(launch_kp_scale(fp64, ctx->kp_Xr[q], ctx->kp_Xi[q], ctx->kp_nsplit, K, ns, ctx->kp_L[q], S.dmu,
                              ctx->kp_Yr[q], ctx->kp_Yi[q], st));
    int pi = prof_begin(ctx, 2, st);
    for (int q = 0; q < nk; ++q)
      LRDM_CU(launch_kp_gemm2(fp64, ctx->kp_pr[q], ctx->kp_pi[q], ns, S.Ng, ctx->kp_Yr[q], ctx->kp_Yi[q], K,
                              factor * ctx->kp_w[q], ctx->kp_drho, st));
    prof_end(ctx, pi, st);
    count(ctx, 2 * nk);
  }
  return LRDM_OK;
}

}  // namespace

namespace lrdm {
namespace api {

// The k-point forward: dV_k = V_H[v_k] + f_x v_k, a_k = w dV_k (zero in the
// grid padding), the response with factor g, f_k = drho_k - v_k.
lrdm_status kp_forward(lrdm_ctx* ctx, const void* v, int K, void* f_out, double* dmu_out, cudaStream_t st) {
  SysState& S = ctx->sys[0];
  const int fp64 = ctx->opt.prec == LRDM_FP64;
  const int io = ctx->opt.io_dtype;
  LRDM_CU(launch_spin_sum(v, io, K, 1, S.Ng, S.fft_real, fp64, st, S.Ng));
  LRDM_CK(hartree(ctx, S, K, st));
  LRDM_CU(launch_dv_weights(v, io, S.fft_real, S.ch[0].fx, S.ch[0].fx, K, 1, S.Ng, S.Ng_pad, S.w, S.a,
                            fp64, st, S.Ng));
  count(ctx, 3);
  LRDM_CK(kp_response(ctx, K, S.g, dmu_out, st));
  if (is_tc(ctx->opt.prec)) {
    KpSumArgs B{};
    for (int q = 0; q < ctx->kp_nk; ++q) B.part[q] = ctx->kp_out[q];
    B.nk = ctx->kp_nk;
    LRDM_CU(launch_kp_sum(B, v, io, (long long)K * S.Ng, f_out, st));
  } else {
    LRDM_CU(launch_kp_finish(ctx->kp_drho, v, io, (long long)K * S.Ng, f_out, st));
  }
  count(ctx, 1);
  return LRDM_OK;
}

// Adjoint of lrdm_kp_gateaux with respect to the directions: the response of
// the weights fbar with factor w g, then vbar = V_H[dVbar] + f_x dVbar - fbar.
// Eigenvalue / occupation gradients are not defined for k-point contexts.
lrdm_status kp_backward(lrdm_ctx* ctx, const void* const* f_bar, void* const* v_bar,
                        double* const* eps_bar, double* const* occ_bar, cudaStream_t st) {
  if ((eps_bar && (eps_bar[0] || eps_bar[1])) || (occ_bar && (occ_bar[0] || occ_bar[1])))
    return LRDM_ERR_UNSUPPORTED;
  SysState& S = ctx->sys[0];
  const int K = S.last_K;
  if (K < 0) return LRDM_ERR_INVALID_ARG;      // no forward call yet
  if (K == 0) return LRDM_OK;
  if (!f_bar[0] || !v_bar[0]) return LRDM_ERR_INVALID_ARG;
  const int fp64 = ctx->opt.prec == LRDM_FP64;
  const int io = ctx->opt.io_dtype;
  LRDM_CU(launch_scale_weights(f_bar[0], io, K, 1, S.Ng, S.Ng_pad, 1.0, S.a, fp64, st));
  LRDM_CK(kp_response(ctx, K, S.w * S.g, nullptr, st));
  if (is_tc(ctx->opt.prec)) {
    KpSumArgs B{};
    for (int q = 0; q < ctx->kp_nk; ++q) B.part[q] = ctx->kp_out[q];
    B.nk = ctx->kp_nk;
    LRDM_CU(launch_kp_collect(&B, nullptr, K, S.Ng, S.Ng_pad, S.a, fp64, st));
  } else {
    LRDM_CU(launch_kp_collect(nullptr, ctx->kp_drho, K, S.Ng, S.Ng_pad, S.a, fp64, st));
  }
  LRDM_CU(launch_spin_sum_padded(S.a, K, 1, S.Ng, S.Ng_pad, S.fft_real, fp64, st, S.Ng));
  LRDM_CK(hartree(ctx, S, K, st));
  LRDM_CU(launch_adjoint_potential(S.a, S.fft_real, S.ch[0].fx, S.ch[0].fx, f_bar[0], io, K, 1, S.Ng,
                                   S.Ng_pad, v_bar[0], fp64, st, S.Ng));
  count(ctx, 5);
  return LRDM_OK;
}

}  // namespace api
}  // namespace lrdm

namespace {

lrdm_status kp_setup(lrdm_ctx* ctx, const lrdm_kpoint_system& in, cudaStream_t st) {
  const lrdm_options& o = ctx->opt;
  const int prec = o.prec;
  const int fp64 = prec == LRDM_FP64;
  const bool tc = is_tc(prec);
  const size_t csz = fp64 ? sizeof(double) : sizeof(float);
  SysState& S = ctx->sys[0];
  for (int d = 0; d < 3; ++d) {
    S.n[d] = in.n[d];
    S.h[d] = in.h[d];
  }
  S.Ng = (long long)in.n[0] * in.n[1] * in.n[2];
  S.Ngrid = S.Ng;
  S.Ng_pad = tc ? (S.Ng + TC_PAD_GRID - 1) / TC_PAD_GRID * TC_PAD_GRID : S.Ng;
  S.nspin = 1;
  S.kmax = in.k_max > 0 ? in.k_max : o.k_max;
  S.w = in.h[0] * in.h[1] * in.h[2];
  S.g = in.occ_factor > 0.0 ? in.occ_factor : 2.0;
  S.kT = in.kT;
  S.ne = in.n_electrons;
  const int nk = in.nk, ns = in.ns;
  ctx->kp = true;
  ctx->kp_nk = nk;
  ctx->kp_ns = ns;
  ctx->kp_w.assign(in.k_weights, in.k_weights + nk);
  std::vector<std::vector<double>> eps(nk, std::vector<double>(ns)), occ(nk, std::vector<double>(ns));
  for (int q = 0; q < nk; ++q)
    LRDM_CU(cudaMemcpy(eps[q].data(), in.eps[q], ns * sizeof(double), cudaMemcpyDeviceToHost));
  LRDM_CK(solve_mu_kp_host(eps, ctx->kp_w, S.ne, S.kT, S.g, &S.mu));
  // CUDA cores: row ranges of the projection, about two blocks per SM at
  // k_max directions; tensor cores: the whole grid per tile
  ctx->kp_nsplit = 1;
  if (!tc) {
    const int nt = (ns + 63) / 64;
    const long long blocks = (long long)nt * (nt + 1) / 2 * S.kmax;
    const int sms = ctx->sm_count > 0 ? ctx->sm_count : 152;
    long long split = (2LL * sms + blocks - 1) / blocks;
    if (split > S.Ng / 256) split = S.Ng / 256;
    if (split > 64) split = 64;
    ctx->kp_nsplit = (int)(split < 1 ? 1 : split);
  }
  const size_t npsi = (size_t)S.Ng * ns, mat = (size_t)ns * ns;
  ctx->kp_pr.assign(nk, nullptr);
  ctx->kp_pi.assign(nk, nullptr);
  ctx->kp_eps.assign(nk, nullptr);
  ctx->kp_occ.assign(nk, nullptr);
  ctx->kp_L.assign(nk, nullptr);
  ctx->kp_Xr.assign(nk, nullptr);
  ctx->kp_Xi.assign(nk, nullptr);
  ctx->kp_Yr.assign(nk, nullptr);
  ctx->kp_Yi.assign(nk, nullptr);
  if (tc) {
    ctx->kp_ch.assign(nk, Channel());
    ctx->kp_pid.assign(nk, -1);
    ctx->kp_out.assign(nk, nullptr);
  }
  Channel& ch = S.ch[0];
  ch.ns = ns;
  LRDM_CK(dalloc(ctx, &ch.rho, S.Ng, false));
  const size_t xc = (size_t)ctx->kp_nsplit * S.kmax * mat;
  const int io = o.io_dtype;
  const size_t isz = io == LRDM_DTYPE_F64 ? sizeof(double) : sizeof(float);
  void* stack = nullptr;                       // tensor cores: [N_g][2 N_s] io dtype, set-up only
  if (tc && cudaMalloc(&stack, npsi * 2 * isz) != cudaSuccess) return LRDM_ERR_OOM;
  lrdm_status rc = LRDM_OK;
  for (int q = 0; q < nk && rc == LRDM_OK; ++q) {
    rc = [&]() -> lrdm_status {
      for (int i = 0; i < ns; ++i) occ[q][i] = fermi_host((eps[q][i] - S.mu) / S.kT);
      LRDM_CK(dalloc(ctx, &ctx->kp_eps[q], ns, false));
      LRDM_CK(dalloc(ctx, &ctx->kp_occ[q], ns, false));
      LRDM_CU(cudaMemcpyAsync(ctx->kp_eps[q], eps[q].data(), ns * sizeof(double), cudaMemcpyHostToDevice, st));
      LRDM_CU(cudaMemcpyAsync(ctx->kp_occ[q], occ[q].data(), ns * sizeof(double), cudaMemcpyHostToDevice, st));
      LRDM_CK(dalloc(ctx, &ctx->kp_L[q], mat, false));
      LRDM_CU(launch_loewner(ctx->kp_eps[q], ctx->kp_occ[q], ns, S.mu, S.kT, 0, o.degen_tol, 0,
                             ctx->kp_L[q], st));
      if (!tc) {
        LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ctx->kp_pr[q]), npsi * csz, false));
        LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ctx->kp_pi[q]), npsi * csz, false));
        LRDM_CU(launch_kp_copy(fp64, in.psi_re[q], io, in.ld_psi, S.Ng, ns, ctx->kp_pr[q], ns, 0, st));
        LRDM_CU(launch_kp_copy(fp64, in.psi_im[q], io, in.ld_psi, S.Ng, ns, ctx->kp_pi[q], ns, 0, st));
        LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ctx->kp_Xr[q]), xc * csz));
        LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ctx->kp_Xi[q]), xc * csz));
        LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ctx->kp_Yr[q]), (size_t)S.kmax * mat * csz));
        LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ctx->kp_Yi[q]), (size_t)S.kmax * mat * csz));
        if (!in.rho)
          LRDM_CU(launch_kp_density(fp64, ctx->kp_pr[q], ctx->kp_pi[q], ns, ns, S.Ng, ctx->kp_occ[q],
                                    S.g * ctx->kp_w[q], q == 0, in.rho_floor, ch.rho, st));
        return LRDM_OK;
      }
      // stacked operand C = [Re Psi, Im Psi] in the layouts of the real contractions
      Channel& c = ctx->kp_ch[q];
      c.ns = 2 * ns;
      c.ns_pad = (2 * ns + TC_PAD_STATES - 1) / TC_PAD_STATES * TC_PAD_STATES;
      const int dio = io == LRDM_DTYPE_F64;
      LRDM_CU(launch_kp_copy(dio, in.psi_re[q], io, in.ld_psi, S.Ng, ns, stack, 2 * ns, 0, st));
      LRDM_CU(launch_kp_copy(dio, in.psi_im[q], io, in.ld_psi, S.Ng, ns, stack, 2 * ns, ns, st));
      if (!in.rho)
        LRDM_CU(launch_kp_density(dio, stack, static_cast<const char*>(stack) + ns * isz, ns, 2 * ns, S.Ng,
                                  ctx->kp_occ[q], S.g * ctx->kp_w[q], q == 0, in.rho_floor, ch.rho, st));
      const size_t npad = (size_t)S.Ng_pad * c.ns_pad;
      const size_t ld2 = (size_t)c.ns_pad * c.ns_pad;
      if (prec == LRDM_TF32) {
        LRDM_CK(dalloc(ctx, &c.psiR32, npad, false));
        LRDM_CK(dalloc(ctx, &c.psiT32, npad, false));
        LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&c.Xpp), (size_t)S.kmax * ld2 * sizeof(float)));
      } else {
        LRDM_CK(dalloc(ctx, &c.psiR_hi, npad, false));
        LRDM_CK(dalloc(ctx, &c.psiR_lo, npad, false));
        LRDM_CK(dalloc(ctx, &c.psiT_hi, npad, false));
        LRDM_CK(dalloc(ctx, &c.psiT_lo, npad, false));
        LRDM_CK(dalloc(ctx, &c.psiTf, npad, false));
        LRDM_CK(dalloc(ctx, reinterpret_cast<__nv_bfloat16**>(&c.Xpp), (size_t)S.kmax * ld2));
        LRDM_CK(dalloc(ctx, reinterpret_cast<__nv_bfloat16**>(&c.Xpp_lo), (size_t)S.kmax * ld2));
      }
      LRDM_CU(launch_convert_psi(stack, io, 2 * ns, S.Ng, 2 * ns, c, prec, S.Ng_pad, st));
      LRDM_CU(cudaStreamSynchronize(st));      // the stacked copy is reused for the next point
      // room for up to 4 grid-row ranges of the projection (kp_choose_split),
      // fewer where that would exceed 1 GB per point
      int cap = 4;
      while (cap > 1 && (size_t)cap * S.kmax * ld2 * sizeof(float) > ((size_t)1 << 30)) --cap;
      ctx->kp_split_cap = cap;
      LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&c.Xpart), (size_t)cap * S.kmax * ld2 * sizeof(float)));
      LRDM_CK(dalloc(ctx, &ctx->kp_out[q], (size_t)S.kmax * S.Ng));
      return LRDM_OK;
    }();
  }
  if (stack) cudaFree(stack);
  LRDM_CK(rc);
  if (in.rho) LRDM_CU(launch_copy_rho(in.rho, io, S.Ng, ch.rho, st));
  LRDM_CK(dalloc(ctx, &ch.fx, S.Ng, false));
  LRDM_CU(launch_fx(ch.rho, S.Ng, 0, ch.fx, st));
  LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&S.a), (size_t)S.kmax * S.Ng_pad * csz));
  LRDM_CK(dalloc(ctx, &S.dmu, S.kmax));
  if (!tc) LRDM_CK(dalloc(ctx, &ctx->kp_drho, (size_t)S.kmax * S.Ng));
  LRDM_CK(setup_poisson(ctx, S, st));
  if (tc) {
    for (int q = 0; q < nk; ++q) {
      TcProblem pr;
      if (!build_tc_problem(prec, ctx->kp_ch[q], S, 0, pr)) return LRDM_ERR_CUDA;
      LRDM_CK(dalloc(ctx, &pr.part, (size_t)G2_MAX_SPLIT * S.Ng));
      ctx->kp_pid[q] = (int)ctx->tc_host.size();
      ctx->tc_host.push_back(pr);
    }
    LRDM_CK(dalloc(ctx, reinterpret_cast<char**>(&ctx->tc_dev), ctx->tc_host.size() * sizeof(TcProblem), false));
    LRDM_CU(cudaMemcpy(ctx->tc_dev, ctx->tc_host.data(), ctx->tc_host.size() * sizeof(TcProblem),
                       cudaMemcpyHostToDevice));
    ctx->tc_entries.reserve(nk);
  }
  LRDM_CU(cudaStreamSynchronize(st));   // the host eps / occ vectors end here
  return LRDM_OK;
}

}  // namespace

extern "C" {

lrdm_status lrdm_kp_create(lrdm_ctx** out, const lrdm_kpoint_system* sys, const lrdm_options* opt,
                           void* stream) {
  NvtxRange nvtx_("lrdm_kp_create");
  if (!out) return LRDM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!sys || sys->nk < 1 || sys->nk > KP_MAX || sys->ns < 1 || sys->ld_psi < sys->ns)
    return LRDM_ERR_INVALID_ARG;
  if (!sys->psi_re || !sys->psi_im || !sys->eps || !sys->k_weights) return LRDM_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (sys->n[d] < 2 || !(sys->h[d] > 0.0)) return LRDM_ERR_INVALID_ARG;
  double wsum = 0.0;
  for (int q = 0; q < sys->nk; ++q) {
    if (!sys->psi_re[q] || !sys->psi_im[q] || !sys->eps[q] || !(sys->k_weights[q] > 0.0))
      return LRDM_ERR_INVALID_ARG;
    wsum += sys->k_weights[q];
  }
  if (!(fabs(wsum - 1.0) <= 1e-12) || !(sys->kT > 0.0) || !(sys->n_electrons > 0.0))
    return LRDM_ERR_INVALID_ARG;
  lrdm_options o;
  if (opt) o = *opt;
  else lrdm_default_options(&o);
  if (o.prec < LRDM_FP64 || o.prec > LRDM_BF16X3) return LRDM_ERR_INVALID_ARG;
  if (o.io_dtype != LRDM_DTYPE_F64 && o.io_dtype != LRDM_DTYPE_F32) return LRDM_ERR_INVALID_ARG;
  if (o.k_max < 1 || o.k_max > KMAX_LIMIT || sys->k_max < 0 || sys->k_max > KMAX_LIMIT)
    return LRDM_ERR_INVALID_ARG;
  if (is_tc(o.prec) && !tc_supported()) return LRDM_ERR_UNSUPPORTED;
  if (!(o.degen_tol >= 0.0) || (o.poisson_symbol != 0 && o.poisson_symbol != 1)) return LRDM_ERR_INVALID_ARG;
  lrdm_ctx* ctx = new (std::nothrow) lrdm_ctx();
  if (!ctx) return LRDM_ERR_OOM;
  ctx->nsys = 1;
  ctx->opt = o;
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  ctx->sys = new (std::nothrow) SysState[1];
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
    if ((rc = kp_setup(ctx, *sys, st)) != LRDM_OK) break;
    if (is_tc(o.prec) && o.autotune && (rc = autotune(ctx, st)) != LRDM_OK) break;
    if (cudaGetLastError() != cudaSuccess) rc = LRDM_ERR_CUDA;
  } while (0);
  if (rc != LRDM_OK) {
    free_ctx(ctx);
    return rc;
  }
  *out = ctx;
  return LRDM_OK;
}

lrdm_status lrdm_kp_get_split(lrdm_ctx* ctx, int K, int* split) {
  if (!ctx || !ctx->kp || !split || K < 1 || K > ctx->sys[0].kmax) return LRDM_ERR_INVALID_ARG;
  *split = is_tc(ctx->opt.prec) ? kp_choose_split(ctx, K) : ctx->kp_nsplit;
  return LRDM_OK;
}

lrdm_status lrdm_kp_gateaux(lrdm_ctx* ctx, const void* v, int K, void* f_out, double* dmu_out,
                            void* stream) {
  NvtxRange nvtx_("lrdm_kp_gateaux");
  if (!ctx || !ctx->kp) return LRDM_ERR_INVALID_ARG;
  SysState& S = ctx->sys[0];
  if (K < 0 || K > S.kmax) return LRDM_ERR_INVALID_ARG;
  if (K == 0) {
    S.last_K = 0;
    return LRDM_OK;
  }
  if (!v || !f_out) return LRDM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  S.last_K = K;
  if (use_graph(ctx, st)) {
    const std::vector<const void*> key = {v, f_out, reinterpret_cast<const void*>((intptr_t)K), dmu_out, st};
    return graph_call(ctx, key, st, [&] { return kp_forward(ctx, v, K, f_out, dmu_out, st); });
  }
  return kp_forward(ctx, v, K, f_out, dmu_out, st);
}

}  // extern "C"
