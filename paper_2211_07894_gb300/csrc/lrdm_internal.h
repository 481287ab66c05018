// Internal declarations shared by the host orchestration (lrdm_api.cu) and
// the kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lrdm.h"
#include "tc_problem.h"

namespace lrdm {

// Rounds to the TF32 grid (nearest, ties away from zero): the values the TF32
// response GEMM reads as its X'' operand.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
  return __uint_as_float(t);
}

// Four consecutive shared-memory values (16-byte aligned) with 128-bit loads:
// the register tiles of the CUDA-core contractions.
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// NVTX range for the profilers' timelines (one per API call and per phase of
// the forward / adjoint); no cost beyond a call when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Bits of the sticky device status word.
enum : int {
  STATUS_TIMEOUT = 1,
  STATUS_NONFINITE = 2,
  STATUS_SINGULAR = 4,
};

constexpr int KMAX_LIMIT = 64;       // directions per system per call
constexpr int SIMT_TILE = 64;        // CUDA-core GEMM tile edge (states)
constexpr int LS_CHUNK = 64;         // grid points per staged chunk in the Gram kernel
constexpr int LS_BLOCKS = 304;       // 2 x 152 SMs
constexpr int UPD_BLOCKS = 608;

// Tensor-core operand layout (BF16X3 / TF32): padded edges.
constexpr int TC_PAD_STATES = 128;   // states padded to a multiple of this
constexpr int TC_PAD_GRID = 128;     // grid rows padded to a multiple of this

struct Channel {
  int ns = 0;
  int ns_pad = 0;                    // tensor-core padded state count
  double* eps = nullptr;             // [ns]
  double* occ = nullptr;             // [ns]
  double* L = nullptr;               // [ns][ns] Loewner matrix
  float* Lf = nullptr;               // [ns_pad][ns_pad] FP32 copy, zero padded (tensor-core modes)
  double* fx = nullptr;              // [Ng] xc kernel
  double* rho = nullptr;             // [Ng] density used for fx
  // Psi operand copies (which ones exist depends on the precision)
  double* psi64 = nullptr;           // [Ng][ns]
  float* psi32 = nullptr;            // [Ng][ns]           (FP32 SIMT)
  float* psiT32 = nullptr;           // Psi^T tile-major [ns_pad/128][Ng_pad/16][128][16] (TF32, GEMM1)
  float* psiR32 = nullptr;           // [Ng_pad][ns_pad]   (TF32, GEMM2 operand)
  __nv_bfloat16* psiT_hi = nullptr;  // Psi^T tile-major [ns_pad/128][Ng_pad/32][128][32] (BF16X3, GEMM1)
  __nv_bfloat16* psiT_lo = nullptr;
  float* psiTf = nullptr;            // Psi^T tile-major FP32 [ns_pad/128][Ng_pad/32][128][32] (BF16X3, GEMM1 A)
  __nv_bfloat16* psiR_hi = nullptr;  // [Ng_pad][ns_pad]   (BF16X3, GEMM2)
  __nv_bfloat16* psiR_lo = nullptr;
  // workspaces
  void* Xpart = nullptr;             // [nsplit][kmax][ns][ns] forward X (acc type)
  void* Gpart = nullptr;             // [nsplit][kmax][ns][ns] backward Gbar
  void* Xpp = nullptr;               // GEMM2 operand (layout depends on precision)
  void* Xpp_lo = nullptr;            // BF16X3 low part
};

struct SysState {
  int n[3] = {0, 0, 0};
  double h[3] = {0, 0, 0};
  long long Ng = 0;                  // grid rows held (all N_g, or one slab of a row-sharded grid)
  long long Ngrid = 0;               // points of the full grid (the Poisson solve's size)
  long long r0 = 0;                  // first row held
  long long Ng_pad = 0;
  int nspin = 1;
  int kmax = 0;
  double w = 0, g = 2, kT = 0, ne = 0, mu = 0;
  bool occ_given = false;
  Channel ch[2];
  int xslots = 0;                    // tensor cores: direction slots of the X / G buffers (>= kmax;
                                     // grid-row partials of a K-direction call use nsplit * K of them)
  int nsplit = 1;                    // grid-row splits of GEMM1 (CUDA cores: fixed at create;
                                     // tensor cores: chosen per call from K, nsplit * K <= xslots)
  // Poisson
  cufftHandle plan_r2c = 0, plan_c2r = 0;
  bool plans = false;
  void* fft_real = nullptr;          // [kmax][Ngrid] compute type
  void* fft_cplx = nullptr;          // [kmax][n0][n1][n2/2+1]
  double* sym = nullptr;             // [n0][n1][n2/2+1] Poisson symbol / N_g
  void* a = nullptr;                 // [kmax][nspin][Ng_pad] GEMM1 weights (compute type)
  double* dmu = nullptr;             // [kmax]
  double* tbar = nullptr;            // [kmax] backward trace terms
  int last_K = -1;                   // K of the most recent forward call
};

// The caller's sum over the ranks of a grid-row-sharded system.
struct AllReduce {
  lrdm_allreduce_fn fn = nullptr;
  void* user = nullptr;
};

}  // namespace lrdm

struct lrdm_ctx {
  int nsys = 0;
  lrdm_options opt{};
  int device = 0;
  lrdm::SysState* sys = nullptr;
  int* d_status = nullptr;
  unsigned* d_round = nullptr;       // round counter of the tensor-core contractions (zeroed per launch)
  double* ls_partial = nullptr;      // [LS_BLOCKS][max values]
  double* ls_coef = nullptr;         // [KMAX_LIMIT]
  double* ls_scal = nullptr;         // [4]: r2, s_rel scratch
  double* upd_partial = nullptr;     // [UPD_BLOCKS]
  double* gs_scratch = nullptr;      // Gram-Schmidt partial sums (Krylov step)
  double* gs_norm = nullptr;         // [1] norm of the last normalised direction
  std::vector<void*> allocs;         // every device allocation, freed by lrdm_destroy
  // tensor-core problem table: one entry per (system, channel)
  std::vector<lrdm::TcProblem> tc_host;
  lrdm::TcProblem* tc_dev = nullptr;
  std::vector<int> tc_pid;           // [2 * sys + channel] -> index, -1 if absent
  std::vector<lrdm::TcEntry> tc_entries;   // scratch list for one grouped launch
  // CUDA graph of lrdm_gateaux_batch (use_graph)
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<const void*> graph_key;
  lrdm::TcTune tune;                 // launch shape of the tensor-core contractions
  // grid-row sharding (lrdm_create_rows): the rows this context holds and the
  // caller's sum over the ranks
  bool rows = false;
  long long rows_begin = 0, rows_n = 0;
  lrdm::AllReduce ar;
  int sm_count = 0;
  std::vector<double> inv_trace;     // per system 1 / sum_s sum_i L_ii
  // profiling (lrdm_profile_enable / lrdm_profile_read)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // pairs: [2 i] start, [2 i + 1] end
  std::vector<int> prof_kind;        // 1 = GEMM1, 2 = GEMM2 per pair
  int prof_n = 0;
  long long launches = 0;            // library kernel launches while profiling
  // Brillouin-zone-sampled system (lrdm_kp_create): one periodic system, nk
  // complex subspaces sharing mu, the grid and the Poisson plans of sys[0]
  bool kp = false;
  int kp_nk = 0, kp_ns = 0, kp_nsplit = 1;
  std::vector<double> kp_w;          // BZ weights
  std::vector<void*> kp_pr, kp_pi;   // [nk] Psi planes [N_g][N_s] compute type
  std::vector<double*> kp_eps, kp_occ, kp_L;
  std::vector<void*> kp_Xr, kp_Xi;   // [nk] [nsplit][kmax][N_s][N_s]
  std::vector<void*> kp_Yr, kp_Yi;   // [nk] [kmax][N_s][N_s] Loewner-scaled
  double* kp_drho = nullptr;         // [kmax][N_g] FP64 accumulator
  // tensor-core modes: per k-point the stacked real operand C = [Re Psi, Im Psi]
  // (N_g x 2 N_s) as one channel of the real contractions, its problem index
  // and its FP32 density contribution [kmax][N_g]
  std::vector<lrdm::Channel> kp_ch;
  std::vector<int> kp_pid;
  std::vector<float*> kp_out;
  int kp_split_cap = 1;              // tensor cores: grid-row ranges the P buffers hold
};

namespace lrdm {

// ---------------- setup kernels (k_setup.cu) ----------------
cudaError_t launch_convert_psi(const void* src, int io_dtype, int ld, long long Ng, int ns,
                               Channel& c, int prec, long long Ng_pad, cudaStream_t st);
cudaError_t launch_density(const void* psi_src, int io_dtype, int ld, long long Ng, int ns,
                           const double* occ, double g, double floor, double* rho, cudaStream_t st);
cudaError_t launch_copy_rho(const void* src, int io_dtype, long long Ng, double* rho, cudaStream_t st);
cudaError_t launch_fx(const double* rho, long long Ng, int spin_polarized, double* fx, cudaStream_t st);
cudaError_t launch_loewner(const double* eps, const double* occ, int ns, double mu, double kT,
                           int occ_mode, double degen_tol, int fermi_T, double* L,
                           cudaStream_t st);
cudaError_t launch_to_io(const double* src, long long n, void* dst, int io_dtype, cudaStream_t st);
// Lf[i][j] = (float) L[i][j] for i, j < ns, 0 in the padding
cudaError_t launch_loewner_f32(const double* L, int ns, int ns_pad, float* Lf, cudaStream_t st);

// ---------------- Brillouin-zone-sampled response (k_kpoint.cu) ----------------
constexpr int KP_MAX = 32;           // k-points per context
struct KpDmuArgs {
  const void* Xr[KP_MAX];            // Re X (CUDA cores) or the stacked Gram P (tensor cores)
  const double* L[KP_MAX];
  double kw[KP_MAX];
  int nk, ns, K, nsplit, fp64;
  int ld;                            // leading dimension of the X planes
  int stacked;                       // 1: Re X_ii = P_ii + P_(ns+i)(ns+i)
};
struct KpSumArgs {
  const float* part[KP_MAX];         // [K][N_g] per k-point, factor included
  int nk;
};
// X_kappa (re, im) = Psi^H diag(a_k) Psi over nsplit grid-row ranges
cudaError_t launch_kp_gemm1(int fp64, const void* pr, const void* pi, int ns, long long Ng,
                            const void* a, long long a_stride, int K, void* Xr, void* Xi, int nsplit,
                            cudaStream_t st);
// mu'_k from the BZ-averaged traceless condition
cudaError_t launch_kp_dmu(const KpDmuArgs& A, double* dmu, double* dmu_out, cudaStream_t st);
// Y = c L o conj(X - mu' I), upper part
cudaError_t launch_kp_scale(int fp64, const void* Xr, const void* Xi, int nsplit, int K, int ns,
                            const double* L, const double* dmu, void* Yr, void* Yi, cudaStream_t st);
// drho[k] += factor * Re diag-form of Y over Psi
cudaError_t launch_kp_gemm2(int fp64, const void* pr, const void* pi, int ns, long long Ng,
                            const void* Yr, const void* Yi, int K, double factor, double* drho,
                            cudaStream_t st);
cudaError_t launch_kp_finish(const double* drho, const void* v, int io, long long n, void* f,
                             cudaStream_t st);
cudaError_t launch_kp_density(int fp64, const void* pr, const void* pi, int ns, int ld, long long Ng,
                              const double* occ, double gw, int first, double floor, double* rho,
                              cudaStream_t st);
// dst[r][col0 + i] = src[r][i] (compute type, leading dimension ldd)
cudaError_t launch_kp_copy(int fp64, const void* src, int io, int ld, long long Ng, int ns, void* dst,
                           int ldd, int col0, cudaStream_t st);
// tensor-core modes: M'' for the real GEMM2 from the stacked Gram P, layout 1
// (TF32) or 2 (BF16 hi/lo), [K][ld][ld]
cudaError_t launch_kp_scale_tc(const float* P, int nsplit, int K, int ns, int ld, const double* L,
                               const double* dmu, int layout, void* out, void* out_lo, cudaStream_t st);
// out[k][r] (compute type, row stride ld, zero padding) = sum_kappa
// A->part[kappa][k][r] (A given) or drho[k][r]
cudaError_t launch_kp_collect(const KpSumArgs* A, const double* drho, int K, long long Ng, long long ld,
                              void* out, int fp64, cudaStream_t st);
// f = sum_kappa part_kappa - v (io dtype)
cudaError_t launch_kp_sum(const KpSumArgs& A, const void* v, int io, long long n, void* f,
                          cudaStream_t st);

// ---------------- element-wise / reduction kernels (k_elem.cu) ----------------
// fft_real[k][r] = sum_s v[k][s][r]  (compute type = double if fp64 else float)
// out[k * out_stride + r] = sum_s v[k][s][r] for r < Ng (out_stride = Ng, or the
// full grid's N_g when the rows are one slab of it)
cudaError_t launch_spin_sum(const void* v, int io_dtype, int K, int nspin, long long Ng,
                            void* fft_real, int fp64, cudaStream_t st, long long out_stride);
// sym[m] = 4 pi / |G_m|^2 / N_g on the half-complex grid (G = 0 -> 0); kind 1
// uses the second-order finite-difference symbol (once per system)
cudaError_t launch_poisson_table(const int* n, const double* h, int kind, double* sym,
                                 cudaStream_t st);
// cplx[k][m] *= sym[m] for k < K
cudaError_t launch_poisson_symbol(void* cplx, int K, long long per, const double* sym, int fp64,
                                  cudaStream_t st);
// a[k][s][r] = scale * (VH[k][r] + fx_s[r] * v[k][s][r]);  mode 1 (adjoint):
// out[k][s][r] = VH[k][r] + fx_s[r] * dvbar[k][s][r] - fbar[k][s][r] (io dtype)
// (VH rows k at VH + k * vh_stride)
cudaError_t launch_dv_weights(const void* v, int io_dtype, const void* VH, const double* fx0,
                              const double* fx1, int K, int nspin, long long Ng, long long Ng_pad,
                              double scale, void* a, int fp64, cudaStream_t st, long long vh_stride);
cudaError_t launch_adjoint_potential(const void* dvbar, const void* VH, const double* fx0,
                                     const double* fx1, const void* fbar, int io_dtype, int K,
                                     int nspin, long long Ng, long long Ng_pad, void* vbar,
                                     int fp64, cudaStream_t st, long long vh_stride);
// a[k][s][r] = scale * fbar[k][s][r]
cudaError_t launch_scale_weights(const void* fbar, int io_dtype, int K, int nspin, long long Ng,
                                 long long Ng_pad, double scale, void* a, int fp64, cudaStream_t st);
// mu'_k = sum_s sum_i L_ii X_ii / sum_s sum_i L_ii (X summed over splits)
cudaError_t launch_dmu(const SysState& S, const void* const* Xparts, int K, int acc_fp64,
                       double* dmu, double* dmu_out, int* status, cudaStream_t st);
// X''[i][j] = c_ij L_ij (X_ij - delta_ij mu'), c = 2 (i<j), 1 (i=j), 0 (i>j)
// (adjoint = 1: Ybar = L o G - delta_ij L_ii tbar_k / sum L, same weights)
cudaError_t launch_loewner_scale(const SysState& S, int s, const void* Xpart, int K, int acc_fp64,
                                 const double* shift, int adjoint, double inv_trace_L,
                                 int prec, cudaStream_t st);
cudaError_t launch_get_projection(const SysState& S, int s, int k, int acc_fp64, double* out,
                                  cudaStream_t st);
// backward: eps_bar / occ_bar of channel s
cudaError_t launch_trace_bar(const SysState& S, const void* const* Gparts, int K, int acc_fp64,
                             double* tbar, cudaStream_t st);
cudaError_t launch_spin_sum_padded(const void* d, int K, int nspin, long long Ng, long long Ng_pad,
                                   void* out, int fp64, cudaStream_t st, long long out_stride);
cudaError_t launch_eps_occ_bar(const SysState& S, int s, int K, int acc_fp64,
                               double inv_trace_L, double degen_tol, double* eps_bar,
                               double* occ_bar, cudaStream_t st);

// ---------------- CUDA-core GEMMs (k_simt.cu) ----------------
// Xpart[split][q][i][j] (tiles I <= J) = sum_r psi[r][i] a[q][r] psi[r][j]
cudaError_t launch_gemm1_simt(int fp64, const void* psi, int ns, long long Ng, const void* a,
                              long long a_stride, int nq, void* Xpart, int nsplit, cudaStream_t st);
// out[q][r] = factor * sum_j sum_i psi[r][i] Xpp[q][i][j] psi[r][j] (- v[q][r] if sub_v)
cudaError_t launch_gemm2_simt(int fp64, const void* psi, int ns, long long Ng, const void* Xpp,
                              int nq, double factor, const void* v, long long v_stride,
                              void* out, long long out_stride, int out_io_dtype, int out_is_io,
                              cudaStream_t st);

// ---------------- least squares (k_ls.cu) ----------------
// out = (t - sum_{k<K} <t, u_k> u_k) / ||.||_w (Krylov step, k_krylov.cu);
// norm_out[0] = the norm before scaling.  scratch: gram_schmidt_scratch() doubles.
// (ar, ar_failed as for launch_ls: the partial sums over the ranks of a row-sharded system)
cudaError_t launch_gram_schmidt(const void* U, int K, const void* t, int io, long long n, double w,
                                void* out, double* scratch, double* norm_out, cudaStream_t st,
                                const AllReduce* ar = nullptr, int* ar_failed = nullptr);
size_t gram_schmidt_scratch();
// norm_out[0] = ||x||_w (scratch: gram_schmidt_scratch() doubles)
cudaError_t launch_norm(const void* x, int io, long long n, double w, double* scratch,
                        double* norm_out, cudaStream_t st, const AllReduce* ar = nullptr,
                        int* ar_failed = nullptr);
// ar (may be null): the Gram partial sums and the residual partial sums are
// summed over the ranks before they are reduced; *ar_failed = 1 (and an early
// return) if the callback fails
cudaError_t launch_ls(const void* R, const void* v, const void* f, int io_dtype, int K,
                      long long n, double w, double alpha, double rcond, void* rho_inout,
                      double* coef, double* coeff_out, double* s_rel_out, double* partial,
                      double* scal, double* upd_partial, int* status, cudaStream_t st,
                      const AllReduce* ar = nullptr, int* ar_failed = nullptr);

// allocation-free least-squares step (k_ls.cu, static device scratch)
int static_k_max();
cudaError_t launch_ls_static(const void* R, const void* v, const void* f, int io_dtype, int K,
                             long long n, double w, double alpha, double rcond, void* rho_inout,
                             double* coeff_out, double* s_rel_out, int* status_out,
                             cudaStream_t st);

// ---------------- tensor-core GEMMs (k_tc.cu) ----------------
// Descriptor of channel ch of system S for the tensor-core kernels (false if a
// tensor map cannot be encoded).
bool build_tc_problem(int prec, const Channel& c, const SysState& S, int ch, TcProblem& pr);
// Grouped launches over n problems (each with its own K; K = 0 entries skipped).
// nch_lim / nR_lim > 0 cap the grid reduction (GEMM1) or the row blocks
// (GEMM2) per problem: partial work with the same item structure (tuning).
// stall != 0 (test only): CTA 0 of the first launch never publishes its
// first weighted stage, so its bounded wait expires (timeout status).
// sync (may be null): a device counter the launches use to start each round
// of work items on all CTAs together (zeroed before every launch that uses
// it; only launches whose items are all equally long use it).
cudaError_t launch_gemm1_tc_group(int prec, const TcEntry* e, int n, int* status, cudaStream_t st,
                                  const TcTune& t, int nch_lim = 0, int stall = 0,
                                  unsigned* sync = nullptr);
// launches (may be null) counts the kernels enqueued: one per 16 problems, plus
// one part-sum kernel per problem whose items were split (K = 1)
cudaError_t launch_gemm2_tc_group(int prec, const TcEntry* e, int n, int out_io, int out_is_io,
                                  int* status, cudaStream_t st, const TcTune& t, int nR_lim = 0,
                                  int* launches = nullptr, unsigned* sync = nullptr);
bool tc_supported();
// CTA pairs the pair-tile projection kernel keeps resident on the current
// device (its persistent grid is twice this many CTAs).
int tc_pair_units(int prec);

}  // namespace lrdm
