// Per-(system, channel) descriptor of the tensor-core contractions, built once
// by lrdm_create and kept in device memory: the TMA tensor maps of both
// contractions (which only reference context-owned buffers) and the sizes.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace lrdm {

struct TcProblem {
  CUtensorMap g1a;                      // GEMM1 A: Psi^T tile-major FP32 (TF32: rounded), box 128 rows
  CUtensorMap g1b0, g1b1;               // GEMM1 B: Psi^T tile-major bf16 hi / lo (TF32: = A)
  CUtensorMap g2a0, g2a1, g2b0, g2b1;   // GEMM2: Psi rows (A), X'' [k_max][j][i] (B)
  long long Ng;                          // grid points
  long long a_stride;                    // direction stride of the GEMM1 weights
  const float* a;                        // GEMM1 weights of this channel (direction 0)
  const void* psi0;                      // GEMM2 epilogue rows: bf16 hi / fp32
  const void* psi1;                      // bf16 lo
  double* part;                          // GEMM2 j-tile part sums [G2_MAX_SPLIT][Ng] (small K)
  int ns, ns_pad, nI, NJ, ntiles, ntiles_w, nch, nR, kmax;   // GEMM1: nI blocks, ntiles tiles; GEMM2: NJ, nR
  int ntiles_p;                          // GEMM1 on CTA pairs: 256 x 256 tiles with I <= J
};

constexpr int TC_MAX_SLOTS = 16;        // problems per grouped launch
// GEMM2 at small K: a (row block, direction) item split into up to
// G2_MAX_SPLIT parts over its j-tiles (at most G2_MAX_NJ tiles), parts * K <=
// G2_MAX_SPLIT so that the part sums fit the problem's part buffer
constexpr int G2_MAX_SPLIT = 4;
constexpr int G2_MAX_NJ = 64;

// Launch shape of the tensor-core contractions (chosen by the autotuner or
// the defaults): GEMM1 MMA width (128: square tiles with 1 or 2 directions;
// 256: 128 x 256 tiles, one direction; G1_PAIR: 256 x 256 tiles, one
// direction, on a CTA pair), directions per GEMM1 square tile,
// GEMM2 j-tile width (128, 256; G2_PAIR: 256-wide j-tiles over 256-row
// blocks on a CTA pair) and GEMM2 direction group (directions sharing one Psi
// row block: 1, 2, 4).
constexpr int G1_PAIR = 512;
constexpr int G2_PAIR = 512;           // g2_bn: 256-wide j-tiles on CTA pairs (256-row blocks)

struct TcTune {
  int g1_nb = G1_PAIR;
  int g1_dpt = 1;
  int g2_bn = G2_PAIR;
  int g2_kgroup = 4;
};

}  // namespace lrdm

namespace lrdm {

// One problem's share of a grouped launch (host side).
struct TcEntry {
  const TcProblem* dev_base = nullptr;   // device array of all problems of the context
  const TcProblem* host = nullptr;       // host copy of this problem
  int pid = 0;                           // index into the device array
  int K = 0;                             // directions this call
  void* X = nullptr;                     // GEMM1 output [split][K][ns_pad][ns_pad] FP32
  int split = 1;                         // GEMM1 grid-row ranges (partials summed by the consumers)
  double factor = 0.0;                   // GEMM2: out = factor * drho (- v)
  const void* v = nullptr;
  long long v_stride = 0;
  void* out = nullptr;
  long long out_stride = 0;
};

}  // namespace lrdm
