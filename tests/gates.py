"""Error gates of the GPU parity tests: relative w-norm error per direction
against the FP64 oracle (X_k: relative Frobenius error).

* FP64 1e-10 and split-BF16x3 1e-5 on f are the stated targets themselves;
  BF16x3 intermediates (X_k, drho_k, mu'_k) carry three error terms of up to
  2^-16 per product (the two operand splits and the dropped lo x lo product),
  so their bound is 3 * 2^-16 = 4.6e-5 -> 1e-4.
* FP32 on the CUDA cores: 1e-4 (FP32 accumulation over the grid).
* TF32 operands carry 10 mantissa bits (unit roundoff 2^-11 = 4.9e-4).  The
  error of f is the average of many such roundings and falls with the
  problem size; it meets the 1e-5 target only at the largest sizes tested.
  Each TF32 case has its own gate at about three times the error measured on
  GB300 (the table below), so that a regression well below the old blanket
  bound still fails, and every check prints the measured error and whether it
  meets 1e-5.
"""

from __future__ import annotations

TARGET = {"fp64": 1e-10, "bf16x3": 1e-5, "tf32": 1e-5}
TOL = {"fp64": 1e-10, "fp32": 1e-4, "bf16x3": 1e-5}
TOL_X = {"fp64": 1e-10, "fp32": 1e-4, "bf16x3": 1e-4}

# TF32 gates per (case, quantity): about 3x the largest error measured on
# GB300 for that case (in brackets).  X: relative Frobenius error of X_k (the
# operand rounding, 3.5-4.1e-4 in every case); dmu: |mu' error| / max |X_ii|.
TF32 = {
    "projection_ragged_tiles:X": 1.2e-3,                  # [3.60e-4]
    "projection_and_forward_odd_block_count:X": 1.2e-3,   # [3.61e-4]
    "projection_and_forward_odd_block_count:f": 4e-4,     # [1.34e-4]
    "small_k_row_range_split:X": 1.2e-3,                  # [3.59e-4]
    "small_k_row_range_split:f": 3.5e-5,                  # [1.12e-5]
    "small_k_row_range_split:dmu": 8e-5,                  # [2.65e-5]
    "forward_toy16:f": 5e-4,                              # [1.61e-4]
    "forward_toy16:dmu": 3.3e-5,                          # [1.08e-5]
    "forward_ragged_tiles:f": 3.2e-4,                     # [1.05e-4]
    "forward_ragged_tiles:X": 1.3e-3,                     # [4.05e-4] (drho)
    "forward_ragged_tiles:dmu": 2.2e-4,                   # [7.27e-5]
    "batched_uneven_equals_separate:f": 1.5e-3,           # [4.74e-4]
    "forced_launch_shapes:f": 1.5e-3,                     # [4.74e-4]
    "forced_launch_shapes:X": 1.3e-3,                     # (Frobenius, as elsewhere)
    "maximum_directions:f": 5e-4,                         # [1.58e-4]
    "maximum_directions:dmu": 1.2e-3,                     # [3.71e-4]
    "response_split_over_j_tiles:f": 1.6e-4,              # [5.08e-5]
    "pair_projection_tiles:X": 1.2e-3,                    # [3.66e-4]
    "pair_projection_tiles:f": 4e-4,                      # [1.29e-4]
    "pair_projection_tiles:dmu": 2.2e-4,                  # [7.26e-5]
    "pair_projection_small_k_and_batch:X": 1.2e-3,        # [3.54e-4]
    "pair_projection_small_k_and_batch:f": 1.5e-3,        # [4.74e-4]
    "precision_72cube:f": 3e-5,                           # [9.78e-6]
    "single_system_48cube:f": 3.5e-5,                     # [1.16e-5]
    "single_system_48cube:dmu": 4e-5,                     # [1.32e-5]
    "kpoint_gateaux_matches_oracle:f": 7e-4,              # [2.26e-4] (f and drho)
    "kpoint_tensor_cores_edge_cases:f": 5.5e-4,           # [1.76e-4]
    "pair_response_tiles:f": 4e-4,                        # [1.19e-4]
    "pair_response_tiles:X": 9e-4,                        # [2.88e-4] (drho)
    "pair_response_split_and_batch:f": 1.5e-3,            # [4.74e-4]
    "sampled_rows_96cube:f": 1.5e-5,                      # [5.00e-6] (96^3 / 4096 / 16)
    "sampled_rows_96cube:dmu": 9e-5,                      # [2.96e-5]
}
# until a case is measured (not expected in a committed table)
TF32_UNMEASURED = 5e-3


def gate(prec: str, case: str, what: str = "f") -> float:
    if prec != "tf32":
        return (TOL if what == "f" else TOL_X)[prec]
    return TF32.get(f"{case}:{what}", TF32_UNMEASURED)


def check(prec: str, case: str, err: float, what: str = "f", factor: float = 1.0) -> None:
    """assert err < factor * gate, printing the comparison."""
    g = factor * gate(prec, case, what)
    note = ""
    if prec == "tf32":
        if what == "f":
            hit = "meets" if err <= TARGET["tf32"] else "misses"
            note = f" ({hit} the 1e-5 target)"
        if f"{case}:{what}" not in TF32:
            note += " [tf32 gate unmeasured]"
    print(f"[gate] {prec} {case}:{what} err {err:.3e} < {g:.1e}{note}")
    assert err < g, f"{prec} {case}:{what}: error {err:.3e} not below its gate {g:.1e}"
