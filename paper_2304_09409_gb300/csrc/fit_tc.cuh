// Tensor-core fitting net (BF16 operands, FP32 accumulation).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "path.cuh"

namespace dpgb {

// BF16 copies of the hidden fitting layers' weights (both orientations) on the device; with
// `split` also their low halves W - bf16(W) for the three-pass products of the FP32 mode.
int prepare_fit_bf16(DeviceModel& m, const double* params_host, bool split = false);
// The hidden fitting layers fit the tensor-core kernels (widths multiples of 16 and <= 256,
// inputs multiples of 8, skips of kind 0 or 1, no skip on the first layer).
bool fit_tc_supported(const DeviceModel& m);

// Energies (and their FP64 sum) and dE/dD [N][M*M_<] (FP32) from the BF16 descriptor.
// Tensor map of fitting layer l of type t (dir 0: W^T [n_out][n_in], dir 1: W [n_in][n_out]),
// box of 64 columns x box_rows rows, cached on the model.
// lo selects the low halves (split operands).
const CUtensorMap* fit_weight_map(const DeviceModel& m, int t, int l, int dir, int box_rows, bool lo = false);
// The whole fitting net (forward to E_i, backward to dE/dD in BF16) in one kernel per 128-atom
// tile, for nets of at most four hidden layers of width <= 256 (multiples of 16) with skips of
// kind 0 or 1.
bool fit_fused_supported(const DeviceModel& m);
int run_fitting_fused(const DeviceModel& m, const PathConst& pc, const __nv_bfloat16* Dbf, const PathIO& io,
                      Arena& ar, cudaStream_t st, const __nv_bfloat16** gDh_out);

// The whole FP32-mode fitting net in one kernel per 128-atom tile on split BF16 operands (three
// passes), for nets of at most four hidden layers of width <= 256 (multiples of 16) with skips of
// kind 0 or 1; Dhi / Dlo the descriptor's high and low halves; dE/dD FP32 [rows][KD].  With Tm
// (T [rows][M][4]) and gT given and M_< = 16, dE/dD is not stored: the kernel forms dE/dT of the
// se_e2_a contraction into gT (m-major [M][rows][4]) and *gD_out is set to null.
bool fit_split_supported(const DeviceModel& m);
int run_fitting_split(const DeviceModel& m, const PathConst& pc, const __nv_bfloat16* Dhi, const __nv_bfloat16* Dlo,
                      const PathIO& io, Arena& ar, cudaStream_t st, const float** gD_out, const float* Tm = nullptr,
                      float* gT = nullptr);

// dE/dD of every atom: FP32 [rows][KD] into *gD_out, or BF16 into *gDh_out when that is given.
// With Dlo (the low halves of the descriptor, FP32 mode) every GEMM runs on split operands
// (three passes, hi.hi + hi.lo + lo.hi) and dE/dD is FP32.
// The BF16 array is tile-blocked: the rows of each type form tiles of 128 from the type's first
// row; tile rows [row0, row0 + nr) occupy [row0 * KD, (row0 + nr) * KD) and element (row0 + r, col)
// sits at ((col / 8) * nr + r) * 8 + col % 8 within it (8-column groups, rows contiguous), so
// thread-per-row epilogues write whole 512-byte runs per warp.
// Tm / gT as for run_fitting_split: used when the split kernel runs (then *gD_out is null and gT holds
// dE/dT), ignored otherwise.
int run_fitting_tc(const DeviceModel& m, const PathConst& pc, const __nv_bfloat16* Dbf, const PathIO& io, Arena& ar,
                   cudaStream_t st, const float** gD_out, const __nv_bfloat16** gDh_out = nullptr,
                   const __nv_bfloat16* Dlo = nullptr, const float* Tm = nullptr, float* gT = nullptr);

}  // namespace dpgb
