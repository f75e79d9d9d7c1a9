// Compressed embedding contraction and its backward on the tensor cores (mom.cu).
#pragma once
#include "path.cuh"

namespace dpgb {

// Output width padded for the moment kernels (16, 32, 64, 112 or 128; 0 if M > 128).
int mom_npad_of(int M);
// Whether a compressed model runs its embedding contraction on the tensor cores: FP32 or the
// mixed (BF16) precision, M <= 128 and M_< <= 16.
bool mom_supported(const DeviceModel& m);
// FP16 (mixed) or BF16 high/low (FP32) operand tables and their tensor maps; needs the FP64
// quintic tables.  No-op for models the moment path does not cover.
int build_mom_tables(DeviceModel& m);
// Energy, forces and virial with the moment kernels (env rows, T and D, fitting, backward).
int run_mom(const DeviceModel& m, const PathConst& pc, const PathIO& io, Arena& ar, cudaStream_t st);

}  // namespace dpgb
