// Tensor-core fitting net (BF16 operands, FP32 accumulation).
#pragma once
#include <cuda_bf16.h>

#include "path.cuh"

namespace dpgb {

// BF16 copies of the hidden fitting layers' weights (both orientations) on the device.
int prepare_fit_bf16(DeviceModel& m, const double* params_host);

// Energies (and their FP64 sum) and dE/dD [N][M*M_<] (FP32) from the BF16 descriptor.
// dE/dD of every atom: FP32 into *gD_out, or BF16 into *gDh_out when that is given.
int run_fitting_tc(const DeviceModel& m, const PathConst& pc, const __nv_bfloat16* Dbf, const PathIO& io, Arena& ar,
                   cudaStream_t st, const float** gD_out, const __nv_bfloat16** gDh_out = nullptr);

}  // namespace dpgb
