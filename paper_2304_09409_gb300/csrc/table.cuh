// Compressed embedding (Eq. (compress)): table construction and the fused path.
#pragma once
#include "path.cuh"

namespace dpgb {

// Build the quintic tables of every embedding net on the model's device (FP64, plus an
// FP32 copy).  Layout: [net][interval][coefficient a..f][M] so that a warp reading one
// coefficient for consecutive outputs m issues one coalesced load.
int build_tables(DeviceModel& m);

// Copy the tables to host in the oracle's layout [net][interval][M][6] (tests).
int export_tables(const DeviceModel& m, double* out);

// Energy, forces and virial with the tabulated embedding fused with G^T R.
int run_compressed(const DeviceModel& m, const PathConst& pc, const PathIO& io, Arena& ar, cudaStream_t st);

}  // namespace dpgb
