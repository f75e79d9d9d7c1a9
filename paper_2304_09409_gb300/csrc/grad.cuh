// Parameter gradient of an energy + force objective (grad.cu).
#pragma once
#include "path.cuh"

namespace dpgb {

// Offset of each embedding net's first-layer weights in the flat parameter array.
struct NetOffsets {
  int nets;
  long w[kMaxNets];
};

// dPhi/dtheta for Phi = sum_f a_f E_f + b * D E, D E the derivative of E along the pair-displacement
// tangent dr_ij = (w_j - w_i) + g_f r_ij (b = -1 gives sum_f a_f E_f + sum_i w_i . F_i +
// sum_f g_f : Xi_f), into `grad` [n_params] FP64 (device).  a_dev [frames], w_dev [N][3] (input
// atom order), gv_dev [frames][9] (row-major g_ab, or null) are device arrays.  Uncompressed
// FP64 / FP32 models.  With ar.measure set, only sizes the scratch.
int run_param_grad(const DeviceModel& m, const PathConst& pc, const PathIO& io, const double* w_dev,
                   const double* a_dev, const double* gv_dev, double b, double* grad, Arena& ar, cudaStream_t st);

}  // namespace dpgb
