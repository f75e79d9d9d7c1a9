// Per-pair environment quantities shared by the path kernels: Eq. (switch) and the unit
// vector of r_ij, evaluated in the path's precision.
#pragma once
#include "path.cuh"

namespace dpgb {

template <class R>
__device__ __forceinline__ void switch_eval(R r, R rs, R rc, R& s, R& ds) {
  if (r < rs) {
    s = R(1) / r;
    ds = -s / r;
  } else if (r >= rc) {
    s = R(0);
    ds = R(0);
  } else {
    const R w = rc - rs;
    const R x = (r - rs) / w;
    const R u = x * x * x * (R(-6) * x * x + R(15) * x - R(10)) + R(1);
    const R du = R(-30) * x * x * (x - R(1)) * (x - R(1)) / w;
    s = u / r;
    ds = -u / (r * r) + du / r;
  }
}

// r, s(r), ds/dr and the unit vector of one pair, in the path's precision.
template <class R>
__device__ __forceinline__ void pair_env(double d0, double d1, double d2, double r2, double rs, double rc,
                                         double near2, R& r, R& s, R& ds, R* u);

template <>
__device__ __forceinline__ void pair_env<double>(double d0, double d1, double d2, double r2, double rs, double rc,
                                                 double, double& r, double& s, double& ds, double* u) {
  r = sqrt(r2);
  switch_eval<double>(r, rs, rc, s, ds);
  const double ir = 1.0 / r;
  u[0] = d0 * ir;
  u[1] = d1 * ir;
  u[2] = d2 * ir;
}

template <>
__device__ __forceinline__ void pair_env<float>(double d0, double d1, double d2, double r2, double rs, double rc,
                                                double near2, float& r, float& s, float& ds, float* u) {
  if (r2 >= near2) {
    const double rd = sqrt(r2);
    double sd, dsd;
    switch_eval<double>(rd, rs, rc, sd, dsd);
    r = (float)rd;
    s = (float)sd;
    ds = (float)dsd;
    const double ir = 1.0 / rd;
    u[0] = (float)(d0 * ir);
    u[1] = (float)(d1 * ir);
    u[2] = (float)(d2 * ir);
  } else {
    r = sqrtf((float)r2);
    switch_eval<float>(r, (float)rs, (float)rc, s, ds);
    const float ir = 1.0f / r;
    u[0] = (float)d0 * ir;
    u[1] = (float)d1 * ir;
    u[2] = (float)d2 * ir;
  }
}


__device__ __forceinline__ int slot_block(const PathConst& pc, int k) {
  int t = 0;
  while (t + 1 < pc.ntypes && k >= pc.sel_off[t + 1]) ++t;
  return t;
}

__device__ __forceinline__ int net_of(const PathConst& pc, int ti, int tj) {
  return pc.type_one_side ? tj : ti * pc.ntypes + tj;
}

}  // namespace dpgb
