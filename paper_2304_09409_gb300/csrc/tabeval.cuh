// Evaluation of the quintic tables of Eq. (compress), shared by the compressed kernels: the
// node grid (stride1 on [x0, split), stride2 on [split, xmax]), the interval of an argument, and a
// piece's value and slope at t = x - x_l.  Table layout [net][interval][output][kCoefStride] with
// the coefficients a..f padded to eight values (two 16-byte loads in FP32).
#pragma once
#include "dp_internal.cuh"

namespace dpgb {

struct TabConst {
  double s0, stride1, stride2, split, smax;
  int n1, n2, lc;
};

// Coefficients of one (interval, output) pair: a..f padded to 8 values (two 16-byte loads in
// FP32), table layout [net][interval][output][8].
constexpr int kCoefStride = 8;

inline TabConst tab_const(const DeviceModel& m) {
  TabConst c;
  c.s0 = m.tab.s0;
  c.stride1 = m.tab.stride1;
  c.stride2 = m.tab.stride2;
  c.n1 = m.tab.n1;
  c.n2 = m.tab.n2;
  c.lc = c.n1 + c.n2;
  c.split = c.s0 + c.n1 * c.stride1;
  c.smax = c.split + c.n2 * c.stride2;
  return c;
}

__host__ __device__ inline double node_at(const TabConst& c, int l) {
  return l <= c.n1 ? c.s0 + l * c.stride1 : c.s0 + c.n1 * c.stride1 + (l - c.n1) * c.stride2;
}

// One interval's coefficients of one output, loaded with 16-byte vector loads.
template <class R>
struct Quint {
  R a, b, c, d, e, f;
};
__device__ __forceinline__ Quint<float> load_quint(const float* __restrict__ p) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  const float4 y = *reinterpret_cast<const float4*>(p + 4);
  return Quint<float>{x.x, x.y, x.z, x.w, y.x, y.y};
}
__device__ __forceinline__ Quint<double> load_quint(const double* __restrict__ p) {
  const double2 x = reinterpret_cast<const double2*>(p)[0];
  const double2 y = reinterpret_cast<const double2*>(p)[1];
  const double2 z = reinterpret_cast<const double2*>(p)[2];
  return Quint<double>{x.x, x.y, y.x, y.y, z.x, z.y};
}
template <class R>
__device__ __forceinline__ R quint_value(const Quint<R>& q, R t) {
  return ((((q.a * t + q.b) * t + q.c) * t + q.d) * t + q.e) * t + q.f;
}
template <class R>
__device__ __forceinline__ R quint_slope(const Quint<R>& q, R t) {
  return (((R(5) * q.a * t + R(4) * q.b) * t + R(3) * q.c) * t + R(2) * q.d) * t + q.e;
}

template <class R>
__device__ __forceinline__ int tab_interval(const TabConst& tc, R s, R& tt, bool& oor) {
  int l;
  if (s < R(tc.split)) {
    l = (int)floor((s - R(tc.s0)) * R(1.0 / tc.stride1));
    l = l < 0 ? 0 : (l > tc.n1 - 1 ? tc.n1 - 1 : l);
    tt = s - (R(tc.s0) + R(l) * R(tc.stride1));
  } else {
    l = tc.n1 + (int)floor((s - R(tc.split)) * R(1.0 / tc.stride2));
    if (l > tc.lc - 1) l = tc.lc - 1;
    tt = s - (R(tc.split) + R(l - tc.n1) * R(tc.stride2));
    if (s > R(tc.smax)) oor = true;
  }
  return l;
}


}  // namespace dpgb
