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

// FP32 form from an FP32 displacement.  Near r_c the polynomial of Eq. (switch) is evaluated in
// the equivalent form 1 - x^3 (6x^2 - 15x + 10) = y^3 (6y^2 - 15y + 10) with
// y = 1 - x = (r_c - r)/(r_c - r_s), which has no cancellation as r -> r_c, so FP32 keeps full
// relative precision there.
__device__ __forceinline__ void pair_env_f32(float x0, float x1, float x2, double rs, double rc, float& r, float& s,
                                             float& ds, float* u) {
  r = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));  // explicit: the same rounding at every call site
  const float frs = (float)rs, frc = (float)rc;
  if (r < frs) {
    s = 1.0f / r;
    ds = -s / r;
  } else if (r >= frc) {
    s = 0.0f;
    ds = 0.0f;
  } else {
    const float w = frc - frs;
    const float y = (frc - r) / w;
    const float y3 = y * y * y;
    const float uu = y3 * ((6.0f * y - 15.0f) * y + 10.0f);
    const float du_dy = 30.0f * y * y * (y - 1.0f) * (y - 1.0f);
    s = uu / r;
    ds = -uu / (r * r) - du_dy / (w * r);
  }
  const float ir = 1.0f / r;
  u[0] = x0 * ir;
  u[1] = x1 * ir;
  u[2] = x2 * ir;
}

// The same with one reciprocal square root and no division (inv_w = 1 / (r_c - r_s)): a few ulps
// of FP32, for the moment path, whose values go on as FP16 or split-BF16 tensor-core operands.
__device__ __forceinline__ void pair_env_f32_fast(float x0, float x1, float x2, float frs, float frc, float inv_w,
                                                  float& r, float& s, float& ds, float* u) {
  const float r2 = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
  const float ir = rsqrtf(r2);
  r = r2 * ir;
  if (r < frs) {
    s = ir;
    ds = -ir * ir;
  } else if (r >= frc) {
    s = 0.0f;
    ds = 0.0f;
  } else {
    const float y = (frc - r) * inv_w;
    const float y3 = y * y * y;
    const float uu = y3 * fmaf(fmaf(6.0f, y, -15.0f), y, 10.0f);
    const float du_dy = 30.0f * y * y * (y - 1.0f) * (y - 1.0f);
    s = uu * ir;
    ds = -(uu * ir) * ir - du_dy * inv_w * ir;
  }
  u[0] = x0 * ir;
  u[1] = x1 * ir;
  u[2] = x2 * ir;
}

// FP32 form from the exact FP64 displacement (which cancels large coordinates).
template <>
__device__ __forceinline__ void pair_env<float>(double d0, double d1, double d2, double, double rs, double rc,
                                                double, float& r, float& s, float& ds, float* u) {
  pair_env_f32((float)d0, (float)d1, (float)d2, rs, rc, r, s, ds, u);
}

// FP32 -> FP64 widening with integer operations: exact for normal numbers (subnormals flush to
// zero), and it keeps the conversion off GB300's narrow FP64 pipe.
__device__ __forceinline__ double widen_f32(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu;
  unsigned long long bits = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0xFFu)
    bits |= 0x7FF0000000000000ull | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  else if (e != 0u)
    bits |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(float x) { return widen_f32(x); }
__device__ __forceinline__ double widen(double x) { return x; }

// Frame of atom i and that frame's cell rows / image-shift table.
__device__ __forceinline__ int frame_of(const PathConst& pc, int i) { return pc.atom_frame ? pc.atom_frame[i] : 0; }

// Exact FP64 displacement of a listed pair of frame fr; the same-image case needs no shift term.
__device__ __forceinline__ void listed_disp(const double* __restrict__ xi, const double* __restrict__ xj, int code,
                                            const PathConst& pc, int fr, double& d0, double& d1, double& d2) {
  int n0, n1, n2;
  unpack_shift(code, n0, n1, n2);
  if ((n0 | n1 | n2) == 0) {
    d0 = __dsub_rn(xj[0], xi[0]);
    d1 = __dsub_rn(xj[1], xi[1]);
    d2 = __dsub_rn(xj[2], xi[2]);
  } else if (pc.tshift && n0 >= -1 && n0 <= 1 && n1 >= -1 && n1 <= 1 && n2 >= -1 && n2 <= 1) {
    // t(n) precomputed with the builder's formula: (x_j + t) - x_i, bit for bit
    const double* t = pc.tshift + (long)fr * 81 + 3 * ((n0 + 1) * 9 + (n1 + 1) * 3 + (n2 + 1));
    d0 = __dsub_rn(__dadd_rn(xj[0], t[0]), xi[0]);
    d1 = __dsub_rn(__dadd_rn(xj[1], t[1]), xi[1]);
    d2 = __dsub_rn(__dadd_rn(xj[2], t[2]), xi[2]);
  } else {
    const double* h = pc.boxes ? pc.boxes + 9L * fr : pc.h;
    pair_disp_exact(xi, xj, n0, n1, n2, h, pc.periodic, d0, d1, d2);
  }
}

__device__ __forceinline__ int slot_block(const PathConst& pc, int k) {
  int t = 0;
  while (t + 1 < pc.ntypes && k >= pc.sel_off[t + 1]) ++t;
  return t;
}

// List slot read by slot k of the current part (the same position in the same type block).
__device__ __forceinline__ int list_slot(const PathConst& pc, int k) {
  const int t = slot_block(pc, k);
  return pc.lsel_off[t] + (k - pc.sel_off[t]);
}

__device__ __forceinline__ int net_of(const PathConst& pc, int ti, int tj) {
  return pc.type_one_side ? tj : ti * pc.ntypes + tj;
}

}  // namespace dpgb
