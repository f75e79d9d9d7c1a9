// Model deviation of an ensemble of models on one frame (Sec. II.C).
//
// Every model of the ensemble evaluates the frame (the models' own kernels, one after the other
// on the caller's stream, coordinates uploaded once); then one kernel forms, per atom, the
// ensemble mean force <F_i> and the deviation
//   eps_F,i = sqrt( < |F_i(theta_k) - <F_i>|^2 > )     (<.>: mean over the n_m models)
// (or its relative form eps_F,i / (|<F_i>| + nu)) with per-block partial maximum, minimum and sum,
// and a second kernel reduces the partials in a fixed order and forms the virial deviation
//   eps_Xi,ab = (1/N) sqrt( < (Xi_ab(theta_k) - <Xi_ab>)^2 > )
// (relative form: divided by |<Xi>| + nu, |.| the Frobenius norm) with its maximum, mean and
// minimum over the nine components.  All of it in FP64.
#include <algorithm>

#include "capi_internal.cuh"

namespace dpgb {

namespace {

constexpr int kDeviThreads = 256;

__global__ void __launch_bounds__(kDeviThreads)
    k_devi_force(const double* __restrict__ F, int nm, int N, double nu, double* __restrict__ devi,
                 double* __restrict__ fmean, double* __restrict__ part) {
  __shared__ double s_max[kDeviThreads / 32], s_min[kDeviThreads / 32], s_sum[kDeviThreads / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0, emax = 0.0, emin = 1e300, esum = 0.0;
  if (i < N) {
    double m[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < nm; ++k)
      for (int a = 0; a < 3; ++a) m[a] += F[((long)k * N + i) * 3 + a];
    for (int a = 0; a < 3; ++a) m[a] /= nm;
    double v = 0.0;
    for (int k = 0; k < nm; ++k)
      for (int a = 0; a < 3; ++a) {
        const double d = F[((long)k * N + i) * 3 + a] - m[a];
        v += d * d;
      }
    e = sqrt(v / nm);
    if (nu > 0.0) e /= sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) + nu;
    if (devi) devi[i] = e;
    if (fmean)
      for (int a = 0; a < 3; ++a) fmean[3L * i + a] = m[a];
    emax = emin = esum = e;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    emin = fmin(emin, __shfl_xor_sync(0xffffffffu, emin, off));
    esum += __shfl_xor_sync(0xffffffffu, esum, off);
  }
  if (lane == 0) {
    s_max[w] = emax;
    s_min[w] = emin;
    s_sum[w] = esum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = s_max[0], b = s_min[0], c = s_sum[0];
    for (int k = 1; k < kDeviThreads / 32; ++k) {
      a = fmax(a, s_max[k]);
      b = fmin(b, s_min[k]);
      c += s_sum[k];
    }
    part[3L * blockIdx.x] = a;
    part[3L * blockIdx.x + 1] = b;
    part[3L * blockIdx.x + 2] = c;
  }
}

// One block: the partials in a fixed order, then the virial deviation (threads 0..8).
__global__ void k_devi_final(const double* __restrict__ part, int nblk, const double* __restrict__ V, int nm, int N,
                             double nu, double* __restrict__ devi_v, double* __restrict__ stats) {
  __shared__ double s_v[9];
  const int t = threadIdx.x;
  if (t == 0) {
    double a = 0.0, b = 1e300, c = 0.0;
    for (int k = 0; k < nblk; ++k) {
      a = fmax(a, part[3L * k]);
      b = fmin(b, part[3L * k + 1]);
      c += part[3L * k + 2];
    }
    stats[0] = a;
    stats[1] = c / N;
    stats[2] = b;
  }
  if (t < 9) {
    double m = 0.0;
    for (int k = 0; k < nm; ++k) m += V[9L * k + t];
    m /= nm;
    double v = 0.0;
    for (int k = 0; k < nm; ++k) {
      const double d = V[9L * k + t] - m;
      v += d * d;
    }
    s_v[t] = sqrt(v / nm) / N;
    if (nu > 0.0) {  // |<Xi>| + nu, the Frobenius norm of the mean virial
      double n2 = 0.0;
      for (int q = 0; q < 9; ++q) {
        double mq = 0.0;
        for (int k = 0; k < nm; ++k) mq += V[9L * k + q];
        mq /= nm;
        n2 += mq * mq;
      }
      s_v[t] /= sqrt(n2) + nu;
    }
    devi_v[t] = s_v[t];
  }
  __syncthreads();
  if (t == 0) {
    double a = s_v[0], b = s_v[0], c = 0.0;
    for (int q = 0; q < 9; ++q) {
      a = fmax(a, s_v[q]);
      b = fmin(b, s_v[q]);
      c += s_v[q];
    }
    stats[3] = a;
    stats[4] = c / 9.0;
    stats[5] = b;
  }
}

}  // namespace
}  // namespace dpgb

using namespace dpgb;

extern "C" int dp_model_deviation(dp_model** models, int nmodels, int natoms, const double* coord, const int* type,
                                  const double* box, double nu, double* devi_f, double* devi_v, double* stats,
                                  double* force_mean, void* stream) {
  if (!models || nmodels < 2 || natoms < 1 || !coord || !type || !stats || nu < 0.0) {
    set_error("dp_model_deviation: at least two models, one atom, coordinates, types and stats are needed");
    return DP_E_ARG;
  }
  for (int k = 0; k < nmodels; ++k)
    if (!models[k] || models[k]->m.device != models[0]->m.device) {
      set_error("dp_model_deviation: every model must exist and live on the same device");
      return DP_E_ARG;
    }
  DP_CUDA_TRY(cudaSetDevice(models[0]->m.device));
  cudaStream_t st = (cudaStream_t)stream;
  const long N = natoms;
  const bool host_c = !is_device_ptr(coord), host_t = !is_device_ptr(type);
  if (host_c) {
    const int rc = check_finite_host(coord, 3 * N);
    if (rc != DP_OK) return rc;
  }
  const int nblk = (int)((N + kDeviThreads - 1) / kDeviThreads);
  // device work space: the ensemble's forces, virials and energies, the inputs when they are
  // host arrays, the per-atom outputs and the partials (one allocation, stream ordered)
  const size_t nF = (size_t)nmodels * N * 3, nV = 9 * (size_t)nmodels;
  const size_t bytes = sizeof(double) * (nF + nV + nmodels + (host_c ? 3 * N : 0) + N + 3 * N + 3 * nblk + 9 + 6) +
                       sizeof(int) * (host_t ? N : 0) + 1024;
  char* ws = nullptr;
  DP_CUDA_TRY(cudaMallocAsync(&ws, bytes, st));
  size_t off = 0;
  auto take = [&](size_t b) {
    char* p = ws + off;
    off += (b + 255) & ~(size_t)255;
    return p;
  };
  double* dF = reinterpret_cast<double*>(take(sizeof(double) * nF));
  double* dV = reinterpret_cast<double*>(take(sizeof(double) * nV));
  double* dE = reinterpret_cast<double*>(take(sizeof(double) * nmodels));
  double* dC = host_c ? reinterpret_cast<double*>(take(sizeof(double) * 3 * N)) : const_cast<double*>(coord);
  int* dT = host_t ? reinterpret_cast<int*>(take(sizeof(int) * N)) : const_cast<int*>(type);
  double* dDevi = reinterpret_cast<double*>(take(sizeof(double) * N));
  double* dMean = reinterpret_cast<double*>(take(sizeof(double) * 3 * N));
  double* dPart = reinterpret_cast<double*>(take(sizeof(double) * 3 * nblk));
  double* dDv = reinterpret_cast<double*>(take(sizeof(double) * 9));
  double* dStats = reinterpret_cast<double*>(take(sizeof(double) * 6));
  int rc = DP_OK;
  cudaError_t e = cudaSuccess;
  if (host_c) e = cudaMemcpyAsync(dC, coord, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && host_t) e = cudaMemcpyAsync(dT, type, sizeof(int) * N, cudaMemcpyHostToDevice, st);
  for (int k = 0; e == cudaSuccess && k < nmodels; ++k) {
    const int r = dp_compute(models[k], nullptr, natoms, dC, dT, box, dE + k, dF + (size_t)k * N * 3, dV + 9L * k,
                             nullptr, stream);
    if (r != DP_OK && r != DP_E_SEL_OVERFLOW && r != DP_E_RANGE) {
      rc = r;
      break;
    }
  }
  if (e == cudaSuccess && rc == DP_OK) {
    k_devi_force<<<nblk, kDeviThreads, 0, st>>>(dF, nmodels, natoms, nu, dDevi, dMean, dPart);
    k_devi_final<<<1, 32, 0, st>>>(dPart, nblk, dV, nmodels, natoms, nu, dDv, dStats);
    e = cudaGetLastError();
    auto out = [&](double* dst, const double* src, size_t n) {
      if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDefault, st);
    };
    out(devi_f, dDevi, N);
    out(devi_v, dDv, 9);
    out(stats, dStats, 6);
    out(force_mean, dMean, 3 * N);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFreeAsync(ws, st);
  if (e != cudaSuccess) {
    set_error(std::string("dp_model_deviation: ") + cudaGetErrorString(e));
    return DP_E_CUDA;
  }
  return rc;
}
