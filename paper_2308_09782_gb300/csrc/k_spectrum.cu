// Post-propagation reductions on the device series of a trajectory:
//   k_conductivity - sigma_i(w) = (1/E0) int_0^T e^{iwt} J_i(t) e^{-t/tau0} dt and
//                    eps_i(w) = 1 + 4 pi i sigma_i(w) / w   (Eqs. 15, 16),
//                    trapezoid rule on the levels t = (n - n0) dt, one CTA per w;
//   k_group_charge - Q_g(t_n) - Q_g(t_0) with Q_I = -(q_I - Z_I) summed over an
//                    atom group (charge transfer between atom classes, Sec. 3.3),
//                    one CTA per stored level.
// Fixed-order block reductions: results are bitwise reproducible.
#include "vgtb_internal.h"

namespace vgtb {

constexpr int kSpecThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int s = kSpecThreads / 2; s > 0; s >>= 1) {
    if (tid < s) sh[tid] += sh[tid + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSpecThreads) k_conductivity(const double* __restrict__ J, int n0, int n1, double dt,
                                                               double e0, double tau0,
                                                               const double* __restrict__ omega, double* sigma,
                                                               double* eps) {
  __shared__ double sh[kSpecThreads];
  const double w = omega[blockIdx.x];
  double acc[6] = {0, 0, 0, 0, 0, 0};  // (re, im) for x, y, z
  for (int n = n0 + threadIdx.x; n <= n1; n += kSpecThreads) {
    const double t = (n - n0) * dt;
    const double wt = (n == n0 || n == n1) ? 0.5 * dt : dt;
    const double f = wt * exp(-t / tau0);
    double s, c;
    sincos(w * t, &s, &c);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double j = f * J[3LL * n + a];
      acc[2 * a] += c * j;
      acc[2 * a + 1] += s * j;
    }
  }
  for (int i = 0; i < 6; ++i) acc[i] = block_sum(acc[i], sh);
  if (threadIdx.x == 0) {
    const double k = 4.0 * M_PI / w;
    for (int a = 0; a < 3; ++a) {
      const double sr = acc[2 * a] / e0, si = acc[2 * a + 1] / e0;
      double* so = sigma + 6LL * blockIdx.x + 2 * a;
      so[0] = sr;
      so[1] = si;
      double* eo = eps + 6LL * blockIdx.x + 2 * a;
      eo[0] = 1.0 - k * si;  // 1 + 4 pi i (sr + i si) / w
      eo[1] = k * sr;
    }
  }
}

void launch_conductivity(const double* J, int n0, int n1, double dt, double e0, double tau0, const double* omega,
                         int n_omega, double* sigma, double* eps, cudaStream_t st) {
  k_conductivity<<<n_omega, kSpecThreads, 0, st>>>(J, n0, n1, dt, e0, tau0, omega, sigma, eps);
}

__global__ void __launch_bounds__(kSpecThreads) k_group_charge(const double* __restrict__ q, int nat,
                                                               const int* __restrict__ group, int n_groups,
                                                               double* out) {
  __shared__ double sh[kSpecThreads];
  const double* ql = q + (long long)blockIdx.x * nat;
  for (int g = 0; g < n_groups; ++g) {
    double v = 0.0;
    for (int I = threadIdx.x; I < nat; I += kSpecThreads)
      if (group[I] == g) v += -(ql[I] - q[I]);  // Q_I(t) - Q_I(0) with Q_I = -(q_I - Z_I)
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[(long long)blockIdx.x * n_groups + g] = v;
  }
}

void launch_group_charge(const double* q, int nat, const int* group, int n_groups, int n_levels, double* out,
                         cudaStream_t st) {
  k_group_charge<<<n_levels, kSpecThreads, 0, st>>>(q, nat, group, n_groups, out);
}

}  // namespace vgtb
