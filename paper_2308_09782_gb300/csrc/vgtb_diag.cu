// vgtb_diag_split_chain: the two tcgen05 products on caller matrices (unit test hook).
#include <cuda_runtime.h>

#include <cstring>

#include <string>
#include <vector>

#include "../../include/vgtb.h"
#include "../../include/vgtb_diag.h"
#include "tc_kernel.cuh"
#include "vgtb_internal.h"
#include "vgtb_tc.h"

using namespace vgtb;

namespace {
struct Scratch {
  std::vector<void*> p;
  ~Scratch() {
    for (void* q : p) cudaFree(q);
  }
  template <class T>
  T* get(size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) return nullptr;
    cudaMemset(q, 0, n * sizeof(T));
    p.push_back(q);
    return (T*)q;
  }
};

void to_padded(const double* src, std::vector<double2>& dst, int n, int Np) {
  dst.assign((size_t)Np * Np, make_double2(0.0, 0.0));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) dst[(size_t)i * Np + j] = make_double2(src[2 * ((size_t)i * n + j)], src[2 * ((size_t)i * n + j) + 1]);
}
}  // namespace

extern "C" int vgtb_diag_split_chain(int n, const double* a, const double* r, const double* s, double* w_out,
                                     double* x_out) {
  return vgtb_diag_split_chain_variant(n, a, r, s, -1, w_out, x_out);
}

extern "C" int vgtb_diag_num_variants() { return tc_num_variants(); }

extern "C" int vgtb_diag_split_chain_variant(int n, const double* a, const double* r, const double* s, int variant,
                                             double* w_out, double* x_out) {
  if (variant >= tc_num_variants()) return VGTB_E_INVALID;
  if (n < 1 || !a || !r || !s || !w_out || !x_out) return VGTB_E_INVALID;
  if (!tc_gemm_supported()) return VGTB_E_UNSUPPORTED;
  const int Np = (n + 127) / 128 * 128;
  const size_t NN = (size_t)Np * Np;
  Scratch m;
  double2* dsrc = m.get<double2>(NN);
  __nv_bfloat16* a_p = m.get<__nv_bfloat16>(4 * NN);
  __nv_bfloat16* d0_p = m.get<__nv_bfloat16>(4 * NN);
  __nv_bfloat16* s_p = m.get<__nv_bfloat16>(4 * NN);
  __nv_bfloat16* r_e = m.get<__nv_bfloat16>(8 * NN);
  __nv_bfloat16* z_e = m.get<__nv_bfloat16>(8 * NN);
  __nv_bfloat16* w_e = m.get<__nv_bfloat16>(8 * NN);
  float* xf = m.get<float>(2 * NN);
  if (!dsrc || !a_p || !d0_p || !s_p || !r_e || !z_e || !w_e || !xf) return VGTB_E_NOMEM;
  cudaStream_t st = 0;
  std::vector<double2> h;
  to_padded(a, h, n, Np);
  cudaMemcpy(dsrc, h.data(), NN * sizeof(double2), cudaMemcpyHostToDevice);
  launch_split_planar(dsrc, a_p, n, Np, st);
  cudaDeviceSynchronize();
  to_padded(s, h, n, Np);
  cudaMemcpy(dsrc, h.data(), NN * sizeof(double2), cudaMemcpyHostToDevice);
  launch_split_planar(dsrc, s_p, n, Np, st);
  cudaDeviceSynchronize();
  to_padded(r, h, n, Np);
  cudaMemcpy(dsrc, h.data(), NN * sizeof(double2), cudaMemcpyHostToDevice);
  launch_split_embedded(dsrc, r_e, Np, st);
  if (cudaDeviceSynchronize() != cudaSuccess) return VGTB_E_CUDA;
  std::vector<TcSysView> views(1);
  views[0].Np = Np;
  views[0].nk = 1;
  views[0].n_items = 1;
  views[0].Sinv_p = s_p;
  views[0].D0_p = d0_p;
  views[0].dD_p = a_p;
  views[0].Hemb_p = r_e;
  views[0].dHemb_p = z_e;
  views[0].Wemb_p = w_e;
  std::vector<DevItem> items(1);
  memset(&items[0], 0, sizeof(DevItem));
  items[0].Wemb_p = w_e;
  items[0].Xf = xf;
  TcPlan *p1 = nullptr, *p2 = nullptr;
  std::string msg;
  const int force[2] = {variant, variant};
  if (tc_build_plans(views, items, 2000000000LL, 0, force, st, &p1, &p2, &msg)) return VGTB_E_CUDA;
  int rc = VGTB_OK;
  if (tc_launch(p1, st) || tc_launch(p2, st)) rc = VGTB_E_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) rc = VGTB_E_CUDA;
  if (rc == VGTB_OK && (tc_status(p1, st) || tc_status(p2, st))) rc = VGTB_E_TIMEOUT;
  tc_destroy_plan(p1);
  tc_destroy_plan(p2);
  if (rc != VGTB_OK) return rc;
  std::vector<__nv_bfloat16> we(8 * NN);
  std::vector<float> xh(2 * NN);
  cudaMemcpy(we.data(), w_e, 8 * NN * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost);
  cudaMemcpy(xh.data(), xf, 2 * NN * sizeof(float), cudaMemcpyDeviceToHost);
  const size_t ld = 2 * (size_t)Np, P = 4 * NN;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const size_t o = 2 * ((size_t)i * n + j);
      w_out[o] = (double)__bfloat162float(we[i * ld + j]) + (double)__bfloat162float(we[P + i * ld + j]);
      w_out[o + 1] = (double)__bfloat162float(we[i * ld + Np + j]) + (double)__bfloat162float(we[P + i * ld + Np + j]);
      x_out[o] = xh[i * ld + j];
      x_out[o + 1] = xh[i * ld + Np + j];
    }
  return VGTB_OK;
}

namespace {
__global__ void k_diag_convert(int n, const double* d_in, const float* f_in, float* fb, float* fr, double* db,
                               double* dr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  fb[i] = d2f_bits(d_in[i]);
  fr[i] = __double2float_rn(d_in[i]);
  db[i] = f2d_bits(f_in[i]);
  dr[i] = (double)f_in[i];
}
}  // namespace

extern "C" int vgtb_diag_convert(int n, const double* d_in, const float* f_in, float* f_bits, float* f_ref,
                                 double* d_bits, double* d_ref) {
  if (n < 0) return VGTB_E_INVALID;
  if (n == 0) return VGTB_OK;
  if (!d_in || !f_in || !f_bits || !f_ref || !d_bits || !d_ref) return VGTB_E_INVALID;
  Scratch sc;
  double* di = sc.get<double>(n);
  float* fi = sc.get<float>(n);
  float* fb = sc.get<float>(n);
  float* fr = sc.get<float>(n);
  double* db = sc.get<double>(n);
  double* dr = sc.get<double>(n);
  if (!di || !fi || !fb || !fr || !db || !dr) return VGTB_E_CUDA;
  if (cudaMemcpy(di, d_in, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(fi, f_in, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return VGTB_E_CUDA;
  k_diag_convert<<<(n + 255) / 256, 256>>>(n, di, fi, fb, fr, db, dr);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return VGTB_E_CUDA;
  if (cudaMemcpy(f_bits, fb, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(f_ref, fr, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(d_bits, db, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(d_ref, dr, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return VGTB_E_CUDA;
  return VGTB_OK;
}

namespace {
// One thread waits for an event that never happens, with the product kernels'
// bounded wait routines: mbar_wait on a phase nobody completes, or sk_wait_flag
// on a flag nobody sets.  Both give up after P.timeout_ns and set a bit of *P.err.
__global__ void k_diag_wait(const __grid_constant__ TcParams P, int which) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  bool ok;
  if (which == 0)
    ok = mbar_wait(b, 0, P.timeout_ns, &abort_flag, P.err);
  else
    ok = sk_wait_flag(P, 0, &abort_flag);
  if (ok) atomicOr(P.err, 16);  // the wait ended without its event
}
}  // namespace

extern "C" int vgtb_diag_bounded_wait(long long limit_ns, int which) {
  if ((which != 0 && which != 1) || limit_ns < 1 || limit_ns > 10000000000LL) return VGTB_E_INVALID;
  if (!tc_gemm_supported()) return VGTB_E_UNSUPPORTED;
  Scratch sc;
  int* err = sc.get<int>(1);
  int* flags = sc.get<int>(1);
  if (!err || !flags) return VGTB_E_CUDA;
  TcParams P;
  memset(&P, 0, sizeof(P));
  P.err = err;
  P.flags = flags;
  P.timeout_ns = limit_ns;
  k_diag_wait<<<1, 32>>>(P, which);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return VGTB_E_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return VGTB_E_CUDA;
  if (h & 16) return VGTB_OK;
  return (h & 3) ? VGTB_E_TIMEOUT : VGTB_E_CUDA;
}
