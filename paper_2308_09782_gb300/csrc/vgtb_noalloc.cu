// vgtb_split_cgemm_noalloc: the tcgen05 BF16x3 complex product C = A R^dagger
// for callers that cannot allocate device memory.
//
// All scratch (the BF16 hi/lo pieces of A and of the embedded R, the FP32
// product, the one-entry problem table and the error word) lives in one
// file-scope static __device__ array of fixed size, so a call performs no
// cudaMalloc, cudaFree or allocating library call.  Host code cannot pass the
// array's name to a kernel (in host code it is only a stand-in, not a device
// address): the first call on each device looks the address up with
// cudaGetSymbolAddress and keeps it together with the identity of the CUDA
// context it belongs to; a call made under another context of that device (after
// cudaDeviceReset, say) repeats the set-up.  The set-up runs under a mutex, so
// first calls from several host threads do not race on the cached values.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/vgtb.h"
#include "tc_kernel.cuh"

namespace vgtb {
namespace {

constexpr int kNaMaxN = 256;                                        // largest supported n
constexpr size_t kNaPieceA = 2ull * kNaMaxN * (2 * kNaMaxN);        // BF16 elements, planar pieces of A
constexpr size_t kNaPieceR = 2ull * (2 * kNaMaxN) * (2 * kNaMaxN);  // BF16 elements, embedded pieces of R
constexpr size_t kNaOut = (size_t)kNaMaxN * (2 * kNaMaxN);          // FP32 elements, planar product
constexpr size_t kOffA = 0;
constexpr size_t kOffR = kOffA + kNaPieceA * 2;
constexpr size_t kOffOut = kOffR + kNaPieceR * 2;
constexpr size_t kOffProb = kOffOut + kNaOut * 4;
constexpr size_t kOffErr = kOffProb + 256;
constexpr size_t kNaScratchBytes = kOffErr + 256;                   // 2 MiB + 512 bytes

static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

constexpr int kMaxDevices = 64;

// Per-device set-up state, read and written under g_na_mu only.
struct NaDevice {
  unsigned long long ctx_id = 0;  // identity of the context the address belongs to
  unsigned char* addr = nullptr;  // device address of g_na_scratch in that context
};
std::mutex g_na_mu;
NaDevice g_na_dev[kMaxDevices];
PFN_cuTensorMapEncodeTiled_v12000 g_na_encode = nullptr;
PFN_cuCtxGetCurrent_v4000 g_na_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_na_ctx_id = nullptr;

template <typename F>
F na_entry(const char* name, int version) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(f);
}

// Planar BF16 pieces [Re(row) | Im(row)] of an n x n complex matrix, padded to Np
// with zeros (every element of the Np x 2Np region is written).
__global__ void k_na_planar(const double2* __restrict__ a, int n, int Np, __nv_bfloat16* dst) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Np * Np) return;
  const int i = (int)(idx / Np), j = (int)(idx % Np);
  const double2 v = (i < n && j < n) ? a[(long long)i * n + j] : make_double2(0.0, 0.0);
  const long long P = 2LL * Np * Np, o = (long long)i * 2 * Np + j;
  const __nv_bfloat16 rh = __double2bfloat16(v.x), ih = __double2bfloat16(v.y);
  dst[o] = rh;
  dst[P + o] = __double2bfloat16(v.x - (double)__bfloat162float(rh));
  dst[o + Np] = ih;
  dst[P + o + Np] = __double2bfloat16(v.y - (double)__bfloat162float(ih));
}

// Embedded BF16 pieces [[Re, Im], [-Im, Re]] of an n x n complex matrix, padded to Np.
__global__ void k_na_embedded(const double2* __restrict__ r, int n, int Np, __nv_bfloat16* dst) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Np * Np) return;
  const int i = (int)(idx / Np), j = (int)(idx % Np);
  const double2 v = (i < n && j < n) ? r[(long long)i * n + j] : make_double2(0.0, 0.0);
  const long long ld = 2LL * Np, P = 4LL * Np * Np;
  const __nv_bfloat16 rh = __double2bfloat16(v.x), ih = __double2bfloat16(v.y);
  const __nv_bfloat16 rl = __double2bfloat16(v.x - (double)__bfloat162float(rh));
  const __nv_bfloat16 il = __double2bfloat16(v.y - (double)__bfloat162float(ih));
  const long long i00 = i * ld + j, i01 = i * ld + Np + j, i10 = (Np + i) * ld + j, i11 = (Np + i) * ld + Np + j;
  dst[i00] = rh;
  dst[P + i00] = rl;
  dst[i01] = ih;
  dst[P + i01] = il;
  dst[i10] = __hneg(ih);
  dst[P + i10] = __hneg(il);
  dst[i11] = rh;
  dst[P + i11] = rl;
}

// The one-entry problem table of the product kernel, and the error word cleared.
__global__ void k_na_prob(TcProb* prob, int* err, int Np, float* out) {
  TcProb p;
  p.sys = 0;
  p.a_b[0] = p.a_b[1] = 0;
  p.b_b[0] = p.b_b[1] = 0;
  p.tiles_m = Np / BM;
  p.tiles_n = 2 * Np / 256;
  p.tile0 = 0;
  p.Np = Np;
  p.out = out;
  p.kt = 0;
  p.iter0 = 0;
  p.kofs = nullptr;  // every k-panel
  p.kidx = nullptr;
  p.cofs = nullptr;  // column tiles of 256
  *prob = p;
  *err = 0;
}

// FP32 planar product -> n x n complex128 interleaved output; nothing is
// written when the product kernel set its error word (a bounded wait expired).
__global__ void k_na_out(const float* __restrict__ x, int n, int Np, const int* __restrict__ err, double2* c) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n || *err != 0) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  c[idx] = make_double2(x[(long long)i * 2 * Np + j], x[(long long)i * 2 * Np + Np + j]);
}

// Per-device set-up, run with that device current: the device address of the
// scratch array (cudaGetSymbolAddress, checked) and the shared-memory limit of
// the product kernel.  Done once per device and context; *addr receives the
// address.
int na_setup(int dev, unsigned char** addr) {
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_encode) g_na_encode = na_entry<PFN_cuTensorMapEncodeTiled_v12000>("cuTensorMapEncodeTiled", 12000);
  if (!g_na_ctx_current) g_na_ctx_current = na_entry<PFN_cuCtxGetCurrent_v4000>("cuCtxGetCurrent", 4000);
  if (!g_na_ctx_id) g_na_ctx_id = na_entry<PFN_cuCtxGetId_v12000>("cuCtxGetId", 12000);
  if (!g_na_encode || !g_na_ctx_current || !g_na_ctx_id) return VGTB_E_CUDA;
  CUcontext cu = nullptr;
  if (g_na_ctx_current(&cu) != CUDA_SUCCESS) return VGTB_E_CUDA;
  if (!cu) {
    // no context current on this thread yet: cudaSetDevice makes the device's
    // primary context current (CUDA 12 and later)
    if (cudaSetDevice(dev) != cudaSuccess || g_na_ctx_current(&cu) != CUDA_SUCCESS || !cu) return VGTB_E_CUDA;
  }
  unsigned long long id = 0;
  if (g_na_ctx_id(cu, &id) != CUDA_SUCCESS) return VGTB_E_CUDA;
  NaDevice& d = g_na_dev[dev];
  if (d.addr && d.ctx_id == id) {
    *addr = d.addr;
    return VGTB_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess || !p) return VGTB_E_CUDA;
  e = cudaFuncSetAttribute(k_tc_gemm<256, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           2 * (2 * BM * BK * 2 + 2 * 256 * BK * 2) + 1024 + 256);
  if (e != cudaSuccess) return VGTB_E_CUDA;
  d.addr = static_cast<unsigned char*>(p);
  d.ctx_id = id;
  *addr = d.addr;
  return VGTB_OK;
}

// g_na_encode is set by na_setup() before any call of this function.
bool na_map(CUtensorMap* m, void* base, int cols, int rows, int box_rows) {
  cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)rows, 2, 1};
  cuuint64_t strides[3] = {(cuuint64_t)cols * 2, (cuuint64_t)cols * rows * 2, (cuuint64_t)cols * rows * 4};
  cuuint32_t box[4] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return g_na_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace
}  // namespace vgtb

using namespace vgtb;

extern "C" int vgtb_split_cgemm_noalloc(int n, const double* a, const double* r, double* c, void* stream) {
  if (n < 1 || n > kNaMaxN) return VGTB_E_INVALID;  // the scratch array holds n <= 256 only
  if (!a || !r || !c) return VGTB_E_INVALID;
  if (!tc_gemm_supported()) return VGTB_E_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VGTB_E_CUDA;
  unsigned char* base = nullptr;
  int rc = na_setup(dev, &base);
  if (rc != VGTB_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  __nv_bfloat16* ap = reinterpret_cast<__nv_bfloat16*>(base + kOffA);
  __nv_bfloat16* rp = reinterpret_cast<__nv_bfloat16*>(base + kOffR);
  float* xo = reinterpret_cast<float*>(base + kOffOut);
  TcProb* prob = reinterpret_cast<TcProb*>(base + kOffProb);
  int* err = reinterpret_cast<int*>(base + kOffErr);
  const int Np = (n + BM - 1) / BM * BM;
  const long long tot = (long long)Np * Np;
  k_na_planar<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2*>(a), n, Np, ap);
  k_na_embedded<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2*>(r), n, Np, rp);
  k_na_prob<<<1, 1, 0, st>>>(prob, err, Np, xo);
  TcParams P;
  memset(&P, 0, sizeof(P));
  if (!na_map(&P.mA[0][0], ap, 2 * Np, Np, BM) || !na_map(&P.mB[0][0], rp, 2 * Np, 2 * Np, 256))
    return VGTB_E_CUDA;
  P.probs = prob;
  P.n_prob = 1;
  P.total_tiles = (Np / BM) * (2 * Np / 256);
  P.nseg = 1;
  P.err = err;
  P.timeout_ns = 2000000000LL;
  const int smem = 2 * (2 * BM * BK * 2 + 2 * 256 * BK * 2) + 1024 + 256;
  k_tc_gemm<256, 2, 1><<<P.total_tiles, 192, smem, st>>>(P);
  k_na_out<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, st>>>(xo, n, Np, err, reinterpret_cast<double2*>(c));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return VGTB_E_CUDA;
  int herr = 0;
  e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return VGTB_E_CUDA;
  return herr ? VGTB_E_TIMEOUT : VGTB_OK;
}
