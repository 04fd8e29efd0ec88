// vgtb_split_cgemm_noalloc: the tcgen05 BF16x3 complex product C = A R^dagger
// for callers that cannot allocate device memory.
//
// All scratch (the BF16 hi/lo pieces of A and of the embedded R, the FP32
// product, the one-entry problem table and the error word) lives in one
// file-scope static __device__ array of fixed size, so a call performs no
// cudaMalloc, cudaFree or allocating library call.  Host code cannot pass the
// array's name to a kernel (in host code it is only a stand-in, not a device
// address): the first call on each device looks the address up with
// cudaGetSymbolAddress and caches it.
#include <cuda_runtime.h>

#include <cstring>

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
unsigned char* g_na_addr[kMaxDevices] = {nullptr};

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
  *prob = p;
  *err = 0;
}

// FP32 planar product -> n x n complex128 interleaved output.
__global__ void k_na_out(const float* __restrict__ x, int n, int Np, double2* c) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  c[idx] = make_double2(x[(long long)i * 2 * Np + j], x[(long long)i * 2 * Np + Np + j]);
}

// Per-device set-up: the device address of the scratch array and the shared
// memory limit of the product kernel.  Runs with that device current.
int na_setup(int dev) {
  if (g_na_addr[dev]) return VGTB_OK;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess || !p) return VGTB_E_CUDA;
  e = cudaFuncSetAttribute(k_tc_gemm<256, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           2 * (2 * BM * BK * 2 + 2 * 256 * BK * 2) + 1024 + 256);
  if (e != cudaSuccess) return VGTB_E_CUDA;
  g_na_addr[dev] = static_cast<unsigned char*>(p);
  return VGTB_OK;
}

bool na_map(CUtensorMap* m, void* base, int cols, int rows, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)rows, 2, 1};
  cuuint64_t strides[3] = {(cuuint64_t)cols * 2, (cuuint64_t)cols * rows * 2, (cuuint64_t)cols * rows * 4};
  cuuint32_t box[4] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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
  int rc = na_setup(dev);
  if (rc != VGTB_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = g_na_addr[dev];
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
  k_na_out<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, st>>>(xo, n, Np, reinterpret_cast<double2*>(c));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return VGTB_E_CUDA;
  int herr = 0;
  e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return VGTB_E_CUDA;
  return herr ? VGTB_E_TIMEOUT : VGTB_OK;
}
