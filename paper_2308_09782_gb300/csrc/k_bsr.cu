// Block-sparse first product of the commutator (Eq. 6):
//
//   W = sum_seg A_seg R_seg^dagger
//
// FP64 path: W = D H (one segment; D at the level of the step's parity) or, in
// the delta form, W = dD H + D0 dH.  Split form: W = dD H + D0 dH in FP32 with
// the output stored as the embedded BF16 hi/lo pieces that the tcgen05 second
// product (X = S^-1 W^dagger) reads.
//
// R = H_k (or dH_k) is nonzero only on the target pattern: atom blocks (J, K)
// whose atoms lie within the two-centre cutoff (Eqs. 7-12), 5.7 % of the
// blocks at 512 atoms.  With R's rows in atom blocks of 4 orbitals,
//
//   W[i, 4J+c] = sum_{K: (J,K) target} sum_r A[i, 4K+r] conj(R_JK[c][r])
//              = conj( sum_K sum_r R_JK[c][r] A[4K+r, i] )      (A Hermitian)
//
// because every A here (D, dD, D0) is exactly Hermitian: the library keeps the
// Hermitian part of the initial density and the leapfrog update is mirror-exact.
// Reading A[4K+r, i] instead of A[i, 4K+r] makes the loads of a warp (32
// consecutive i) coalesced.  This costs 8 nnz(R) N flops per segment instead of
// the dense 8 N^3.
//
// Work unit = (item, atom group, column chunk): a CTA owns the output rows
// i in one chunk of columns of A and the 4G output columns of G consecutive
// atoms J.  It stages the group's R blocks (contiguous: targets are sorted by
// row atom) in shared memory and walks the union of the group's column atoms K
// once; for each K the four rows of A are loaded once and applied to every J of
// the group that has the block (J, K) (uniform branches: every thread of the
// CTA sees the same K).  Accumulation is in registers.  k_bsr (one output row
// per thread, 4 atoms per group) serves the FP64 path; k_bsr_f32x2 (below) the
// split form.
#include "vgtb_internal.h"

namespace vgtb {

namespace {

template <typename T>
struct Cx;
template <>
struct Cx<float> {
  using t = float2;
};
template <>
struct Cx<double> {
  using t = double2;
};

// slot of member j of a group entry: G shorts packed little-endian in 32-bit words
template <int G>
struct Slots {
  int w[G / 2];
  __device__ __forceinline__ int get(int j) const { return (int)(short)((uint32_t)w[j >> 1] >> (16 * (j & 1))); }
};

template <int G>
__device__ __forceinline__ Slots<G> load_slots(const short* p) {
  Slots<G> s;
  if constexpr (G == 8) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(p));
    s.w[0] = v.x;
    s.w[1] = v.y;
    s.w[2] = v.z;
    s.w[3] = v.w;
  } else {
    static_assert(G == 4, "atom groups of 4 or 8");
    const int2 v = __ldg(reinterpret_cast<const int2*>(p));
    s.w[0] = v.x;
    s.w[1] = v.y;
  }
  return s;
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// hi/lo BF16 pieces of four floats, packed for one 8-byte store each
__device__ __forceinline__ void split4(const float (&x)[4], uint2& hi, uint2& lo) {
  __nv_bfloat16 h[4], l[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    h[c] = __float2bfloat16_rn(x[c]);
    l[c] = __float2bfloat16_rn(x[c] - __bfloat162float(h[c]));
  }
  hi = make_uint2(bf16x2_bits(h[0], h[1]), bf16x2_bits(h[2], h[3]));
  lo = make_uint2(bf16x2_bits(l[0], l[1]), bf16x2_bits(l[2], l[3]));
}

}  // namespace

template <typename T, int G>
__global__ void __launch_bounds__(kBsrThreads) k_bsr(const BsrItem* __restrict__ items,
                                                     const BsrSys* __restrict__ sysv, const int* __restrict__ step) {
  using T2 = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char bsr_smem[];
  T2* sR = reinterpret_cast<T2*>(bsr_smem);
  pdl_wait();
  pdl_trigger();
  const BsrItem& it = items[blockIdx.y];
  const BsrSys& S = sysv[it.sys];
  const int Np = S.Np;
  const int nch = Np / kBsrThreads;
  const int u = blockIdx.x;
  if (u >= S.n_grp * nch) return;
  const int g = u / nch, ch = u - g * nch;
  const int i = ch * kBsrThreads + threadIdx.x;  // row of W = column of A
  const int t0 = S.grp_t0[g], nt = S.grp_t0[g + 1] - t0;
  const int e0 = S.grp_e0[g], e1 = S.grp_e0[g + 1];
  const int par = step ? (*step & 1) : 0;
  T ar[G][4], ai[G][4];
#pragma unroll
  for (int j = 0; j < G; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) ar[j][c] = ai[j][c] = T(0);

  for (int sg = 0; sg < it.nseg; ++sg) {
    const T2* R = reinterpret_cast<const T2*>(it.R[sg]) + 16LL * t0;
    __syncthreads();  // the previous segment's readers of sR are done
    for (int x = threadIdx.x; x < 16 * nt; x += kBsrThreads) sR[x] = R[x];
    __syncthreads();
    const T2* A = reinterpret_cast<const T2*>(it.A[sg]) + (sg == 0 ? par * it.a_par : 0LL) + i;
    // software pipeline: the four A rows of the next entry are in flight while
    // the current entry is applied
    T2 a[4], an[4];
    if (e0 < e1) {
      const T2* p = A + (long long)(4 * __ldg(S.ent_K + e0)) * Np;
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = p[(long long)r * Np];
    }
    for (int e = e0; e < e1; ++e) {
      if (e + 1 < e1) {
        const T2* p = A + (long long)(4 * __ldg(S.ent_K + e + 1)) * Np;
#pragma unroll
        for (int r = 0; r < 4; ++r) an[r] = p[(long long)r * Np];
      }
      const Slots<G> sl = load_slots<G>(S.ent_slot + (long long)G * e);
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const int s = sl.get(j);
        if (s >= 0) {
          const T2* b = sR + 16 * s;  // R_JK[c][r] at b[4c + r]
#pragma unroll
          for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const T2 v = b[4 * c + r];
              ar[j][c] = fma(v.x, a[r].x, ar[j][c]);
              ar[j][c] = fma(-v.y, a[r].y, ar[j][c]);
              ai[j][c] = fma(v.x, a[r].y, ai[j][c]);
              ai[j][c] = fma(v.y, a[r].x, ai[j][c]);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = an[r];
    }
  }

  // W[i, 4J + c] = conj(acc[j][c]) for the group's atoms J = G g + j < nat
  const int J0 = G * g;
  const int cnt = min(G, S.nat - J0);
  if constexpr (sizeof(T) == 8) {
    double2* W = reinterpret_cast<double2*>(it.W) + (long long)i * Np + 4 * J0;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      if (j < cnt) {
#pragma unroll
        for (int c = 0; c < 4; ++c) W[4 * j + c] = make_double2(ar[j][c], -ai[j][c]);
      }
    }
  } else {
    // embedded pieces [[Re W, Im W], [-Im W, Re W]] (row stride 2 Np), hi at
    // offset 0 and lo at 4 Np^2: top row i = [Wr | Wi], bottom row Np + i = [-Wi | Wr]
    __nv_bfloat16* P = reinterpret_cast<__nv_bfloat16*>(it.W);
    const long long P1 = 4LL * Np * Np, ld = 2LL * Np;
    const long long top = (long long)i * ld + 4 * J0, bot = (long long)(Np + i) * ld + 4 * J0;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      if (j < cnt) {
        float wr[4], wi[4], nwi[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          wr[c] = (float)ar[j][c];
          wi[c] = -(float)ai[j][c];
          nwi[c] = (float)ai[j][c];
        }
        uint2 rh, rl, ih, il, nh, nl;
        split4(wr, rh, rl);
        split4(wi, ih, il);
        split4(nwi, nh, nl);
        const long long o = 4 * j;
        *reinterpret_cast<uint2*>(P + top + o) = rh;
        *reinterpret_cast<uint2*>(P + P1 + top + o) = rl;
        *reinterpret_cast<uint2*>(P + top + Np + o) = ih;
        *reinterpret_cast<uint2*>(P + P1 + top + Np + o) = il;
        *reinterpret_cast<uint2*>(P + bot + o) = nh;
        *reinterpret_cast<uint2*>(P + P1 + bot + o) = nl;
        *reinterpret_cast<uint2*>(P + bot + Np + o) = rh;
        *reinterpret_cast<uint2*>(P + P1 + bot + Np + o) = rl;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Split form (FP32): the same product with two output rows per thread and the
// group's 8 atoms split between two warp groups of 4 warps (4 atoms each).
// A thread reads its two columns of each A row as one float4 (a warp reads 512
// contiguous bytes per row), so every block (J, K) value it loads from shared
// memory feeds 2 x 4 complex multiply-adds, and the A rows of an entry, loaded
// by both warp groups, are shared through L1.  Loads run one entry ahead.
// ---------------------------------------------------------------------------
constexpr int kBsr2Threads = 256;            // 2 warp groups x 128 threads, 2 columns each
constexpr int kBsr2Cols = kBsr2Threads;      // columns of A (rows of W) per CTA
constexpr int kBsr2PerWg = kBsrGroupF32 / 2; // atoms per warp group

__device__ __forceinline__ void cmac2(float& xr, float& xi, float br, float bi, float ar, float ai) {
  xr = fmaf(br, ar, xr);
  xr = fmaf(-bi, ai, xr);
  xi = fmaf(br, ai, xi);
  xi = fmaf(bi, ar, xi);
}

__global__ void __launch_bounds__(kBsr2Threads, 2) k_bsr_f32x2(const BsrItem* __restrict__ items,
                                                               const BsrSys* __restrict__ sysv) {
  extern __shared__ __align__(16) unsigned char bsr_smem[];
  float4* sR = reinterpret_cast<float4*>(bsr_smem);  // block (J, K) = 8 float4: row c = sR[8 s + 2c], [8 s + 2c + 1]
  pdl_wait();
  pdl_trigger();
  const BsrItem& it = items[blockIdx.y];
  const BsrSys& S = sysv[it.sys];
  const int Np = S.Np;
  const int nch = (Np + kBsr2Cols - 1) / kBsr2Cols;
  const int u = blockIdx.x;
  if (u >= S.n_grp * nch) return;
  const int g = u / nch, ch = u - g * nch;
  const int wg = threadIdx.x >> 7, tl = threadIdx.x & 127;
  const int i0 = ch * kBsr2Cols + 2 * tl;  // this thread's rows of W: i0, i0 + 1
  // Np is a multiple of 128, so in the last chunk of an Np that is not a multiple
  // of 256 whole warps (64 threads of each warp group) fall outside the matrix
  const bool live = i0 < Np;
  const int t0 = S.grp_t0[g], nt = S.grp_t0[g + 1] - t0;
  const int e0 = S.grp_e0[g], e1 = S.grp_e0[g + 1];
  // acc[j][c]: W rows i0 (x, y) and i0 + 1 (z, w) in (re, im) pairs
  float4 acc[kBsr2PerWg][4];
#pragma unroll
  for (int j = 0; j < kBsr2PerWg; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = make_float4(0.f, 0.f, 0.f, 0.f);

  for (int sg = 0; sg < it.nseg; ++sg) {
    const float4* R = reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(it.R[sg]) + 16LL * t0);
    __syncthreads();
    for (int x = threadIdx.x; x < 8 * nt; x += kBsr2Threads) sR[x] = R[x];
    __syncthreads();
    const float2* A = reinterpret_cast<const float2*>(it.A[sg]) + i0;
    auto load = [&](int e, float4 (&a)[4]) {
      const float2* p = A + (long long)(4 * __ldg(S.ent_K + e)) * Np;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        a[r] = live ? *reinterpret_cast<const float4*>(p + (long long)r * Np) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    float4 a0[4], a1[4];
    if (e0 < e1) load(e0, a0);
    for (int e = e0; e < e1; ++e) {
      if (e + 1 < e1) load(e + 1, a1);
      // this warp group's members 4 wg .. 4 wg + 3: four shorts of the entry's eight
      const int2 sw = __ldg(reinterpret_cast<const int2*>(S.ent_slot + (long long)kBsrGroupF32 * e) + wg);
#pragma unroll
      for (int j = 0; j < kBsr2PerWg; ++j) {
        const int word = (j < 2) ? sw.x : sw.y;
        const int s = (int)(short)((uint32_t)word >> (16 * (j & 1)));
        if (s >= 0) {
          const float4* b = sR + 8 * s;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 b01 = b[2 * c], b23 = b[2 * c + 1];  // R_JK[c][0..3] as (re, im) pairs
            float4& x = acc[j][c];
            cmac2(x.x, x.y, b01.x, b01.y, a0[0].x, a0[0].y);
            cmac2(x.z, x.w, b01.x, b01.y, a0[0].z, a0[0].w);
            cmac2(x.x, x.y, b01.z, b01.w, a0[1].x, a0[1].y);
            cmac2(x.z, x.w, b01.z, b01.w, a0[1].z, a0[1].w);
            cmac2(x.x, x.y, b23.x, b23.y, a0[2].x, a0[2].y);
            cmac2(x.z, x.w, b23.x, b23.y, a0[2].z, a0[2].w);
            cmac2(x.x, x.y, b23.z, b23.w, a0[3].x, a0[3].y);
            cmac2(x.z, x.w, b23.z, b23.w, a0[3].z, a0[3].w);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) a0[r] = a1[r];
    }
  }

  // W[i, 4J + c] = conj(acc) for J = 8 g + 4 wg + j < nat, rows i0 and i0 + 1,
  // as embedded BF16 pieces (row stride 2 Np; hi at 0, lo at 4 Np^2):
  // top row i = [Wr | Wi], bottom row Np + i = [-Wi | Wr]
  const int J0 = kBsrGroupF32 * g + kBsr2PerWg * wg;
  const int cnt = live ? min(kBsr2PerWg, S.nat - J0) : 0;
  __nv_bfloat16* P = reinterpret_cast<__nv_bfloat16*>(it.W);
  const long long P1 = 4LL * Np * Np, ld = 2LL * Np;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = i0 + h;
    const long long top = (long long)i * ld + 4 * J0, bot = (long long)(Np + i) * ld + 4 * J0;
#pragma unroll
    for (int j = 0; j < kBsr2PerWg; ++j) {
      if (j < cnt) {
        float wr[4], wi[4], nwi[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float xr = h ? acc[j][c].z : acc[j][c].x, xi = h ? acc[j][c].w : acc[j][c].y;
          wr[c] = xr;
          wi[c] = -xi;
          nwi[c] = xi;
        }
        uint2 rh, rl, ih, il, nh, nl;
        split4(wr, rh, rl);
        split4(wi, ih, il);
        split4(nwi, nh, nl);
        const long long o = 4 * j;
        *reinterpret_cast<uint2*>(P + top + o) = rh;
        *reinterpret_cast<uint2*>(P + P1 + top + o) = rl;
        *reinterpret_cast<uint2*>(P + top + Np + o) = ih;
        *reinterpret_cast<uint2*>(P + P1 + top + Np + o) = il;
        *reinterpret_cast<uint2*>(P + bot + o) = nh;
        *reinterpret_cast<uint2*>(P + P1 + bot + o) = nl;
        *reinterpret_cast<uint2*>(P + bot + Np + o) = rh;
        *reinterpret_cast<uint2*>(P + P1 + bot + Np + o) = rl;
      }
    }
  }
}

int bsr_group(int fp64) { return fp64 ? kBsrGroupF64 : kBsrGroupF32; }

size_t bsr_smem_bytes(int fp64, int max_grp_targets) {
  return (size_t)max_grp_targets * 16 * (fp64 ? sizeof(double2) : sizeof(float2));
}

int bsr_configure(int fp64, int max_grp_targets) {
  const size_t smem = bsr_smem_bytes(fp64, max_grp_targets);
  if (smem > 227 * 1024) return -1;
  cudaError_t e = fp64 ? cudaFuncSetAttribute(k_bsr<double, kBsrGroupF64>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                       : cudaFuncSetAttribute(k_bsr_f32x2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e == cudaSuccess ? 0 : -1;
}

int bsr_units(int fp64, int n_grp, int Np) {
  return n_grp * (fp64 ? Np / kBsrThreads : (Np + kBsr2Cols - 1) / kBsr2Cols);
}

void launch_bsr(const BsrItem* items, const BsrSys* sys, int n_items, int max_units, int fp64, int max_grp_targets,
                const int* step, cudaStream_t st) {
  const dim3 grid(max_units, n_items);
  const size_t smem = bsr_smem_bytes(fp64, max_grp_targets);
  if (fp64)
    launch_pdl(k_bsr<double, kBsrGroupF64>, grid, kBsrThreads, smem, st, items, sys, step);
  else
    launch_pdl(k_bsr_f32x2, grid, kBsr2Threads, smem, st, items, sys);
}

}  // namespace vgtb
