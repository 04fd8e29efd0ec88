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
// per thread, 4 atoms per group) serves the FP64 path; k_bsr_f32p (below) the
// split form.
#include <algorithm>

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
// Split form (FP32), persistent: k_bsr_f32p.  A CTA of 128 threads takes
// units (item, group of 8 atoms, chunk of 128 A columns) from a global counter
// until none is left; one thread owns one column of A (one row of W) and the
// 8 x 4 complex accumulators of the group's atoms.  Each thread stages its own
// four A values of an entry through a ring of kBsrStages shared-memory slots
// with cp.async (no other thread reads them, so no CTA barrier is needed per
// entry), so kBsrStages - 1 entries are in flight while one is applied; the
// ring runs on across the segment boundary.  The R blocks of the group's current
// segment sit in shared memory.  The last CTA to run out of units resets the
// counters for the next launch.
// ---------------------------------------------------------------------------
constexpr int kBsrPThreads = 128;
constexpr int kBsrStages = 6;

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(kBsrPThreads, 3) k_bsr_f32p(const BsrItem* __restrict__ items,
                                                             const BsrSys* __restrict__ sysv,
                                                             const int* __restrict__ item_u0, int n_items,
                                                             int* __restrict__ ctr, int max_tg) {
  extern __shared__ __align__(16) unsigned char bsr_smem[];
  float4* sR = reinterpret_cast<float4*>(bsr_smem);                  // [max_tg][8] float4
  float2* sA = reinterpret_cast<float2*>(bsr_smem + (long long)max_tg * 128);  // [kBsrStages][4][kBsrPThreads]
  __shared__ int s_unit;
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x;
  const int total = item_u0[n_items];
  const uint32_t sA_u32 = (uint32_t)__cvta_generic_to_shared(sA);
  for (;;) {
    __syncthreads();  // the previous unit's readers of sR are done
    if (tid == 0) s_unit = atomicAdd(ctr, 1);
    __syncthreads();
    const int uu = s_unit;
    if (uu >= total) break;
    int itx = 0;
    while (itx + 1 < n_items && item_u0[itx + 1] <= uu) ++itx;
    const BsrItem& it = items[itx];
    const BsrSys& S = sysv[it.sys];
    const int Np = S.Np;
    const int nch = Np / kBsrPThreads;
    const int u = uu - item_u0[itx];
    const int g = u / nch, ch = u - g * nch;
    const int i = ch * kBsrPThreads + tid;
    const int t0 = S.grp_t0[g], nt = S.grp_t0[g + 1] - t0;
    const int e0 = S.grp_e0[g], ne = S.grp_e0[g + 1] - e0;
    auto stage_r = [&](int sg) {
      const float4* R = reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(it.R[sg]) + 16LL * t0);
      for (int x = tid; x < 8 * nt; x += kBsrPThreads) sR[x] = R[x];
    };
    stage_r(0);
    __syncthreads();
    const int nsteps = it.nseg * ne;  // entries of segment 0, then of segment 1
    auto issue = [&](int st) {
      if (st < nsteps) {
        const int sg = st >= ne ? 1 : 0;
        const int e = e0 + st - sg * ne;
        const float2* p = reinterpret_cast<const float2*>(it.A[sg]) + (long long)(4 * __ldg(S.ent_K + e)) * Np + i;
        const uint32_t d = sA_u32 + (uint32_t)(((st % kBsrStages) * 4 * kBsrPThreads + tid) * 8);
#pragma unroll
        for (int r = 0; r < 4; ++r) cp_async8(d + r * kBsrPThreads * 8, p + (long long)r * Np);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int st = 0; st < kBsrStages - 1; ++st) issue(st);
    float ar[kBsrGroupF32][4], ai[kBsrGroupF32][4];
#pragma unroll
    for (int j = 0; j < kBsrGroupF32; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) ar[j][c] = ai[j][c] = 0.f;
    for (int st = 0; st < nsteps; ++st) {
      if (st == ne) {  // segment 1 begins: its R blocks replace segment 0's
        __syncthreads();
        stage_r(1);
        __syncthreads();
      }
      issue(st + kBsrStages - 1);
      cp_async_wait<kBsrStages - 1>();
      const int sg = st >= ne ? 1 : 0;
      const int e = e0 + st - sg * ne;
      const float2* a_s = sA + (st % kBsrStages) * 4 * kBsrPThreads + tid;
      const float2 a0 = a_s[0], a1 = a_s[kBsrPThreads], a2 = a_s[2 * kBsrPThreads], a3 = a_s[3 * kBsrPThreads];
      const Slots<kBsrGroupF32> sl = load_slots<kBsrGroupF32>(S.ent_slot + (long long)kBsrGroupF32 * e);
      const float4* Rs = sR;
#pragma unroll
      for (int j = 0; j < kBsrGroupF32; ++j) {
        const int s = sl.get(j);
        if (s >= 0) {
          const float4* b = Rs + 8 * s;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 b01 = b[2 * c], b23 = b[2 * c + 1];  // R_JK[c][0..3] as (re, im) pairs
            float xr = ar[j][c], xi = ai[j][c];
            xr = fmaf(b01.x, a0.x, xr); xr = fmaf(-b01.y, a0.y, xr); xi = fmaf(b01.x, a0.y, xi); xi = fmaf(b01.y, a0.x, xi);
            xr = fmaf(b01.z, a1.x, xr); xr = fmaf(-b01.w, a1.y, xr); xi = fmaf(b01.z, a1.y, xi); xi = fmaf(b01.w, a1.x, xi);
            xr = fmaf(b23.x, a2.x, xr); xr = fmaf(-b23.y, a2.y, xr); xi = fmaf(b23.x, a2.y, xi); xi = fmaf(b23.y, a2.x, xi);
            xr = fmaf(b23.z, a3.x, xr); xr = fmaf(-b23.w, a3.y, xr); xi = fmaf(b23.z, a3.y, xi); xi = fmaf(b23.w, a3.x, xi);
            ar[j][c] = xr;
            ai[j][c] = xi;
          }
        }
      }
    }
    cp_async_wait<0>();
    // W[i, 4J + c] = conj(acc) as embedded BF16 pieces (row stride 2 Np; hi at 0,
    // lo at 4 Np^2): top row i = [Wr | Wi], bottom row Np + i = [-Wi | Wr]
    const int J0 = kBsrGroupF32 * g;
    const int cnt = min(kBsrGroupF32, S.nat - J0);
    __nv_bfloat16* P = reinterpret_cast<__nv_bfloat16*>(it.W);
    const long long P1 = 4LL * Np * Np, ld = 2LL * Np;
    const long long top = (long long)i * ld + 4 * J0, bot = (long long)(Np + i) * ld + 4 * J0;
#pragma unroll
    for (int j = 0; j < kBsrGroupF32; ++j) {
      if (j < cnt) {
        float wr[4], wi[4], nwi[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          wr[c] = ar[j][c];
          wi[c] = -ai[j][c];
          nwi[c] = ai[j][c];
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
  // the last CTA out resets the unit counter for the next launch
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1) == (int)gridDim.x - 1) {
      ctr[0] = 0;
      ctr[1] = 0;
      __threadfence();
    }
  }
}

size_t bsr_p_smem_bytes(int max_grp_targets) {
  return (size_t)max_grp_targets * 128 + (size_t)kBsrStages * 4 * kBsrPThreads * sizeof(float2);
}

// ---------------------------------------------------------------------------
// Crank-Nicolson density at the nonzero pattern (a sampled product):
//   D[4J+c, 4K+r] = 2 sum_n conj(Cd[n, 4J+c]) Cd[n, 4K+r]   for every target (J, K)
// with Cd = C^dagger ([nocc][Np]).  A CTA takes one group of 4 row atoms J (the
// FP64 group tables of the block-sparse product) and walks the occupied states in
// chunks of kCnChunk: the chunk's values at the group's own 16 columns and at the
// columns of the union of its column atoms K are staged in shared memory, and
// each thread accumulates up to kCnOut of the group's block elements in FP64.
// 8 nnz(H) nocc flops instead of the 8 Np^2 nocc of the dense C C^dagger.
// ---------------------------------------------------------------------------
constexpr int kCnThreads = 256;
constexpr int kCnChunk = 8;
constexpr int kCnOut = 12;  // block elements per thread: up to 192 targets per group of 4 atoms

size_t cn_smem_bytes(int max_ent) { return (size_t)kCnChunk * (16 + 4 * max_ent) * sizeof(double2); }

__global__ void __launch_bounds__(kCnThreads) k_cn_density_pattern(const CnDensItem* __restrict__ items,
                                                                  const BsrSys* __restrict__ sysv, int max_ent) {
  extern __shared__ __align__(16) unsigned char cn_smem[];
  double2* sJ = reinterpret_cast<double2*>(cn_smem);  // [kCnChunk][16]
  double2* sK = sJ + kCnChunk * 16;                    // [kCnChunk][4 max_ent]
  const int ldk = 4 * max_ent;
  pdl_wait();
  pdl_trigger();
  const CnDensItem& it = items[blockIdx.y];
  const BsrSys& S = sysv[it.sys];
  const int g = blockIdx.x;
  if (g >= S.n_grp) return;
  const int Np = S.Np;
  const int J0 = kBsrGroupF64 * g;
  const int t0 = S.grp_t0[g], nt = S.grp_t0[g + 1] - t0;
  const int e0 = S.grp_e0[g], ne = S.grp_e0[g + 1] - e0;
  const int nout = 16 * nt;
  // output u of this thread: target t0 + o / 16, element (c, r) = ((o % 16) / 4, o % 4)
  int cj[kCnOut], ck[kCnOut];
  double ar[kCnOut], ai[kCnOut];
#pragma unroll
  for (int u = 0; u < kCnOut; ++u) {
    const int o = threadIdx.x + kCnThreads * u;
    ar[u] = ai[u] = 0.0;
    cj[u] = ck[u] = -1;
    if (o < nout) {
      const int code = S.tgt_ent[t0 + o / 16];
      cj[u] = 4 * (code >> 10) + (o % 16) / 4;  // column of sJ
      ck[u] = 4 * (code & 1023) + o % 4;         // column of sK
    }
  }
  const double2* Cd = it.Cd;
  for (int n0 = 0; n0 < it.nocc; n0 += kCnChunk) {
    __syncthreads();  // the previous chunk's readers are done
    for (int x = threadIdx.x; x < kCnChunk * 16; x += kCnThreads) {
      const int nn = x >> 4, q = x & 15, n = n0 + nn, col = 4 * J0 + q;
      sJ[x] = (n < it.nocc && col < Np) ? Cd[(long long)n * Np + col] : make_double2(0.0, 0.0);
    }
    for (int x = threadIdx.x; x < kCnChunk * 4 * ne; x += kCnThreads) {
      const int nn = x / (4 * ne), q = x - nn * 4 * ne, n = n0 + nn;
      const int col = 4 * __ldg(S.ent_K + e0 + (q >> 2)) + (q & 3);
      sK[nn * ldk + q] = n < it.nocc ? Cd[(long long)n * Np + col] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kCnOut; ++u) {
      if (cj[u] < 0) continue;
#pragma unroll
      for (int nn = 0; nn < kCnChunk; ++nn) {
        const double2 a = sJ[nn * 16 + cj[u]], b = sK[nn * ldk + ck[u]];
        ar[u] = fma(a.x, b.x, fma(a.y, b.y, ar[u]));   // Re(conj(a) b)
        ai[u] = fma(a.x, b.y, fma(-a.y, b.x, ai[u]));  // Im(conj(a) b)
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kCnOut; ++u) {
    if (cj[u] < 0) continue;
    const int o = threadIdx.x + kCnThreads * u;
    const int code = S.tgt_ent[t0 + o / 16];
    const int row = 4 * (J0 + (code >> 10)) + (o % 16) / 4;
    const int col = 4 * __ldg(S.ent_K + e0 + (code & 1023)) + o % 4;
    it.D[(long long)row * Np + col] = make_double2(2.0 * ar[u], 2.0 * ai[u]);
  }
}

int cn_density_max_targets() { return kCnThreads * kCnOut / 16; }

int cn_density_configure(int max_ent) {
  const size_t smem = cn_smem_bytes(max_ent);
  if (smem > 227 * 1024) return -1;
  return cudaFuncSetAttribute(k_cn_density_pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                 cudaSuccess
             ? 0
             : -1;
}

void launch_cn_density_pattern(const CnDensItem* items, const BsrSys* sys, int n_items, int max_groups, int max_ent,
                               cudaStream_t st) {
  launch_pdl(k_cn_density_pattern, dim3(max_groups, n_items), kCnThreads, cn_smem_bytes(max_ent), st, items, sys,
             max_ent);
}

int bsr_group(int fp64) { return fp64 ? kBsrGroupF64 : kBsrGroupF32; }

size_t bsr_smem_bytes(int fp64, int max_grp_targets) {
  return (size_t)max_grp_targets * 16 * (fp64 ? sizeof(double2) : sizeof(float2));
}

int bsr_configure(int fp64, int max_grp_targets) {
  const size_t smem = fp64 ? bsr_smem_bytes(1, max_grp_targets) : bsr_p_smem_bytes(max_grp_targets);
  if (smem > 227 * 1024) return -1;
  cudaError_t e = fp64 ? cudaFuncSetAttribute(k_bsr<double, kBsrGroupF64>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                       : cudaFuncSetAttribute(k_bsr_f32p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e == cudaSuccess ? 0 : -1;
}

int bsr_units(int fp64, int n_grp, int Np) {
  (void)fp64;  // both kernels take 128 columns of A per unit
  return n_grp * (Np / 128);
}

void launch_bsr(const BsrItem* items, const BsrSys* sys, int n_items, int max_units, int total_units,
                const int* item_u0, int* ctr, int fp64, int max_grp_targets, const int* step, cudaStream_t st) {
  if (fp64) {
    launch_pdl(k_bsr<double, kBsrGroupF64>, dim3(max_units, n_items), kBsrThreads, bsr_smem_bytes(1, max_grp_targets),
               st, items, sys, step);
    return;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(total_units, 3 * nsm);  // resident CTAs: 3 per SM (registers, shared memory)
  launch_pdl(k_bsr_f32p, grid, kBsrPThreads, bsr_p_smem_bytes(max_grp_targets), st, items, sys, item_u0, n_items, ctr,
             max_grp_targets);
}

}  // namespace vgtb
