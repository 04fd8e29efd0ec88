// tcgen05 split-precision complex-product kernel (device code), sm_103a.
// Included by k_gemm_tc.cu (plans, autotuner, launches).
//
// A complex product C = A R^dagger (both operands stored as rows) becomes one
// real GEMM  out[m][n'] = sum_k' Aop[m][k'] Bop[n'][k']  with
//   Aop row m  = [Re A(m,:) | Im A(m,:)]                          ("planar", Np x 2Np)
//   Bop rows   = [[Re R, Im R], [-Im R, Re R]]                      ("embedded", 2Np x 2Np)
//   out row m  = [Re C(m,:) | Im C(m,:)].
// Product 1 (EPI 0) takes its B operand with the rows interleaved in blocks of
// four: B row 8b + q is row 4b + q of [Re R, Im R] for q < 4 and row 4b + q - 4
// of [-Im R, Re R] for q >= 4, so a 256-row tile holds the real and imaginary
// rows of 128 rows of R (32 atoms of an sp3 basis) and meets fewer nonzero
// k-panels of the block-sparse H; its output column 8b + q is then Re W(m, 4b+q)
// or Im W(m, 4b+q-4).  Product 2 (EPI 1) keeps the halves [Re | Im] above.
// Each operand is held as BF16 pieces x = x_hi + x_lo; the GEMM accumulates
// x_hi y_hi + x_hi y_lo + x_lo y_hi in FP32 in tensor memory (3 MMAs per slice).
// Segments concatenate along k (product 1 has two: [dD | D0] [H | dH]^dagger).
//
// Kernel: persistent CTAs over 128 x BN output tiles (2-SM pair: 256 x w, with
// the column tiles either all 256 wide or of planned widths w, multiples of 16,
// that balance the tiles over the pairs); warp 0 issues TMA loads
// (SWIZZLE_128B, 4-D maps: k, row, piece, batch) into a STAGES-deep ring,
// warp 1 allocates tensor memory and issues tcgen05.mma from one thread,
// warps 2-5 drain the double-buffered accumulator with tcgen05.ld and store
// either the embedded BF16 pieces of W (product 1) or FP32 planar X (product 2).
// Every mbarrier wait is bounded by %globaltimer: on expiry the kernel sets its
// error word, lets in-flight copies and MMAs finish (bounded), frees tensor
// memory and returns.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include "vgtb_tc.h"

namespace vgtb {


constexpr int kMaxSys = 4;
constexpr int BM = 128, BK = 64;
constexpr long long kDrainNs = 200000000LL;  // 0.2 s for in-flight work after an abort

struct TcProb {
  int sys;
  int a_b[2], b_b[2];  // batch coordinate of each segment's A / B operand
  int tiles_m, tiles_n, tile0, Np;
  void* out;
  int kt;              // k-iterations per tile (stream-K schedule)
  int iter0;           // first global k-iteration of the problem (stream-K schedule)
  // classic schedule with zero panels skipped (null = every panel): the
  // 64-wide k-panels of one segment in which the B rows of column tile nt have
  // a nonzero are kidx[kofs[nt] .. kofs[nt+1]-1]; every segment uses the list
  const int* kofs;
  const short* kidx;
  // 2-SM pair kernel, classic schedule: first B row of each column tile
  // (tiles_n + 1 entries, the last 2 Np; widths multiples of 16 up to 256, so
  // that the tiles can be balanced over the workers); null = tiles of 256
  const int* cofs;
};

struct TcParams {
  CUtensorMap mA[kMaxSys][2];
  CUtensorMap mB[kMaxSys][2];
  const TcProb* probs;
  int n_prob, total_tiles, nseg;
  int* err;
  long long timeout_ns;
  const int* tord;     // classic schedule: worker c takes tiles tord[c], tord[c + G], ... (null = 0, 1, ...;
                       // an entry -1 ends the worker's list)
  int n_tord;          // entries of tord
  int b_rows;          // 2-SM pair kernel: B rows per CTA in one TMA box (0 = 128)
  // stream-K schedule (streamk != 0): the tiles below sk_tile0 (whole waves)
  // go to the workers in turn, as in the classic schedule, so that workers on
  // the same operand rows stay at the same k and share them through L2; worker c
  // then owns the global k-iterations [i0 + R c / G, i0 + R (c+1) / G) of the
  // rest, i0 = sk_iter0, R = total_iters - i0.  A tile shared by several
  // workers is finished by the one holding its k = 0 part, after adding the
  // FP32 partials that the others left in ws[worker] and announced in flags.
  int streamk;
  int sk_tile0;
  long long sk_iter0;
  long long total_iters;
  float* ws;           // per CTA slot: [BN / 4][BM] float4 (see ws_slot)
  int* flags;          // [G], 1 = partial ready (reset to 0 by the finishing CTA)
};

struct TcPlan {
  TcParams P;
  TcProb* d_probs = nullptr;
  int* d_err = nullptr;
  float* d_ws = nullptr;
  int* d_flags = nullptr;
  int* d_kofs = nullptr;    // zero-panel skipping: panel lists of every system, and the tile order
  short* d_kidx = nullptr;
  int* d_tord = nullptr;
  int* d_cofs = nullptr;    // planned column tiles of every system
  int grid = 0, smem = 0, variant = 0, epi = 0, wmax = 0;
  bool skip = false;
  // host copies for the chained schedule: the problem table, every system's
  // column-tile starts and the modelled time of every tile
  std::vector<TcProb> probs_h;
  std::vector<std::vector<int>> starts_h;
  std::vector<double> cost_h;
};

// ----------------------------------------------------------------------------
// PTX helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ long long gtime() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit_ns, volatile int* abort_flag,
                                          int* err, bool check_abort = true) {
  long long t0 = 0;
  for (int it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 31) == 31) {
      if (check_abort && *abort_flag) return false;
      const long long now = gtime();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > limit_ns) {
        *abort_flag = 1;
        atomicOr(err, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version bit 46, layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// The same for a 64-byte swizzle (rows of 32 BF16): 8-row groups 512 bytes
// apart, layout type 4 (SWIZZLE_64B).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

#define TMEM_LD32(taddr, r)                                                                                        \
  asm volatile(                                                                                                    \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19," \
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                                  \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), \
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),     \
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),    \
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                  \
      : "r"(taddr))

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ int find_prob(const TcProb* probs, int n, int t, int p) {
  while (p + 1 < n && probs[p + 1].tile0 <= t) ++p;
  return p;
}

// the problem that owns tile t, by bisection (tiles taken in any order)
__device__ __forceinline__ int find_prob_any(const TcProb* probs, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// k-iterations of tile t of problem pr (classic schedule)
__device__ __forceinline__ int tile_kt(const TcParams& P, const TcProb& pr, int t) {
  if (!pr.kofs) return P.nseg * (2 * pr.Np) / BK;
  const int nt = (t - pr.tile0) / pr.tiles_m;
  return P.nseg * (pr.kofs[nt + 1] - pr.kofs[nt]);
}

// segment and k-panel of k-iteration kk of tile t
__device__ __forceinline__ void tile_panel(const TcProb& pr, int t, int kk, int& sg, int& kt) {
  if (!pr.kofs) {
    const int kts = (2 * pr.Np) / BK;
    sg = kk / kts;
    kt = kk - sg * kts;
    return;
  }
  const int nt = (t - pr.tile0) / pr.tiles_m;
  const int k0 = pr.kofs[nt], cnt = pr.kofs[nt + 1] - k0;
  sg = kk / cnt;
  kt = pr.kidx[k0 + kk - sg * cnt];
}

// first B row and width of column tile nt of the 2-SM pair kernel
__device__ __forceinline__ void col_tile(const TcProb& pr, int nt, int& cb, int& w) {
  if (pr.cofs) {
    cb = pr.cofs[nt];
    w = pr.cofs[nt + 1] - cb;
  } else {
    cb = nt * 256;
    w = 256;
  }
}

// Work units: classic mode walks whole tiles t = blockIdx.x + i G; stream-K
// mode walks this CTA's k-iteration range, split at tile boundaries.  Every
// role of the CTA runs the same cursor, so they agree on the sequence.
struct UnitCursor {
  long long it, e;
  int t_next, p;
};

// first global k-iteration of worker c out of G (a worker is a CTA, or a CTA pair)
__device__ __forceinline__ long long sk_start(const TcParams& P, int c, int G) {
  return P.sk_iter0 + (P.total_iters - P.sk_iter0) * (long long)c / (long long)G;
}

__device__ __forceinline__ void cursor_init(const TcParams& P, UnitCursor& u, int c, int G) {
  u.p = 0;
  u.t_next = c;
  u.it = P.streamk ? sk_start(P, c, G) : 0;
  u.e = P.streamk ? sk_start(P, c + 1, G) : 0;
}

// next unit: global tile t, its k-iterations [kb, ke) out of KT; false when done
__device__ __forceinline__ bool cursor_next(const TcParams& P, UnitCursor& u, int G, int& t, int& kb, int& ke,
                                            int& KT) {
  const int t_classic = P.streamk ? P.sk_tile0 : (P.tord ? P.n_tord : P.total_tiles);
  if (u.t_next < t_classic) {
    t = P.tord ? P.tord[u.t_next] : u.t_next;
    if (t < 0) return false;
    u.t_next += G;
    u.p = P.tord ? find_prob_any(P.probs, P.n_prob, t) : find_prob(P.probs, P.n_prob, t, u.p);
    KT = tile_kt(P, P.probs[u.p], t);
    kb = 0;
    ke = KT;
    return true;
  }
  if (P.streamk) {
    if (u.it >= u.e) return false;
    while (u.p + 1 < P.n_prob && P.probs[u.p + 1].iter0 <= u.it) ++u.p;
    const TcProb& pr = P.probs[u.p];
    KT = pr.kt;
    const long long rel = u.it - pr.iter0;
    const int local = (int)(rel / KT);
    const long long tile_start = pr.iter0 + (long long)local * KT;
    t = pr.tile0 + local;
    kb = (int)(u.it - tile_start);
    ke = (int)((u.e - tile_start) < KT ? (u.e - tile_start) : KT);
    u.it = tile_start + ke;
    return true;
  }
  return false;
}

// last worker that holds part of the tile whose k = 0 part ends worker c's range
__device__ __forceinline__ int sk_last_worker(const TcParams& P, const TcProb& pr, int local, int KT, int c, int G) {
  const long long x = (long long)pr.iter0 + (long long)local * KT + KT - 1;
  int cl = c + 1;
  while (cl + 1 < G && sk_start(P, cl + 1, G) <= x) ++cl;
  return cl;
}

// bounded wait for a stream-K partial flag; false on timeout or abort
__device__ __forceinline__ bool sk_wait_flag(const TcParams& P, int idx, volatile int* abort_flag) {
  long long t0 = 0;
  for (int spin = 0;; ++spin) {
    if (*reinterpret_cast<volatile int*>(P.flags + idx)) return true;
    if ((spin & 31) == 31) {
      if (*abort_flag) return false;
      const long long now = gtime();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > P.timeout_ns) {
        *abort_flag = 1;
        atomicOr(P.err, 2);
        return false;
      }
    }
  }
}

// Stream-K partial of CTA slot c (BM rows x bn FP32 columns): float4 j of row
// rt at [j][rt], so that the 32 rows of a warp store and load 512 contiguous bytes.
__device__ __forceinline__ float4* ws_slot(const TcParams& P, int c, int bn) {
  return reinterpret_cast<float4*>(P.ws) + (size_t)c * BM * (bn / 4);
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ uint4 pack8_bf16(const float (&x)[16], int h, float sgn) {
  return make_uint4(pack_bf16(sgn * x[8 * h], sgn * x[8 * h + 1]), pack_bf16(sgn * x[8 * h + 2], sgn * x[8 * h + 3]),
                    pack_bf16(sgn * x[8 * h + 4], sgn * x[8 * h + 5]), pack_bf16(sgn * x[8 * h + 6], sgn * x[8 * h + 7]));
}

// Product 1 epilogue: 32 accumulator columns gn .. gn + 31 of output row `row`
// (gn a multiple of 32) in the interleaved order (4 Re, 4 Im per block of four W
// columns) become 16 consecutive W columns j0 = gn / 2 .. j0 + 15, stored as the
// embedded BF16 pieces of W that product 2 reads as its B operand: top row m =
// [Re W | Im W], bottom row Np + m = [-Im W | Re W], hi at 0 and lo at 4 Np^2.
// (nh = 1: only the first 16 accumulator columns are the tile's, 8 W columns).
__device__ __forceinline__ void store_w_pieces(__nv_bfloat16* W, int Np, int row, int gn, const uint32_t (&r)[32],
                                               int nh) {
  const long long ld = 2LL * Np, P1 = 4LL * Np * Np;
  const int j0 = gn >> 1;
  float re[16], im[16], rel[16], iml[16];
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      re[4 * b + q] = __uint_as_float(r[8 * b + q]);
      im[4 * b + q] = __uint_as_float(r[8 * b + 4 + q]);
    }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float rh = __bfloat162float(__float2bfloat16_rn(re[i])), ih = __bfloat162float(__float2bfloat16_rn(im[i]));
    rel[i] = re[i] - rh;
    iml[i] = im[i] - ih;
    re[i] = rh;
    im[i] = ih;
  }
  const long long top = (long long)row * ld + j0, bot = (long long)(Np + row) * ld + j0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (h >= nh) break;
    reinterpret_cast<uint4*>(W + top)[h] = pack8_bf16(re, h, 1.f);
    reinterpret_cast<uint4*>(W + P1 + top)[h] = pack8_bf16(rel, h, 1.f);
    reinterpret_cast<uint4*>(W + top + Np)[h] = pack8_bf16(im, h, 1.f);
    reinterpret_cast<uint4*>(W + P1 + top + Np)[h] = pack8_bf16(iml, h, 1.f);
    reinterpret_cast<uint4*>(W + bot)[h] = pack8_bf16(im, h, -1.f);
    reinterpret_cast<uint4*>(W + P1 + bot)[h] = pack8_bf16(iml, h, -1.f);
    reinterpret_cast<uint4*>(W + bot + Np)[h] = pack8_bf16(re, h, 1.f);
    reinterpret_cast<uint4*>(W + P1 + bot + Np)[h] = pack8_bf16(rel, h, 1.f);
  }
}

// ----------------------------------------------------------------------------
// the kernel
// ----------------------------------------------------------------------------
template <int BN, int ST, int EPI>
__global__ void __launch_bounds__(192, 1) k_tc_gemm(const __grid_constant__ TcParams P) {
  constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t TCOLS = 2 * BN;
  constexpr uint32_t IDESC = idesc_bf16(BM, BN);
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + ST * STAGE);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + ST), accf0 = smem_u32(bars + 2 * ST),
                 acce0 = smem_u32(bars + 2 * ST + 2), drain = smem_u32(bars + 2 * ST + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * ST + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);  // [0] abort, [1..2] epilogue ok
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf0, 1);
    mbar_init(accf0 + 8, 1);
    mbar_init(acce0, 4);
    mbar_init(acce0 + 8, 4);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* s_epi_ok = abort_flag + 1;  // indexed by unit parity
  // barriers and TMEM are set up; operands and outputs are touched only after
  // the preceding kernel of the step has completed
  pdl_wait();
  pdl_trigger();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int it = 0, t, kb, ke, KT;
      bool ok = true;
      UnitCursor cur;
      cursor_init(P, cur, blockIdx.x, gridDim.x);
      while (ok && cursor_next(P, cur, gridDim.x, t, kb, ke, KT)) {
        const TcProb& pr = P.probs[cur.p];
        const int local = t - pr.tile0;
        const int mt = local % pr.tiles_m, nt = local / pr.tiles_m;
        for (int kk = kb; kk < ke; ++kk, ++it) {
          int sg, kt;
          tile_panel(pr, t, kk, sg, kt);
          const CUtensorMap* ma = &P.mA[pr.sys][sg];
          const CUtensorMap* mb = &P.mB[pr.sys][sg];
          const int s = it % ST, r = it / ST;
          if (!mbar_wait(empty0 + 8 * s, (r & 1) ^ 1, P.timeout_ns, abort_flag, P.err)) {
            ok = false;
            break;
          }
          const uint32_t base = smem_u32(sm + s * STAGE);
          mbar_expect_tx(full0 + 8 * s, STAGE);
          tma_load_4d(base, ma, kt * BK, mt * BM, 0, pr.a_b[sg], full0 + 8 * s);
          tma_load_4d(base + A_BYTES, ma, kt * BK, mt * BM, 1, pr.a_b[sg], full0 + 8 * s);
          tma_load_4d(base + 2 * A_BYTES, mb, kt * BK, nt * BN, 0, pr.b_b[sg], full0 + 8 * s);
          tma_load_4d(base + 2 * A_BYTES + B_BYTES, mb, kt * BK, nt * BN, 1, pr.b_b[sg], full0 + 8 * s);
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA can exit
        for (int j = (it > ST ? it - ST : 0); j < it; ++j)
          mbar_wait(full0 + 8 * (j % ST), (j / ST) & 1, kDrainNs, abort_flag, P.err, false);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int it = 0, i = 0, t, kb, ke, KT;
      bool ok = true, issued = false;
      UnitCursor cur;
      cursor_init(P, cur, blockIdx.x, gridDim.x);
      while (ok && cursor_next(P, cur, gridDim.x, t, kb, ke, KT)) {
        const int ab = i & 1, u = i >> 1;
        if (!mbar_wait(acce0 + 8 * ab, (u & 1) ^ 1, P.timeout_ns, abort_flag, P.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + ab * BN;
        for (int kk = kb; kk < ke; ++kk, ++it) {
          const int s = it % ST, r = it / ST;
          if (!mbar_wait(full0 + 8 * s, r & 1, P.timeout_ns, abort_flag, P.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(sm + s * STAGE);
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            const uint64_t ah = sw128_desc(base + 32 * j);
            const uint64_t al = sw128_desc(base + A_BYTES + 32 * j);
            const uint64_t bh = sw128_desc(base + 2 * A_BYTES + 32 * j);
            const uint64_t bl = sw128_desc(base + 2 * A_BYTES + B_BYTES + 32 * j);
            tc_mma(d, ah, bh, IDESC, (kk > kb || j > 0) ? 1u : 0u);
            tc_mma(d, ah, bl, IDESC, 1u);
            tc_mma(d, al, bh, IDESC, 1u);
          }
          tc_commit(empty0 + 8 * s);
          issued = true;
        }
        if (!ok) break;
        tc_commit(accf0 + 8 * ab);
        ++i;
      }
      if (!ok && issued) {
        tc_commit(drain);
        mbar_wait(drain, 0, kDrainNs, abort_flag, P.err, false);
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5 -> TMEM lane quarters 2,3,0,1) ----------------
    // Thread 64 takes every wait of the group and publishes the outcome in
    // shared memory before a group barrier, so the four warps always agree.
    const int q = warp & 3;
    const bool leader = threadIdx.x == 64;
    int i = 0, t, kb, ke, KT;
    UnitCursor cur;
    cursor_init(P, cur, blockIdx.x, gridDim.x);
    while (cursor_next(P, cur, gridDim.x, t, kb, ke, KT)) {
      const TcProb& pr = P.probs[cur.p];
      const int local = t - pr.tile0;
      const int mt = local % pr.tiles_m, nt = local / pr.tiles_m;
      const int ab = i & 1, u = i >> 1;
      const bool contrib = P.streamk && kb > 0;
      const bool finish = P.streamk && kb == 0 && ke < KT;
      // CTAs after this one hold the rest of the tile's k-iterations
      const int c_last = finish ? sk_last_worker(P, pr, local, KT, blockIdx.x, gridDim.x) : blockIdx.x;
      if (leader) {
        int ok = mbar_wait(accf0 + 8 * ab, u & 1, P.timeout_ns, abort_flag, P.err) ? 1 : 0;
        for (int c2 = blockIdx.x + 1; ok && finish && c2 <= c_last; ++c2) ok = sk_wait_flag(P, c2, abort_flag) ? 1 : 0;
        __threadfence();
        s_epi_ok[i & 1] = ok;
      }
      epi_bar();
      if (!s_epi_ok[i & 1]) break;
      tc_fence_after();
      const int Np = pr.Np;
      const long long ld = 2LL * Np;
      const int rt = q * 32 + lane;  // row within the tile
      const int row = mt * BM + rt;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ab * BN + c0 + ((uint32_t)(q * 32) << 16);
        TMEM_LD32(taddr, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (contrib) {
          float4* w = ws_slot(P, blockIdx.x, BN) + (c0 / 4) * BM + rt;
#pragma unroll
          for (int v = 0; v < 8; ++v)
            w[v * BM] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]), __uint_as_float(r[4 * v + 2]),
                               __uint_as_float(r[4 * v + 3]));
          continue;
        }
        if (finish) {
          for (int c2 = blockIdx.x + 1; c2 <= c_last; ++c2) {
            const float4* w = ws_slot(P, c2, BN) + (c0 / 4) * BM + rt;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
              const float4 f = __ldcg(w + v * BM);
              r[4 * v] = __float_as_uint(__uint_as_float(r[4 * v]) + f.x);
              r[4 * v + 1] = __float_as_uint(__uint_as_float(r[4 * v + 1]) + f.y);
              r[4 * v + 2] = __float_as_uint(__uint_as_float(r[4 * v + 2]) + f.z);
              r[4 * v + 3] = __float_as_uint(__uint_as_float(r[4 * v + 3]) + f.w);
            }
          }
        }
        const int gn = nt * BN + c0;
        if (EPI == 1) {
          float* X = reinterpret_cast<float*>(pr.out) + row * ld + gn;
#pragma unroll
          for (int v = 0; v < 8; ++v)
            reinterpret_cast<float4*>(X)[v] =
                make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]), __uint_as_float(r[4 * v + 2]),
                            __uint_as_float(r[4 * v + 3]));
        } else {
          store_w_pieces(reinterpret_cast<__nv_bfloat16*>(pr.out), Np, row, gn, r, 2);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * ab);
      if (contrib) {
        // publish the partial: every writer fences, then one flag store
        __threadfence();
        epi_bar();
        if (leader) atomicExch(P.flags + blockIdx.x, 1);
      } else if (finish) {
        // every thread has read the partials: release the slots
        epi_bar();
        if (leader)
          for (int c2 = blockIdx.x + 1; c2 <= c_last; ++c2) atomicExch(P.flags + c2, 0);
      }
      ++i;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  }
}

// ----------------------------------------------------------------------------
// 2-SM pair variant: a cluster of two CTAs computes a 256 x 256 tile with
// tcgen05.mma.cta_group::2 (M = 256: each CTA holds 128 rows of A and of the
// accumulator; N = 256: each CTA holds half of the B tile).  Np is a multiple
// of 128, so 2 Np is a multiple of 256 and only the last row tile can be half
// outside the matrix: its A rows load as TMA zero fill and its stores are
// skipped.  Per SM this moves
// a third less operand data through shared memory and L2 per flop than the
// 128 x 256 single-CTA tile.  The pair's loads all complete on the leader's
// (rank 0) full barrier; the leader's single MMA thread issues every MMA and
// its commits arrive on both CTAs' barriers; both CTAs' epilogue warps arrive
// on the leader's accumulator-empty barrier.  Classic tile loop over pair
// tiles; problem tiles are counted in 256 x 256 units.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_to_rank0(uint32_t saddr) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(0));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tma_load_4d_pair(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                                 uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar_cluster)
      : "memory");
}

__device__ __forceinline__ void tc_mma_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

// KH = 1: one pipeline stage per 64-wide k-panel (128-byte swizzle); KH = 2:
// two stages of 32 columns per panel (64-byte swizzle), so that twice as many
// stages fit and the copies run further ahead of the MMAs.
template <int ST, int EPI, int KH>
__global__ void __launch_bounds__(192, 1) k_tc_gemm2(const __grid_constant__ TcParams P) {
  constexpr int BNP = 256;                                  // pair tile width
  constexpr int BKS = BK / KH;                              // k-columns per stage
  constexpr uint32_t A_BYTES = BM * BKS * 2;                // this CTA's 128 rows of A, per piece
  constexpr uint32_t B_BYTES = (BNP / 2) * BKS * 2;         // this CTA's half of B, per piece
  constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t TCOLS = 2 * BNP;
  // bytes of one stage that the TMA copies (both pieces of A and of this CTA's B rows)
  const uint32_t stage_tx = 2 * A_BYTES + 2 * (uint32_t)(P.b_rows ? P.b_rows : BNP / 2) * BKS * 2;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + ST * STAGE);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + ST), accf0 = smem_u32(bars + 2 * ST),
                 acce0 = smem_u32(bars + 2 * ST + 2), drain = smem_u32(bars + 2 * ST + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * ST + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);  // [0] abort, [1..2] epilogue ok
  volatile int* s_epi_ok = abort_flag + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader_cta = rank == 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf0, 1);
    mbar_init(accf0 + 8, 1);
    mbar_init(acce0, 8);
    mbar_init(acce0 + 8, 8);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();
  pdl_trigger();
  const uint32_t full_l = map_to_rank0(full0), acce_l = map_to_rank0(acce0);
  const int pair = blockIdx.x >> 1, G2 = gridDim.x >> 1;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs) ----------------
      int it = 0, t, kb, ke, KT;
      bool ok = true;
      UnitCursor cur;
      cursor_init(P, cur, pair, G2);
      while (ok && cursor_next(P, cur, G2, t, kb, ke, KT)) {
        const TcProb& pr = P.probs[cur.p];
        const int local = t - pr.tile0;
        const int mt = local % pr.tiles_m, nt = local / pr.tiles_m;
        int cb, w;
        col_tile(pr, nt, cb, w);
        const int arow = mt * (2 * BM) + rank * BM, brow = cb + rank * (w / 2);
        for (int kk = kb; ok && kk < ke; ++kk) {
          int sg, kt;
          tile_panel(pr, t, kk, sg, kt);
          const CUtensorMap* ma = &P.mA[pr.sys][sg];
          const CUtensorMap* mb = &P.mB[pr.sys][sg];
#pragma unroll 1
          for (int h = 0; h < KH; ++h, ++it) {
            const int s = it % ST, r = it / ST;
            if (!mbar_wait(empty0 + 8 * s, (r & 1) ^ 1, P.timeout_ns, abort_flag, P.err)) {
              ok = false;
              break;
            }
            const uint32_t base = smem_u32(sm + s * STAGE);
            if (leader_cta) mbar_expect_tx(full0 + 8 * s, 2 * stage_tx);
            const uint32_t fb = full_l + 8 * s;
            const int x = kt * BK + h * BKS;
            tma_load_4d_pair(base, ma, x, arow, 0, pr.a_b[sg], fb);
            tma_load_4d_pair(base + A_BYTES, ma, x, arow, 1, pr.a_b[sg], fb);
            tma_load_4d_pair(base + 2 * A_BYTES, mb, x, brow, 0, pr.b_b[sg], fb);
            tma_load_4d_pair(base + 2 * A_BYTES + B_BYTES, mb, x, brow, 1, pr.b_b[sg], fb);
          }
        }
      }
      if (!ok) {
        if (leader_cta) {
          // the leader's full barriers also count the peer's bytes of the same iterations
          for (int j = (it > ST ? it - ST : 0); j < it; ++j)
            mbar_wait(full0 + 8 * (j % ST), (j / ST) & 1, kDrainNs, abort_flag, P.err, false);
        } else {
          // the peer cannot wait on the leader's barriers: give its copies time to land
          const long long t0 = gtime();
          while (gtime() - t0 < 200000) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader_cta) {
      // ---------------- MMA issuer (leader CTA only) ----------------
      int it = 0, i = 0, t, kb, ke, KT;
      bool ok = true, issued = false;
      UnitCursor cur;
      cursor_init(P, cur, pair, G2);
      for (; ok && cursor_next(P, cur, G2, t, kb, ke, KT); ++i) {
        const int ab = i & 1, u = i >> 1;
        if (!mbar_wait(acce0 + 8 * ab, (u & 1) ^ 1, P.timeout_ns, abort_flag, P.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + ab * BNP;
        int cb, w;
        {
          const TcProb& pr = P.probs[cur.p];
          col_tile(pr, (t - pr.tile0) / pr.tiles_m, cb, w);
        }
        const uint32_t idesc = idesc_bf16(2 * BM, w);
        for (int ks = kb * KH; ks < ke * KH; ++ks, ++it) {
          const int s = it % ST, r = it / ST;
          if (!mbar_wait(full0 + 8 * s, r & 1, P.timeout_ns, abort_flag, P.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(sm + s * STAGE);
#pragma unroll
          for (int j = 0; j < BKS / 16; ++j) {
            const uint64_t ah = KH == 1 ? sw128_desc(base + 32 * j) : sw64_desc(base + 32 * j);
            const uint64_t al = KH == 1 ? sw128_desc(base + A_BYTES + 32 * j) : sw64_desc(base + A_BYTES + 32 * j);
            const uint64_t bh =
                KH == 1 ? sw128_desc(base + 2 * A_BYTES + 32 * j) : sw64_desc(base + 2 * A_BYTES + 32 * j);
            const uint64_t bl = KH == 1 ? sw128_desc(base + 2 * A_BYTES + B_BYTES + 32 * j)
                                        : sw64_desc(base + 2 * A_BYTES + B_BYTES + 32 * j);
            tc_mma_pair(d, ah, bh, idesc, (ks > kb * KH || j > 0) ? 1u : 0u);
            tc_mma_pair(d, ah, bl, idesc, 1u);
            tc_mma_pair(d, al, bh, idesc, 1u);
          }
          tc_commit_pair(empty0 + 8 * s, 3);
          issued = true;
        }
        if (!ok) break;
        tc_commit_pair(accf0 + 8 * ab, 3);
      }
      if (!ok && issued) {
        tc_commit_pair(drain, 1);
        mbar_wait(drain, 0, kDrainNs, abort_flag, P.err, false);
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5 of both CTAs) ----------------
    // stream-K: each CTA of a pair keeps its own 128 rows of a partial in the
    // slot and flag of index 2 * pair + rank
    const int q = warp & 3;
    const bool leader = threadIdx.x == 64;
    const int me = 2 * pair + (int)rank;
    int i = 0, t, kb, ke, KT;
    UnitCursor cur;
    cursor_init(P, cur, pair, G2);
    for (; cursor_next(P, cur, G2, t, kb, ke, KT); ++i) {
      const TcProb& pr = P.probs[cur.p];
      const int local = t - pr.tile0;
      const int mt = local % pr.tiles_m, nt = local / pr.tiles_m;
      const int ab = i & 1, u = i >> 1;
      const bool contrib = P.streamk && kb > 0;
      const bool finish = P.streamk && kb == 0 && ke < KT;
      const int p_last = finish ? sk_last_worker(P, pr, local, KT, pair, G2) : pair;
      if (leader) {
        int ok = mbar_wait(accf0 + 8 * ab, u & 1, P.timeout_ns, abort_flag, P.err) ? 1 : 0;
        for (int p2 = pair + 1; ok && finish && p2 <= p_last; ++p2)
          ok = sk_wait_flag(P, 2 * p2 + (int)rank, abort_flag) ? 1 : 0;
        __threadfence();
        s_epi_ok[i & 1] = ok;
      }
      epi_bar();
      if (!s_epi_ok[i & 1]) break;
      tc_fence_after();
      const int Np = pr.Np;
      const long long ld = 2LL * Np;
      const int rt = q * 32 + lane;
      const int row = mt * (2 * BM) + rank * BM + rt;
      int cb, w;
      col_tile(pr, nt, cb, w);
#pragma unroll 1
      for (int c0 = 0; c0 < w; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ab * BNP + c0 + ((uint32_t)(q * 32) << 16);
        TMEM_LD32(taddr, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (contrib) {
          float4* wp = ws_slot(P, me, BNP) + (c0 / 4) * BM + rt;
#pragma unroll
          for (int v = 0; v < 8; ++v)
            wp[v * BM] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]), __uint_as_float(r[4 * v + 2]),
                               __uint_as_float(r[4 * v + 3]));
          continue;
        }
        if (finish) {
          for (int p2 = pair + 1; p2 <= p_last; ++p2) {
            const float4* wp = ws_slot(P, 2 * p2 + (int)rank, BNP) + (c0 / 4) * BM + rt;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
              const float4 f = __ldcg(wp + v * BM);
              r[4 * v] = __float_as_uint(__uint_as_float(r[4 * v]) + f.x);
              r[4 * v + 1] = __float_as_uint(__uint_as_float(r[4 * v + 1]) + f.y);
              r[4 * v + 2] = __float_as_uint(__uint_as_float(r[4 * v + 2]) + f.z);
              r[4 * v + 3] = __float_as_uint(__uint_as_float(r[4 * v + 3]) + f.w);
            }
          }
        }
        const int gn = cb + c0;
        const int nv = w - c0 < 32 ? w - c0 : 32;  // 16 in the last chunk of a width 32 m + 16
        if (row >= Np) continue;  // last row tile of an Np that is not a multiple of 256
        if (EPI == 1) {
          float* X = reinterpret_cast<float*>(pr.out) + row * ld + gn;
#pragma unroll
          for (int v = 0; v < 8; ++v)
            if (4 * v < nv)
              reinterpret_cast<float4*>(X)[v] =
                  make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                              __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
        } else {
          store_w_pieces(reinterpret_cast<__nv_bfloat16*>(pr.out), Np, row, gn, r, nv >> 4);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(acce_l + 8 * ab);
      if (contrib) {
        __threadfence();
        epi_bar();
        if (leader) atomicExch(P.flags + me, 1);
      } else if (finish) {
        epi_bar();
        if (leader)
          for (int p2 = pair + 1; p2 <= p_last; ++p2) atomicExch(P.flags + 2 * p2 + (int)rank, 0);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  }
}

}  // namespace vgtb
