// Both tcgen05 products of a step in one persistent launch (the chained
// schedule), sm_103a.  Included by k_gemm_tc.cu after tc_kernel.cuh.
//
// Product 2 (X = S^-1 W^dagger) reads W, which product 1 writes; run as two
// launches, each product ends with a partly filled wave of tiles (at 512 atoms
// 128 tiles of product 1 over 76 CTA pairs leave 24 pairs idle for a whole
// tile).  Here one grid of CTA pairs works through one list of units: every
// tile of product 1, then every tile of product 2.  A tile of product 2 needs
// only the rows of W that its B rows hold (row n' of the embedded W is row
// n' mod Np of W), i.e. one or two 256-row blocks of product 1 tiles; the
// producer of the pair waits (bounded) until the epilogues of all product 1
// tiles of those blocks have stored their pieces of W and counted them in
// ready[].  Every worker takes all its product 1 tiles before its first
// product 2 tile, so a wait is only ever for product 1 tiles, which wait for
// nothing: the schedule cannot deadlock.
//
// A block's count in ready[] grows by 2 x (product 1 column tiles) per launch
// (each CTA of a pair counts its half of every tile); a launch waits for
// (epoch + 1) times that, where epoch counts the completed launches (the last
// CTA to exit advances it), so nothing has to be reset between launches.
#pragma once
#include "tc_kernel.cuh"

namespace vgtb {

struct TcChainExtra {
  const int* ord;                 // worker c takes units ord[c], ord[c + G], ... (-1 ends its list)
  int n_ord;
  int t1;                         // units below t1: product 1 tiles; t1 + t: product 2 tile t
  unsigned long long* ready;      // per (problem, 256-row block of W): product 1 tile halves stored
  const int* blk0;                // index in ready[] of each problem's first block
  unsigned long long* epoch;      // [0] completed launches, [1] CTAs exited from this launch
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// next unit of worker c: product e (0 or 1) and its tile t; false at the end
__device__ __forceinline__ bool chain_next(const TcChainExtra& X, int c, int G, int& j, int& e, int& t) {
  const int i = j * G + c;
  if (i >= X.n_ord) return false;
  const int u = X.ord[i];
  if (u < 0) return false;
  ++j;
  e = u >= X.t1 ? 1 : 0;
  t = e ? u - X.t1 : u;
  return true;
}

// bounded wait until block b of problem p holds this launch's stores of W
__device__ __forceinline__ bool chain_wait_block(const TcChainExtra& X, int p, int b, unsigned long long target,
                                                 long long limit_ns, volatile int* abort_flag, int* err) {
  const unsigned long long* r = X.ready + X.blk0[p] + b;
  long long t0 = 0;
  for (int it = 0;; ++it) {
    if (ld_acquire_u64(r) >= target) return true;
    if ((it & 31) == 31) {
      if (*abort_flag) return false;
      const long long now = gtime();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > limit_ns) {
        *abort_flag = 1;
        atomicOr(err, 2);
        return false;
      }
    }
  }
}

// waits for the blocks of W that B rows cb .. cb + w - 1 of a product 2 tile
// hold (rows n' and n' - Np of the embedded W are row n' mod Np of W)
__device__ __forceinline__ bool chain_wait_rows(const TcChainExtra& X, int p, int Np, int cb, int w,
                                                unsigned long long target, long long limit_ns,
                                                volatile int* abort_flag, int* err) {
  const int seg[2][2] = {{cb, min(cb + w, Np)}, {max(cb, Np) - Np, cb + w - Np}};
  for (int sgi = 0; sgi < 2; ++sgi) {
    if (seg[sgi][1] <= seg[sgi][0]) continue;
    for (int b = seg[sgi][0] / 256; b <= (seg[sgi][1] - 1) / 256; ++b)
      if (!chain_wait_block(X, p, b, target, limit_ns, abort_flag, err)) return false;
  }
  // the rows were stored through the generic proxy; the copies below read them
  // through the async proxy
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return true;
}

// One unit = one 256 x w output tile of product e (Q = P1 or P2), taken whole
// (classic schedule; 3 stages of 64 k-columns).  Roles as in k_tc_gemm2.
template <int ST>
__global__ void __launch_bounds__(192, 1)
    k_tc_chain(const __grid_constant__ TcParams P1, const __grid_constant__ TcParams P2,
               const __grid_constant__ TcChainExtra X) {
  constexpr int BNP = 256;
  constexpr uint32_t A_BYTES = BM * BK * 2;
  constexpr uint32_t B_BYTES = (BNP / 2) * BK * 2;
  constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t TCOLS = 2 * BNP;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + ST * STAGE);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + ST), accf0 = smem_u32(bars + 2 * ST),
                 acce0 = smem_u32(bars + 2 * ST + 2), drain = smem_u32(bars + 2 * ST + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * ST + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);  // [0] abort, [1..2] epilogue ok
  volatile int* s_epi_ok = abort_flag + 1;
  int* err = P1.err;  // one error word for the launch
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader_cta = rank == 0;
  const long long limit = P1.timeout_ns;

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
      const unsigned long long ep1 = X.epoch[0] + 1ULL;
      int it = 0, j = 0, e, t;
      bool ok = true;
      while (ok && chain_next(X, pair, G2, j, e, t)) {
        const TcParams& Q = e ? P2 : P1;
        const int p = find_prob_any(Q.probs, Q.n_prob, t);
        const TcProb& pr = Q.probs[p];
        const int local = t - pr.tile0;
        const int mt = local % pr.tiles_m, nt = local / pr.tiles_m;
        int cb, w;
        col_tile(pr, nt, cb, w);
        if (e && !chain_wait_rows(X, p, pr.Np, cb, w, ep1 * 2ULL * (unsigned long long)P1.probs[p].tiles_n, limit,
                                  abort_flag, err)) {
          ok = false;
          break;
        }
        const uint32_t stage_tx = 2 * A_BYTES + 2 * (uint32_t)(Q.b_rows ? Q.b_rows : BNP / 2) * BK * 2;
        const int arow = mt * (2 * BM) + rank * BM, brow = cb + rank * (w / 2);
        const int KT = tile_kt(Q, pr, t);
        for (int kk = 0; kk < KT; ++kk, ++it) {
          int sg, kt;
          tile_panel(pr, t, kk, sg, kt);
          const CUtensorMap* ma = &Q.mA[pr.sys][sg];
          const CUtensorMap* mb = &Q.mB[pr.sys][sg];
          const int s = it % ST, r = it / ST;
          if (!mbar_wait(empty0 + 8 * s, (r & 1) ^ 1, limit, abort_flag, err)) {
            ok = false;
            break;
          }
          const uint32_t base = smem_u32(sm + s * STAGE);
          if (leader_cta) mbar_expect_tx(full0 + 8 * s, 2 * stage_tx);
          const uint32_t fb = full_l + 8 * s;
          tma_load_4d_pair(base, ma, kt * BK, arow, 0, pr.a_b[sg], fb);
          tma_load_4d_pair(base + A_BYTES, ma, kt * BK, arow, 1, pr.a_b[sg], fb);
          tma_load_4d_pair(base + 2 * A_BYTES, mb, kt * BK, brow, 0, pr.b_b[sg], fb);
          tma_load_4d_pair(base + 2 * A_BYTES + B_BYTES, mb, kt * BK, brow, 1, pr.b_b[sg], fb);
        }
      }
      if (!ok) {
        if (leader_cta) {
          for (int q = (it > ST ? it - ST : 0); q < it; ++q)
            mbar_wait(full0 + 8 * (q % ST), (q / ST) & 1, kDrainNs, abort_flag, err, false);
        } else {
          const long long t0 = gtime();
          while (gtime() - t0 < 200000) {
          }
        }
      }
    }
  }
  else if (warp == 1) {
    if (lane == 0 && leader_cta) {
      // ---------------- MMA issuer (leader CTA only) ----------------
      int it = 0, i = 0, j = 0, e, t;
      bool ok = true, issued = false;
      for (; ok && chain_next(X, pair, G2, j, e, t); ++i) {
        const TcParams& Q = e ? P2 : P1;
        const TcProb& pr = Q.probs[find_prob_any(Q.probs, Q.n_prob, t)];
        const int ab = i & 1, u = i >> 1;
        if (!mbar_wait(acce0 + 8 * ab, (u & 1) ^ 1, limit, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + ab * BNP;
        int cb, w;
        col_tile(pr, (t - pr.tile0) / pr.tiles_m, cb, w);
        const uint32_t idesc = idesc_bf16(2 * BM, w);
        const int KT = tile_kt(Q, pr, t);
        for (int kk = 0; kk < KT; ++kk, ++it) {
          const int s = it % ST, r = it / ST;
          if (!mbar_wait(full0 + 8 * s, r & 1, limit, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(sm + s * STAGE);
#pragma unroll
          for (int q = 0; q < BK / 16; ++q) {
            const uint64_t ah = sw128_desc(base + 32 * q);
            const uint64_t al = sw128_desc(base + A_BYTES + 32 * q);
            const uint64_t bh = sw128_desc(base + 2 * A_BYTES + 32 * q);
            const uint64_t bl = sw128_desc(base + 2 * A_BYTES + B_BYTES + 32 * q);
            tc_mma_pair(d, ah, bh, idesc, (kk > 0 || q > 0) ? 1u : 0u);
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
        mbar_wait(drain, 0, kDrainNs, abort_flag, err, false);
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5 of both CTAs) ----------------
    const int q = warp & 3;
    const bool leader = threadIdx.x == 64;
    int i = 0, j = 0, e, t;
    for (; chain_next(X, pair, G2, j, e, t); ++i) {
      const TcParams& Q = e ? P2 : P1;
      const int p = find_prob_any(Q.probs, Q.n_prob, t);
      const TcProb& pr = Q.probs[p];
      const int local = t - pr.tile0;
      const int mt = local % pr.tiles_m, nt = local / pr.tiles_m;
      const int ab = i & 1, u = i >> 1;
      if (leader) {
        s_epi_ok[i & 1] = mbar_wait(accf0 + 8 * ab, u & 1, limit, abort_flag, err) ? 1 : 0;
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
        const int gn = cb + c0;
        const int nv = w - c0 < 32 ? w - c0 : 32;
        if (row >= Np) continue;
        if (e) {
          float* Xo = reinterpret_cast<float*>(pr.out) + row * ld + gn;
#pragma unroll
          for (int v = 0; v < 8; ++v)
            if (4 * v < nv)
              reinterpret_cast<float4*>(Xo)[v] =
                  make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                              __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
        } else {
          store_w_pieces(reinterpret_cast<__nv_bfloat16*>(pr.out), Np, row, gn, r, nv >> 4);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(acce_l + 8 * ab);
      if (!e) {
        // this CTA's half of the tile's W is stored: count it for product 2
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __threadfence();
        epi_bar();
        if (leader) red_release_add_u64(X.ready + X.blk0[p] + mt, 1ULL);
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
  if (threadIdx.x == 0) {
    // the last CTA out advances the launch count
    __threadfence();
    if (atomicAdd(X.epoch + 1, 1ULL) == (unsigned long long)gridDim.x - 1) {
      X.epoch[1] = 0;
      __threadfence();
      atomicAdd(X.epoch, 1ULL);
    }
  }
}

}  // namespace vgtb
