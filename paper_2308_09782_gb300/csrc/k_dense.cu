// Dense FP64 kernels:
//   k_gemm_f64 - C = sum_seg A_seg R_seg^dagger (complex128, row-major), the two
//                commutator products of Eq. 6 in FP64:
//                  W = D H (= (H D)^dagger),  X = S^-1 W^dagger = S^-1 H D
//   k_leap     - dD/dt = R0 - i (X - X^dagger) (Eq. 6 with X = S^-1 H D) and the
//                leapfrog update of Eq. 13; tile (bi, bj) and (bj, bi) are handled by
//                one CTA so X^dagger is read from shared memory, and each D level is
//                read and written exactly once.
//   helpers    - Hermitian fill, eigenvector transpose, BF16 hi/lo splitting.
// GB300 has no FP64 tensor-core kind, so the FP64 path runs on DFMA.
#include <algorithm>

#include "vgtb_internal.h"

namespace vgtb {

// ---------------------------------------------------------------------------
// FP64 complex GEMM. 64 x 64 output tile per CTA, 256 threads, 4 x 4 outputs
// per thread (rows ty + 16 i, cols tx + 16 j), K tiles of 16 staged in smem.
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_gemm_f64(const GemmF64Item* __restrict__ items,
                                                  const int* __restrict__ step) {
  pdl_wait();
  pdl_trigger();
  __shared__ double2 As[GK][GT + 1];
  __shared__ double2 Rs[GK][GT + 1];
  const GemmF64Item& it = items[blockIdx.z];
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  if (m0 >= it.M || n0 >= it.N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int par = step ? (*step & 1) : 0;
  double cr[4][4], ci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = 0.0;
  for (int sg = 0; sg < it.nseg; ++sg) {
    const double2* A = it.A[sg] + par * it.a_par[sg];
    const double2* R = it.R[sg];
    const int K = it.K[sg], lda = it.lda[sg], ldr = it.ldr[sg];
    const bool ta = it.conj_t & 1, tr = (it.conj_t >> 1) & 1;
    for (int k0 = 0; k0 < K; k0 += GK) {
      // load 64 x 16 of A and of R: thread -> (row = tid/16 + 16 p, col = tid%16);
      // a conjugate-transposed operand is read along its rows instead (coalesced)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int r = ty + 16 * p, c = tx;
        const int idx = tid + 256 * p, tk = idx >> 6, trw = idx & 63;
        if (ta) {
          const int gm = m0 + trw, gk = k0 + tk;
          const double2 v = (gm < it.M && gk < K) ? A[(long long)gk * lda + gm] : make_double2(0.0, 0.0);
          As[tk][trw] = make_double2(v.x, -v.y);
        } else {
          const int gm = m0 + r, gk = k0 + c;
          As[c][r] = (gm < it.M && gk < K) ? A[(long long)gm * lda + gk] : make_double2(0.0, 0.0);
        }
        if (tr) {
          const int gn = n0 + trw, gk = k0 + tk;
          const double2 v = (gn < it.N && gk < K) ? R[(long long)gk * ldr + gn] : make_double2(0.0, 0.0);
          Rs[tk][trw] = make_double2(v.x, -v.y);
        } else {
          const int gn = n0 + r, gk = k0 + c;
          Rs[c][r] = (gn < it.N && gk < K) ? R[(long long)gn * ldr + gk] : make_double2(0.0, 0.0);
        }
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < GK; ++kk) {
        double2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Rs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // a * conj(b)
            cr[i][j] = fma(a[i].x, b[j].x, cr[i][j]);
            cr[i][j] = fma(a[i].y, b[j].y, cr[i][j]);
            ci[i][j] = fma(a[i].y, b[j].x, ci[i][j]);
            ci[i][j] = fma(-a[i].x, b[j].y, ci[i][j]);
          }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= it.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= it.N) continue;
      double2 v = make_double2(cr[i][j], ci[i][j]);
      if (it.epi == 1) {
        const double2 c = it.coef;
        v = make_double2(c.x * v.x - c.y * v.y, c.x * v.y + c.y * v.x);
        if (it.base) {
          const double2 b = it.base[(long long)gm * it.ldb + gn];
          v.x += b.x;
          v.y += b.y;
        }
      }
      it.C[(long long)gm * it.ldc + gn] = v;
    }
  }
}

void launch_gemm_f64(const GemmF64Item* items, int n_items, int max_m, int max_n, const int* step,
                     cudaStream_t st) {
  dim3 grid((max_n + GT - 1) / GT, (max_m + GT - 1) / GT, n_items);
  launch_pdl(k_gemm_f64, grid, 256, 0, st, items, step);
}

// ---------------------------------------------------------------------------
// Leapfrog (Eq. 13) with dD/dt = R0 - i (X - X^dagger):
//   dDr_ij = R0r_ij + Xi_ij + Xi_ji,   dDi_ij = R0i_ij - (Xr_ij - Xr_ji).
// The same floating-point operations give element (j, i) as the exact
// conjugate of (i, j), so Hermiticity is kept bit for bit.
// Step n reads level n from D[n&1]; it writes level n+1 into D[(n+1)&1]:
//   n == 0 : D1 = D0 + dt dD (forward-Euler start);  n > 0 : D_{n+1} = D_{n-1} + 2 dt dD.
// mode 1 writes dD/dt itself into `out` (used to precompute R0).
// The last CTA to finish advances the step counter.
// ---------------------------------------------------------------------------
constexpr int LT = 32;

__device__ __forceinline__ void split_bf16_d(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __double2bfloat16(x);
  lo = __double2bfloat16(x - (double)__bfloat162float(hi));
}

__global__ void __launch_bounds__(256) k_leap(const LeapItem* __restrict__ items, const int* step,
                                              double dt, int* counter, int* step_rw) {
  pdl_wait();
  pdl_trigger();
  __shared__ double2 Xa[LT][LT + 1];
  __shared__ double2 Xb[LT][LT + 1];
  const LeapItem& it = items[blockIdx.y];
  const int Np = it.Np;
  const int nt = Np / LT;
  const int n = step ? *step : 0;
  // map blockIdx.x -> (bi <= bj)
  int p = blockIdx.x, bi = 0;
  const int npairs = nt * (nt + 1) / 2;
  bool active = p < npairs;
  if (active) {
    while (p >= nt - bi) {
      p -= nt - bi;
      ++bi;
    }
  }
  const int bj = bi + p;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if (active) {
    for (int r = ty; r < LT; r += 8) {
      const long long ia = (long long)(bi * LT + r) * Np + bj * LT + tx;
      const long long ib = (long long)(bj * LT + r) * Np + bi * LT + tx;
      const double2* X = (const double2*)it.X;
      Xa[r][tx] = X[ia];
      Xb[r][tx] = X[ib];
    }
  }
  __syncthreads();
  if (active) {
    const int cur = n & 1, nxt = cur ^ 1;
    const bool euler = (n == 0);
    const double coef = it.mode == 1 ? 1.0 : (euler ? dt : 2.0 * dt);
    const double2* base = euler ? it.D[cur] : it.D[nxt];
    for (int half = 0; half < (bi == bj ? 1 : 2); ++half) {
      const int gi0 = half == 0 ? bi : bj, gj0 = half == 0 ? bj : bi;
      for (int r = ty; r < LT; r += 8) {
        const double2 xij = half == 0 ? Xa[r][tx] : Xb[r][tx];
        const double2 xji = half == 0 ? Xb[tx][r] : Xa[tx][r];
        const long long idx = (long long)(gi0 * LT + r) * Np + gj0 * LT + tx;
        double dr = xij.y + xji.y;
        double di = -(xij.x - xji.x);
        if (it.R0) {
          const double2 r0 = it.R0[idx];
          dr = r0.x + dr;
          di = r0.y + di;
        }
        if (it.mode == 1) {
          it.out[idx] = make_double2(dr, di);
          continue;
        }
        const double2 b = base[idx];
        const double2 v = make_double2(b.x + coef * dr, b.y + coef * di);
        it.D[nxt][idx] = v;
        if (it.pieces) {
          const long long P = 2LL * Np * Np;
          const long long pr = (long long)(gi0 * LT + r) * 2 * Np + gj0 * LT + tx;
          __nv_bfloat16 h, l;
          split_bf16_d(v.x, h, l);
          it.pieces[pr] = h;
          it.pieces[P + pr] = l;
          split_bf16_d(v.y, h, l);
          it.pieces[pr + Np] = h;
          it.pieces[P + pr + Np] = l;
        }
      }
    }
  }
  if (counter) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      __threadfence();
      const int total = gridDim.x * gridDim.y;
      const int ticket = atomicAdd(counter, 1);
      if (ticket == total - 1) {
        *counter = 0;
        *step_rw = n + 1;
        __threadfence();
      }
    }
  }
}

void launch_leap(const LeapItem* items, int n_items, int Np_max, int x_f32, const int* step, double dt,
                 int* counter, int* step_rw, cudaStream_t st) {
  (void)x_f32;
  const int nt = Np_max / LT;
  dim3 grid(nt * (nt + 1) / 2, n_items);
  dim3 block(LT, 8);
  launch_pdl(k_leap, grid, block, 0, st, items, step, dt, counter, step_rw);
}

// ---------------------------------------------------------------------------
// Leapfrog of the split form: X (FP32 planar) and R0 (FP32 planar) give
// dD/dt in FP32 with the same mirror-exact operations as k_leap; only the
// master update dD_{n+1} = dD_{n-1} + 2 dt dD/dt is FP64 (GB300's FP64 rate is
// low, so FP64 is kept to the accumulation that needs it).  The operand of the
// next first product is written from the new level's FP32 rounding: its FP32
// copy (block-sparse product) and/or its BF16 hi/lo pieces (dense tcgen05
// product).
// ---------------------------------------------------------------------------
// Thread layout: 16 x 16 threads, each owns two adjacent columns (2 tx, 2 tx + 1)
// of rows ty and ty + 16 of a 32 x 32 tile, so R0 is read and the BF16 pieces
// written two columns per instruction; X is staged as separate real and
// imaginary tiles, whose transposed reads (X_ji) hit distinct banks.
__global__ void __launch_bounds__(256, 4) k_leap_split(const LeapItem* __restrict__ items, const int* step, double dt,
                                                    int* counter, int* step_rw) {
  pdl_wait();
  pdl_trigger();
  __shared__ float Xre[2][LT][LT + 1];  // [0] tile (bi, bj), [1] tile (bj, bi)
  __shared__ float Xim[2][LT][LT + 1];
  const LeapItem& it = items[blockIdx.y];
  const int Np = it.Np;
  const int nt = Np / LT;
  const int n = *step;
  int p = blockIdx.x, bi = 0;
  const int npairs = nt * (nt + 1) / 2;
  const bool active = p < npairs;
  if (active) {
    while (p >= nt - bi) {
      p -= nt - bi;
      ++bi;
    }
  }
  const int bj = bi + p;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 16 x 16
  const int c0 = 2 * tx;
  const float* X = (const float*)it.X;
  if (active) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = ty + 16 * h;
      const long long ra = (long long)(bi * LT + r) * 2 * Np + bj * LT + c0;
      const long long rb = (long long)(bj * LT + r) * 2 * Np + bi * LT + c0;
      const float2 ar = *reinterpret_cast<const float2*>(X + ra), ai = *reinterpret_cast<const float2*>(X + ra + Np);
      const float2 br = *reinterpret_cast<const float2*>(X + rb), bim = *reinterpret_cast<const float2*>(X + rb + Np);
      Xre[0][r][c0] = ar.x;
      Xre[0][r][c0 + 1] = ar.y;
      Xim[0][r][c0] = ai.x;
      Xim[0][r][c0 + 1] = ai.y;
      Xre[1][r][c0] = br.x;
      Xre[1][r][c0 + 1] = br.y;
      Xim[1][r][c0] = bim.x;
      Xim[1][r][c0 + 1] = bim.y;
    }
  }
  __syncthreads();
  if (active) {
    const int cur = n & 1, nxt = cur ^ 1;
    const bool euler = (n == 0);
    const double coef = euler ? dt : 2.0 * dt;
    const double2* base = euler ? it.D[cur] : it.D[nxt];
    const long long P = 2LL * Np * Np;
    for (int half = 0; half < (bi == bj ? 1 : 2); ++half) {
      const int gi0 = half == 0 ? bi : bj, gj0 = half == 0 ? bj : bi;
      const int A = half, B = half ^ 1;  // tile of (i, j) and of its mirror (j, i)
      // all loads of the thread's elements first (D_{n-1} is overwritten in place,
      // element by element, by the same thread), then the updates and stores
      float2 r0r[2], r0i[2];
      double2 b[2][2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = ty + 16 * h;
        const long long idx = (long long)(gi0 * LT + r) * Np + gj0 * LT + c0;
        const long long pr = (long long)(gi0 * LT + r) * 2 * Np + gj0 * LT + c0;
        r0r[h] = it.R0f ? *reinterpret_cast<const float2*>(it.R0f + pr) : make_float2(0.f, 0.f);
        r0i[h] = it.R0f ? *reinterpret_cast<const float2*>(it.R0f + pr + Np) : make_float2(0.f, 0.f);
        b[h][0] = base[idx];
        b[h][1] = base[idx + 1];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = ty + 16 * h;
        const long long idx = (long long)(gi0 * LT + r) * Np + gj0 * LT + c0;
        const long long pr = (long long)(gi0 * LT + r) * 2 * Np + gj0 * LT + c0;
        float fr[2], fi[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c = c0 + e;
          const float xij_re = Xre[A][r][c], xij_im = Xim[A][r][c];
          const float xji_re = Xre[B][c][r], xji_im = Xim[B][c][r];
          const float dr = (e ? r0r[h].y : r0r[h].x) + (xij_im + xji_im);
          const float di = (e ? r0i[h].y : r0i[h].x) + (-(xij_re - xji_re));
          const double2 v = make_double2(fma(coef, f2d_bits(dr), b[h][e].x), fma(coef, f2d_bits(di), b[h][e].y));
          it.D[nxt][idx + e] = v;
          fr[e] = d2f_bits(v.x);
          fi[e] = d2f_bits(v.y);
        }
        if (it.f32) *reinterpret_cast<float4*>(it.f32 + idx) = make_float4(fr[0], fi[0], fr[1], fi[1]);
        if (it.pieces) {
          __nv_bfloat162 rh, rl, ih, il;
          rh.x = __float2bfloat16_rn(fr[0]);
          rh.y = __float2bfloat16_rn(fr[1]);
          ih.x = __float2bfloat16_rn(fi[0]);
          ih.y = __float2bfloat16_rn(fi[1]);
          rl.x = __float2bfloat16_rn(fr[0] - __bfloat162float(rh.x));
          rl.y = __float2bfloat16_rn(fr[1] - __bfloat162float(rh.y));
          il.x = __float2bfloat16_rn(fi[0] - __bfloat162float(ih.x));
          il.y = __float2bfloat16_rn(fi[1] - __bfloat162float(ih.y));
          *reinterpret_cast<__nv_bfloat162*>(it.pieces + pr) = rh;
          *reinterpret_cast<__nv_bfloat162*>(it.pieces + P + pr) = rl;
          *reinterpret_cast<__nv_bfloat162*>(it.pieces + pr + Np) = ih;
          *reinterpret_cast<__nv_bfloat162*>(it.pieces + P + pr + Np) = il;
        }
      }
    }
  }
  if (counter) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      __threadfence();
      const int total = gridDim.x * gridDim.y;
      const int ticket = atomicAdd(counter, 1);
      if (ticket == total - 1) {
        *counter = 0;
        *step_rw = n + 1;
        __threadfence();
      }
    }
  }
}

void launch_leap_split(const LeapItem* items, int n_items, int Np_max, const int* step, double dt, int* counter,
                       int* step_rw, cudaStream_t st) {
  const int nt = Np_max / LT;
  dim3 grid(nt * (nt + 1) / 2, n_items);
  dim3 block(LT / 2, LT / 2);
  launch_pdl(k_leap_split, grid, block, 0, st, items, step, dt, counter, step_rw);
}

// complex128 row-major Np x Np -> FP32 planar [Re(row) | Im(row)]
__global__ void k_to_planar_f32(const double2* src, float* dst, int Np) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Np * Np) return;
  const int i = idx / Np, j = idx % Np;
  const double2 v = src[idx];
  dst[(long long)i * 2 * Np + j] = (float)v.x;
  dst[(long long)i * 2 * Np + Np + j] = (float)v.y;
}

void launch_to_planar_f32(const double2* src, float* dst, int Np, cudaStream_t st) {
  const long long tot = (long long)Np * Np;
  k_to_planar_f32<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(src, dst, Np);
}

// complex128 -> complex64 with the leapfrog's own rounding (d2f_bits), so a
// copy rebuilt from a restored level equals the one the leapfrog wrote
__global__ void k_to_f32(const double2* src, float2* dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = src[i];
  dst[i] = make_float2(d2f_bits(v.x), d2f_bits(v.y));
}

void launch_to_f32(const double2* src, float2* dst, long long n, cudaStream_t st) {
  k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__global__ void k_fill_herm(double2* a, int n, int ld) {
  // the upper triangle (j >= i) is valid; set a[i][j] = conj(a[j][i]) for j < i
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = idx / n, j = idx % n;
  if (j < i) {
    const double2 v = a[(long long)j * ld + i];
    a[(long long)i * ld + j] = make_double2(v.x, -v.y);
  } else if (j == i) {
    a[(long long)i * ld + i].y = 0.0;
  }
}

void launch_fill_hermitian_lower(double2* a, int n, int ld, cudaStream_t st) {
  const long long tot = (long long)n * n;
  k_fill_herm<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a, n, ld);
}

__global__ void k_vt(const double2* ev, double2* vt, int n, int nocc, int ld) {
  // ev row j (j < nocc) = conj of eigenvector j; vt[r][j] = conj(ev[j][r])
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * nocc) return;
  const int r = idx / nocc, j = idx % nocc;
  const double2 v = ev[(long long)j * ld + r];
  vt[(long long)r * nocc + j] = make_double2(v.x, -v.y);
}

void launch_vt_from_evecs(const double2* evec, double2* vt, int n, int nocc, int ld, cudaStream_t st) {
  const long long tot = (long long)n * nocc;
  k_vt<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(evec, vt, n, nocc, ld);
}

__global__ void k_scale(double2* a, long long n, double s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    a[i].x *= s;
    a[i].y *= s;
  }
}

void launch_scale(double2* a, long long n, double s, cudaStream_t st) {
  k_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, s);
}

__global__ void k_split_planar(const double2* src, __nv_bfloat16* dst, int Np) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long NN = (long long)Np * Np;
  if (idx >= NN) return;
  const int i = idx / Np, j = idx % Np;
  const double2 v = src[idx];
  __nv_bfloat16 h, l;
  const long long pr = (long long)i * 2 * Np + j;
  split_bf16_d(v.x, h, l);
  dst[pr] = h;
  dst[2 * NN + pr] = l;
  split_bf16_d(v.y, h, l);
  dst[pr + Np] = h;
  dst[2 * NN + pr + Np] = l;
}

void launch_split_planar(const double2* src, __nv_bfloat16* dst, int N, int Np, cudaStream_t st) {
  (void)N;
  const long long tot = (long long)Np * Np;
  k_split_planar<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(src, dst, Np);
}

// embedded pieces [[Re, Im], [-Im, Re]] of a dense complex matrix (2Np x 2Np per
// piece) in the row order of the first product's B operand: row i of [Re, Im] at
// 8 (i / 4) + i % 4, row i of [-Im, Re] four rows further
__global__ void k_split_embedded(const double2* src, __nv_bfloat16* dst, int Np) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long NN = (long long)Np * Np;
  if (idx >= NN) return;
  const int i = idx / Np, j = idx % Np;
  const double2 v = src[idx];
  const long long ld = 2LL * Np, P = 4 * NN;
  __nv_bfloat16 rh, rl, ih, il;
  split_bf16_d(v.x, rh, rl);
  split_bf16_d(v.y, ih, il);
  const long long rr = 8LL * (i >> 2) + (i & 3), ri = rr + 4;
  const long long i00 = rr * ld + j, i01 = rr * ld + Np + j, i10 = ri * ld + j, i11 = ri * ld + Np + j;
  dst[i00] = rh;
  dst[P + i00] = rl;
  dst[i01] = ih;
  dst[P + i01] = il;
  dst[i10] = __hneg(ih);
  dst[P + i10] = __hneg(il);
  dst[i11] = rh;
  dst[P + i11] = rl;
}

void launch_split_embedded(const double2* src, __nv_bfloat16* dst, int Np, cudaStream_t st) {
  const long long tot = (long long)Np * Np;
  k_split_embedded<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(src, dst, Np);
}

// a := (a + a^dagger) / 2 (exactly Hermitian afterwards); one thread per pair i <= j
__global__ void k_hermitize(double2* a, int n, int ld) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = idx / n, j = idx % n;
  if (j < i) return;
  const double2 x = a[(long long)i * ld + j], y = a[(long long)j * ld + i];
  const double2 v = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
  if (i == j) {
    a[(long long)i * ld + i] = make_double2(v.x, 0.0);
  } else {
    a[(long long)i * ld + j] = v;
    a[(long long)j * ld + i] = make_double2(v.x, -v.y);
  }
}

void launch_hermitize(double2* a, int n, int ld, cudaStream_t st) {
  const long long tot = (long long)n * n;
  k_hermitize<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a, n, ld);
}

// ---------------------------------------------------------------------------
// Crank-Nicolson helpers
// ---------------------------------------------------------------------------
// Sets ST_CN_NOCONV on the item's trajectory when max |a - b| > tol: the last
// two fixed-point iterates still differ, so the sweep count is too small for
// this dt (or the iteration diverges, dt |S^-1 H| / 2 >= 1).
__global__ void k_cn_check(const CnCheckItem* __restrict__ items, const DevTraj* __restrict__ trj, double tol) {
  const CnCheckItem& it = items[blockIdx.y];
  const long long tot = (long long)it.rows * it.cols;
  double m = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / it.cols), c = (int)(e - (long long)r * it.cols);
    const double2 x = it.a[(long long)r * it.ld + c], y = it.b[(long long)r * it.ld + c];
    m = fmax(m, fmax(fabs(x.x - y.x), fabs(x.y - y.y)));
  }
  // a NaN difference also counts as not converged
  if (!(m <= tol)) atomicOr(trj[it.traj].status, ST_CN_NOCONV);
}

void launch_cn_check(const CnCheckItem* items, int n_items, int max_elems, const DevTraj* trj, double tol,
                     cudaStream_t st) {
  const int blocks = std::min(64, (max_elems + 255) / 256);
  k_cn_check<<<dim3(blocks > 0 ? blocks : 1, n_items), 256, 0, st>>>(items, trj, tol);
}

__global__ void k_conj_t(const double2* src, int lds, double2* dst, int ldd, int rows, int cols) {
  __shared__ double2 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int sr = c0 + y, sc = r0 + threadIdx.x;  // src row = dst column
    if (sr < cols && sc < rows) tile[y][threadIdx.x] = src[(long long)sr * lds + sc];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int dr = r0 + y, dc = c0 + threadIdx.x;
    if (dr < rows && dc < cols) {
      const double2 v = tile[threadIdx.x][y];
      dst[(long long)dr * ldd + dc] = make_double2(v.x, -v.y);
    }
  }
}

void launch_conj_transpose(const double2* src, int lds, double2* dst, int ldd, int rows, int cols, cudaStream_t st) {
  k_conj_t<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, st>>>(src, lds, dst, ldd, rows, cols);
}

__global__ void k_inc(int* s) { *s += 1; }
void launch_increment(int* step, cudaStream_t st) { k_inc<<<1, 1, 0, st>>>(step); }

}  // namespace vgtb
