// Block-sparse kernels of one propagation step:
//   k_obs         - Mulliken, current and energy partial sums from D_k(t_n) (Eqs. 10, 14)
//   k_scc_atoms,
//   k_scc_eps     - dq, eps = gamma dq, J, E per trajectory (Eq. 10, Eq. 14)
//   k_phase       - Bloch sum of H_k(t_n) with the vector potential (Eqs. 7-12), FP64
//   k_phase_split - the same sum in FP32, written as embedded BF16 hi/lo pieces
// A half-warp (16 lanes) handles one target (I, J) of one trajectory: it walks the
// target's real-space images (blocks with different L), lanes over the n_I x n_J
// elements (16 for an sp3 pair; larger blocks loop), so the block values are read
// once, coalesced, per step.  All reductions use fixed orders (lane butterflies,
// strided loops, fixed trees, a last-CTA sum), so reruns are bitwise identical.
// GB300 executes FP64 at a small fraction of its FP32 rate, so FP64 is kept to the
// reductions that need it; the split form builds its BF16 operands in FP32.
#include "vgtb_internal.h"

namespace vgtb {

__device__ __forceinline__ int find_traj(const int* pre, int n, int w) {
  int lo = 0, hi = n;  // pre[lo] <= w < pre[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= w) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the 16 lanes of a half-warp (both halves reduce independently)
__device__ __forceinline__ double half_sum(double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Unit {
  bool active;
  int t, tg;
};

// unit = (trajectory, target), one per half-warp
__device__ __forceinline__ Unit unit_of(const int* wpre, int n_traj, int total) {
  const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  Unit r;
  r.active = u < total;
  r.t = r.active ? find_traj(wpre, n_traj, u) : 0;
  r.tg = r.active ? u - wpre[r.t] : 0;
  return r;
}

// ---------------------------------------------------------------------------
// Partial sums per target, summed over k with weights w_k, from the
// time-independent k-space blocks S_k, P_k^a, H0_k (Bloch-summed at setup):
//   s_S = sum Re(D conj(S_k)),  s_a = sum Re(D conj(P^a_k)),  s_H = sum Re(D conj(H0_k))
//   q = s_S                                          (Eq. 10: [D S]_{mu mu})
//   T_a = s_a + (A_a/c) s_S                          (Eq. 14: Tr[D Pi^a], Pi = P + (A/c) S)
//   E_band = s_H + (A/c).(s_x, s_y, s_z) + |A|^2/(2c^2) s_S
// In the delta forms D = D0 + dD and the D0 part of every sum is a constant
// computed once (obs0), so only dD is read.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_obs(const DevSys* __restrict__ sysv, const DevTraj* __restrict__ trj,
                                             const DevItem* __restrict__ items, const int* __restrict__ wpre,
                                             int n_traj, int total, const int* __restrict__ step, int delta,
                                             int fixed_step) {
  pdl_wait();
  pdl_trigger();
  const Unit U = unit_of(wpre, n_traj, total);
  const int lane = threadIdx.x & 15;
  double sS = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, sH = 0.0;
  const DevTraj& T = trj[U.t];
  const DevSys& S = sysv[T.sys];
  int n = 0;
  if (U.active) {
    n = fixed_step >= 0 ? fixed_step : *step;
    const int par = n & 1;
    const int I = S.tgt_I[U.tg], J = S.tgt_J[U.tg];
    const int oi = S.orb_off[I];
    const int oj = S.orb_off[J], nj = S.orb_off[J + 1] - oj;
    const int el0 = S.tgt_el0[U.tg], nel = S.tgt_el0[U.tg + 1] - el0;
    for (int k = 0; k < S.nk; ++k) {
      const double2* Dk = items[T.item0 + k].D[par];
      const long long kb = (long long)k * S.n_el + el0;
      const long long pstride = (long long)S.nk * S.n_el;
      double lS = 0.0, lx = 0.0, ly = 0.0, lz = 0.0, lH = 0.0;
      for (int e = lane; e < nel; e += 16) {
        const int a = e / nj, b = e - a * nj;
        const double2 d = Dk[(long long)(oi + a) * S.Np + (oj + b)];
        const double2 cs = S.kS[kb + e], ch = S.kH0[kb + e];
        const double2 px = S.kP[kb + e], py = S.kP[pstride + kb + e], pz = S.kP[2 * pstride + kb + e];
        lS += d.x * cs.x + d.y * cs.y;
        lx += d.x * px.x + d.y * px.y;
        ly += d.x * py.x + d.y * py.y;
        lz += d.x * pz.x + d.y * pz.y;
        lH += d.x * ch.x + d.y * ch.y;
      }
      const double wk = S.wk[k];
      sS += wk * lS;
      sx += wk * lx;
      sy += wk * ly;
      sz += wk * lz;
      sH += wk * lH;
    }
  }
  sS = half_sum(sS);
  sx = half_sum(sx);
  sy = half_sum(sy);
  sz = half_sum(sz);
  sH = half_sum(sH);
  if (U.active && lane == 0) {
    if (delta) {
      const double* o = S.obs0 + 5LL * U.tg;
      sS += o[0];
      sx += o[1];
      sy += o[2];
      sz += o[3];
      sH += o[4];
    }
    double A0 = 0.0, A1 = 0.0, A2 = 0.0;
    if (T.A) {
      A0 = T.A[3 * n];
      A1 = T.A[3 * n + 1];
      A2 = T.A[3 * n + 2];
    }
    constexpr double ic = 1.0 / kLight;
    const double a0 = A0 * ic, a1 = A1 * ic, a2 = A2 * ic;
    const double alpha = 0.5 * (a0 * a0 + a1 * a1 + a2 * a2);
    double* p = T.part + 5LL * U.tg;
    p[0] = sS;
    p[1] = sx + a0 * sS;
    p[2] = sy + a1 * sS;
    p[3] = sz + a2 * sS;
    p[4] = sH + (a0 * sx + a1 * sy + a2 * sz) + alpha * sS;
  }
}

// Setup: the k-space blocks of one system at one k (half-warp per target).
__global__ void k_kblocks(const DevSys* __restrict__ sysv, int s_idx, int k) {
  const int tg = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int lane = threadIdx.x & 15;
  const DevSys& S = sysv[s_idx];
  if (tg >= S.n_tgt) return;
  const int el0 = S.tgt_el0[tg], nel = S.tgt_el0[tg + 1] - el0;
  const long long kb = (long long)k * S.n_el + el0, pstride = (long long)S.nk * S.n_el;
  for (int e = lane; e < nel; e += 16) {
    double2 s = make_double2(0.0, 0.0), h = s, px = s, py = s, pz = s;
    for (int g = S.tgt_img0[tg]; g < S.tgt_img0[tg + 1]; ++g) {
      const long long off = S.img_off[g] + e;
      const double2 ph = S.phase[(long long)k * S.n_blk + S.img_blk[g]];
      const double sv = S.s[off], hv = S.h0[off];
      s.x += ph.x * sv;
      s.y += ph.y * sv;
      h.x += ph.x * hv;
      h.y += ph.y * hv;
      // ph * (i ds):  (-ph.y ds, ph.x ds)
      const double dx = S.ds[off], dy = S.ds[S.ds_stride + off], dz = S.ds[2 * S.ds_stride + off];
      px.x -= ph.y * dx;
      px.y += ph.x * dx;
      py.x -= ph.y * dy;
      py.y += ph.x * dy;
      pz.x -= ph.y * dz;
      pz.y += ph.x * dz;
    }
    S.kS[kb + e] = s;
    S.kH0[kb + e] = h;
    S.kP[kb + e] = px;
    S.kP[pstride + kb + e] = py;
    S.kP[2 * pstride + kb + e] = pz;
  }
}

void launch_kblocks(const DevSys* sys, int s_idx, int n_tgt, int k, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (n_tgt * 16 + threads - 1) / threads;
  k_kblocks<<<blocks, threads, 0, st>>>(sys, s_idx, k);
}

// Setup (delta forms): obs0[tg] = the k_obs sums of the target evaluated with D0.
__global__ void k_obs0(const DevSys* __restrict__ sysv, int s_idx) {
  const int tg = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int lane = threadIdx.x & 15;
  const DevSys& S = sysv[s_idx];
  const bool active = tg < S.n_tgt;
  double v[5] = {0, 0, 0, 0, 0};
  if (active) {
    const int I = S.tgt_I[tg], J = S.tgt_J[tg];
    const int oi = S.orb_off[I];
    const int oj = S.orb_off[J], nj = S.orb_off[J + 1] - oj;
    const int el0 = S.tgt_el0[tg], nel = S.tgt_el0[tg + 1] - el0;
    const long long NN = (long long)S.Np * S.Np, pstride = (long long)S.nk * S.n_el;
    for (int k = 0; k < S.nk; ++k) {
      const long long kb = (long long)k * S.n_el + el0;
      double l[5] = {0, 0, 0, 0, 0};
      for (int e = lane; e < nel; e += 16) {
        const int a = e / nj, b = e - a * nj;
        const double2 d = S.D0[k * NN + (long long)(oi + a) * S.Np + (oj + b)];
        const double2 c[5] = {S.kS[kb + e], S.kP[kb + e], S.kP[pstride + kb + e], S.kP[2 * pstride + kb + e],
                              S.kH0[kb + e]};
#pragma unroll
        for (int i = 0; i < 5; ++i) l[i] += d.x * c[i].x + d.y * c[i].y;
      }
#pragma unroll
      for (int i = 0; i < 5; ++i) v[i] += S.wk[k] * l[i];
    }
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) v[i] = half_sum(v[i]);
  if (active && lane == 0)
    for (int i = 0; i < 5; ++i) S.obs0[5LL * tg + i] = v[i];
}

// Setup (split form): obs0a[I] = obs0 summed over the targets of row atom I, in target order.
__global__ void k_obs0_atoms(const DevSys* __restrict__ sysv, int s_idx) {
  const DevSys& S = sysv[s_idx];
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= S.nat) return;
  double v[5] = {0, 0, 0, 0, 0};
  for (int tg = S.atom_tgt0[I]; tg < S.atom_tgt0[I + 1]; ++tg)
    for (int i = 0; i < 5; ++i) v[i] += S.obs0[5LL * tg + i];
  for (int i = 0; i < 5; ++i) S.obs0a[5LL * I + i] = v[i];
}

void launch_obs0(const DevSys* sys, int s_idx, int n_tgt, int nat, int split, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (n_tgt * 16 + threads - 1) / threads;
  k_obs0<<<blocks, threads, 0, st>>>(sys, s_idx);
  if (split) k_obs0_atoms<<<(nat + 127) / 128, 128, 0, st>>>(sys, s_idx);
}

__device__ __forceinline__ float half_sum_f(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// k_obs_atoms_split: the split form's observables and per-atom sums in one
// launch.  One CTA of 4 warps per (trajectory, atom I); its threads take the
// nonzeros of the atom's rows (all targets (I, J), ~490 for an sp3 atom, so at
// most a few per thread, whose loads are issued together) and form the dD
// sums in FP64 from the FP64 master dD and the FP64 k-space blocks (S_k, P_k,
// H0_k), so charges, current and energy keep the precision of the master copy.
// Each warp reduces its five sums with one reduce-scatter (nine FP64 additions
// per lane: GB300 issues FP64 warp instructions at a small fraction of the FP32
// rate whatever the number of active lanes), thread 0 adds the warps, the
// constant D0 part (obs0a) and the A terms (both linear in the sums) and writes
// dq_I, q_I and the atom's shares of T and of the band energy, as k_scc_atoms
// does for the FP64 paths.
// ---------------------------------------------------------------------------
constexpr int kObsThreads = 128;
constexpr int kObsChunk = 4;  // nonzeros per thread whose loads are issued together

// Reduce-scatter of eight per-lane values over a warp: afterwards lane l holds
// the warp total of value (l >> 2) & 7 (every lane of a group of four holds the
// same total).  Nine FP64 additions per lane instead of the 5 x 5 of five
// butterflies.
__device__ __forceinline__ double warp_reduce_scatter8(double (&v)[8], int lane) {
  // xor 16: keep values 0-3 (lower half-warp) or 4-7 (upper), add the partner's copy of them
  const bool up16 = lane & 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double send = up16 ? v[i] : v[i + 4];
    const double keep = up16 ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  // xor 8: keep 2 of the 4
  const bool up8 = lane & 8;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double send = up8 ? v[i] : v[i + 2];
    const double keep = up8 ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  // xor 4: keep 1 of the 2
  const bool up4 = lane & 4;
  {
    const double send = up4 ? v[0] : v[1];
    const double keep = up4 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  // lanes with the same bits 4..2 hold the same value: finish over bits 1, 0
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}

__global__ void __launch_bounds__(kObsThreads, 4) k_obs_atoms_split(const DevSys* __restrict__ sysv, DevTraj* trj,
                                                               const DevItem* __restrict__ items, int n_traj,
                                                               int max_nat, const int* __restrict__ step, int stride,
                                                               int fixed_step, int record) {
  pdl_wait();
  pdl_trigger();
  constexpr int NW = kObsThreads / 32;
  __shared__ double s_tot[NW][5];
  const int t = blockIdx.x / max_nat, I = blockIdx.x % max_nat;
  if (t >= n_traj) return;
  DevTraj& T = trj[t];
  const DevSys& S = sysv[T.sys];
  if (I >= S.nat) return;
  const int n = fixed_step >= 0 ? fixed_step : *step;
  const int par = n & 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // S, P_x, P_y, P_z, H0 sums (3 slots unused)
  // the atom's nonzeros are contiguous (targets sorted by row atom); el_off gives
  // each one's offset in the Np x Np matrix
  const int e0 = S.el_atom0[I], e1 = S.el_atom0[I + 1];
  const long long ps = (long long)S.nk * S.n_el;
  for (int k = 0; k < S.nk; ++k) {
    const double2* Dk = items[T.item0 + k].D[par];
    const long long kb = (long long)k * S.n_el;
    double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int eb = e0; eb < e1; eb += kObsThreads * kObsChunk) {
      int ee[kObsChunk];
      bool ok[kObsChunk];
      double2 d[kObsChunk];
#pragma unroll
      for (int u = 0; u < kObsChunk; ++u) {
        const int e = eb + threadIdx.x + kObsThreads * u;
        ok[u] = e < e1;
        ee[u] = ok[u] ? e : e0;
      }
#pragma unroll
      for (int u = 0; u < kObsChunk; ++u) d[u] = ok[u] ? Dk[S.el_off[ee[u]]] : make_double2(0.0, 0.0);
#pragma unroll
      for (int u = 0; u < kObsChunk; ++u) {
        const long long x = kb + ee[u];
        const double2 bs = S.kS[x], bx = S.kP[x], by = S.kP[ps + x], bz = S.kP[2 * ps + x], bh = S.kH0[x];
        // Re(dD conj(X)) for X = S_k, P_k^x, P_k^y, P_k^z, H0_k
        c[0] = fma(d[u].x, bs.x, fma(d[u].y, bs.y, c[0]));
        c[1] = fma(d[u].x, bx.x, fma(d[u].y, bx.y, c[1]));
        c[2] = fma(d[u].x, by.x, fma(d[u].y, by.y, c[2]));
        c[3] = fma(d[u].x, bz.x, fma(d[u].y, bz.y, c[3]));
        c[4] = fma(d[u].x, bh.x, fma(d[u].y, bh.y, c[4]));
      }
    }
    const double w = S.wk[k];
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = fma(w, c[i], v[i]);
  }
  const double tot = warp_reduce_scatter8(v, lane);
  const int slot = (lane >> 2) & 7;
  if ((lane & 3) == 0 && slot < 5) s_tot[warp][slot] = tot;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double r[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    double a = S.obs0a[5LL * I + i];
    for (int w2 = 0; w2 < NW; ++w2) a += s_tot[w2][i];
    r[i] = a;
  }
  double A0 = 0.0, A1 = 0.0, A2 = 0.0;
  if (T.A) {
    A0 = T.A[3 * n];
    A1 = T.A[3 * n + 1];
    A2 = T.A[3 * n + 2];
  }
  constexpr double ic = 1.0 / kLight;
  const double a0 = A0 * ic, a1 = A1 * ic, a2 = A2 * ic;
  const double alpha = 0.5 * (a0 * a0 + a1 * a1 + a2 * a2);
  T.dq[I] = r[0] - S.z[I];
  if (record && T.q && n % stride == 0) T.q[(long long)(n / stride) * S.nat + I] = r[0];
  double* ap = T.apart + 4LL * I;
  ap[0] = r[1] + a0 * r[0];
  ap[1] = r[2] + a1 * r[0];
  ap[2] = r[3] + a2 * r[0];
  ap[3] = r[4] + (a0 * r[1] + a1 * r[2] + a2 * r[3]) + alpha * r[0];
}

void launch_obs_atoms_split(const DevSys* sys, DevTraj* trj, const DevItem* items, int n_traj, int max_nat,
                            const int* step, int stride, int fixed_step, int record, cudaStream_t st) {
  launch_pdl(k_obs_atoms_split, n_traj * max_nat, kObsThreads, 0, st, sys, trj, items, n_traj, max_nat, step, stride,
             fixed_step, record);
}

void launch_obs(const DevSys* sys, const DevTraj* trj, const DevItem* items, const int* warp_prefix,
                int n_traj, int total_units, const int* step, int delta, int fixed_step, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (total_units * 16 + threads - 1) / threads;
  launch_pdl(k_obs, blocks, threads, 0, st, sys, trj, items, warp_prefix, n_traj, total_units, step, delta,
             fixed_step);
}

// ---------------------------------------------------------------------------
// SCC reduction in two launches per step (all trajectories at once):
//   k_scc_atoms: one warp per atom sums the partials of the atom's targets
//                (targets are sorted by row atom): q_I, dq_I, and the atom's
//                share of T_a and of the band energy;
//   k_scc_eps:   kSccRows rows of eps = gamma dq per CTA, one per warp (Eq. 10), and one
//                partial of J, the band energy, dq.eps/2 and the electron count per CTA;
//                scc_finish adds the partials in a fixed order (J of Eq. 14, the energy,
//                the checks): run by the last CTA of k_scc_eps, or, in the split form's
//                step, by a finisher CTA of k_phase_split.
// ---------------------------------------------------------------------------
constexpr int kSccThreads = 32 * kSccRowsPerCta;
constexpr int kSccRows = kSccRowsPerCta;
constexpr int kAtomsPerCta = kSccThreads / 32;

__global__ void __launch_bounds__(kSccThreads) k_scc_atoms(const DevSys* __restrict__ sysv, DevTraj* trj, int n_traj,
                                                          int nblk, const int* __restrict__ step, int stride,
                                                          int fixed_step, int record) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x / nblk, b = blockIdx.x % nblk;
  if (t >= n_traj) return;
  DevTraj& T = trj[t];
  const DevSys& S = sysv[T.sys];
  const int I = b * kAtomsPerCta + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (I >= S.nat) return;
  const int n = fixed_step >= 0 ? fixed_step : *step;
  double v[5] = {0, 0, 0, 0, 0};
  for (int tg = S.atom_tgt0[I] + lane; tg < S.atom_tgt0[I + 1]; tg += 32) {
    const double* p = T.part + 5LL * tg;
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] += p[i];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0) {
    T.dq[I] = v[0] - S.z[I];
    if (record && T.q && n % stride == 0) T.q[(long long)(n / stride) * S.nat + I] = v[0];
    double* a = T.apart + 4LL * I;
    a[0] = v[1];
    a[1] = v[2];
    a[2] = v[3];
    a[3] = v[4];
  }
}

// The trajectory's totals at level n from the per-CTA partials of k_scc_eps, in a
// fixed order (lane-strided sums, then a butterfly): J (Eq. 14), the energy, and
// the checks of the level.  Run by one warp: the last CTA of k_scc_eps, or a
// finisher CTA of k_phase_split (the split form's step, where the phase build
// does not wait for these totals).
__device__ void scc_finish(DevTraj& T, const DevSys& S, int n, int record, int lane) {
  const int myblk = (S.nat + kSccRows - 1) / kSccRows;
  double v[6] = {0, 0, 0, 0, 0, 0};  // Tx, Ty, Tz, E_band, dq.eps, electron count
  for (int c = lane; c < myblk; c += 32) {
    const double* cp = T.cpart + 6LL * c;
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] += cp[i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0) {
    const double J0 = -v[0] * S.inv_omega, J1 = -v[1] * S.inv_omega, J2 = -v[2] * S.inv_omega;
    const double E = v[3] + 0.5 * v[4];
    if (record) {
      T.J[3LL * n] = J0;
      T.J[3LL * n + 1] = J1;
      T.J[3LL * n + 2] = J2;
      T.E[n] = E;
    }
    int st = 0;
    if (!isfinite(J0) || !isfinite(J1) || !isfinite(J2) || !isfinite(E) || !isfinite(v[5])) st |= ST_NONFINITE;
    if (fabs(v[5] - S.nel) > 1e-6 * fmax(1.0, S.nel)) st |= ST_DRIFT;
    if (st) atomicOr(T.status, st);
  }
}

// finish = 1: the last CTA of each trajectory runs scc_finish; finish = 0: the
// CTAs only store their partials (the step's k_phase_split finishes them).
__global__ void __launch_bounds__(kSccThreads) k_scc_eps(const DevSys* __restrict__ sysv, DevTraj* trj, int n_traj,
                                                        int nblk, const int* __restrict__ step, int fixed_step,
                                                        int record, int finish) {
  pdl_wait();
  pdl_trigger();
  constexpr int NW = kSccThreads / 32;
  __shared__ double red[NW][6];
  __shared__ int s_last;
  const int t = blockIdx.x / nblk, b = blockIdx.x % nblk;
  if (t >= n_traj) return;
  DevTraj& T = trj[t];
  const DevSys& S = sysv[T.sys];
  const int myblk = (S.nat + kSccRows - 1) / kSccRows;
  if (b >= myblk) return;
  const int n = fixed_step >= 0 ? fixed_step : *step;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int I = b * kSccRows + warp;  // one warp per row of gamma
  if (tid == 0 && b == 0 && T.af) {
    // A(t_n)/c in FP32 for the phase build
    constexpr double inv_c = 1.0 / kLight;
    for (int a = 0; a < 3; ++a) T.af[a] = (float)((T.A ? T.A[3 * n + a] : 0.0) * inv_c);
  }
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 6; ++i) red[warp][i] = 0.0;
  if (I < S.nat) {
    const double* g = S.gamma + (long long)I * S.nat;
    const double* dq = T.dq;
    // chunks of 512 columns: all 16 loads of a lane are issued before the first
    // FMA, so a chunk costs one memory latency; four partial sums
    double e0 = 0.0, e1 = 0.0, e2 = 0.0, e3 = 0.0;
    for (int base = 0; base < S.nat; base += 512) {
      double gv[16], qv[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int K = base + lane + 32 * j;
        gv[j] = K < S.nat ? g[K] : 0.0;
        qv[j] = K < S.nat ? dq[K] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < 16; j += 4) {
        e0 = fma(gv[j], qv[j], e0);
        e1 = fma(gv[j + 1], qv[j + 1], e1);
        e2 = fma(gv[j + 2], qv[j + 2], e2);
        e3 = fma(gv[j + 3], qv[j + 3], e3);
      }
    }
    const double e = warp_sum((e0 + e1) + (e2 + e3));
    if (lane == 0) {
      // the Hamiltonian's shift: gamma dq (Eq. 10), or the shift of D(0) when
      // frozen; the energy below uses gamma dq either way
      const double eh = S.scc_frozen ? S.eps0[I] : e;
      T.eps[I] = eh;
      if (T.eps_lv) T.eps_lv[(long long)(n & 1) * S.nat + I] = eh;
      if (T.epsf) {
        T.epsf[I] = (float)eh;
        T.depsf[I] = (float)(eh - S.eps0[I]);
      }
      // this atom's shares of T_x, T_y, T_z, the band energy, dq.eps and the electron count
      const double* a = T.apart + 4LL * I;
      red[warp][0] = a[0];
      red[warp][1] = a[1];
      red[warp][2] = a[2];
      red[warp][3] = a[3];
      red[warp][4] = dq[I] * e;
      red[warp][5] = dq[I] + S.z[I];
    }
  }
  __syncthreads();
  // the CTA's partial in a fixed order, then (finish) the last CTA adds the partials
  if (tid == 0) {
    double* cp = T.cpart + 6LL * b;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double v = red[0][i];
      for (int w = 1; w < NW; ++w) v += red[w][i];
      cp[i] = v;
    }
    if (finish) {
      __threadfence();
      s_last = (atomicAdd(T.ticket, 1) == myblk - 1);
    }
  }
  if (!finish) return;
  __syncthreads();
  if (!s_last || warp != 0) return;
  __threadfence();
  scc_finish(T, S, n, record, lane);
  if (lane == 0) *T.ticket = 0;
}

void launch_scc(const DevSys* sys, DevTraj* trj, int n_traj, const int* step, int stride, int fixed_step,
                int record, int max_nat, int atoms_done, cudaStream_t st, int finish) {
  const int nblk_a = (max_nat + kAtomsPerCta - 1) / kAtomsPerCta;
  if (!atoms_done)
    launch_pdl(k_scc_atoms, n_traj * nblk_a, kSccThreads, 0, st, sys, trj, n_traj, nblk_a, step, stride, fixed_step,
               record);
  const int nblk = (max_nat + kSccRows - 1) / kSccRows;
  launch_pdl(k_scc_eps, n_traj * nblk, kSccThreads, 0, st, sys, trj, n_traj, nblk, step, fixed_step, record, finish);
}

int scc_configure(int max_nat) {
  (void)max_nat;  // the reduction needs no dynamic shared memory
  return 0;
}


// ---------------------------------------------------------------------------
// Phase build, FP64 path: H_k(t)_{mu nu} = sum_images e^{-ik.L} v_{mu nu}(L) with
//   plain: v = H0 + (alpha + (eps_I + eps_J)/2) S + (i/c) A.dS        (Eqs. 9-12)
//   delta: H without alpha (its commutator vanishes, remark after Eq. 3) and
//          dH = ((eps_I-eps0_I) + (eps_J-eps0_J))/2 S + (i/c) A.dS.
//   CN:    H(t_{n+1/2}) without alpha (an overall phase of the states, remark
//          after Eq. 3) from A_{n+1/2} = (A_n + A_{n+1})/2 and the shift
//          extrapolated from the two latest levels, (3 eps_n - eps_{n-1})/2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_phase(const DevSys* __restrict__ sysv, const DevTraj* __restrict__ trj,
                                               const DevItem* __restrict__ items, const int* __restrict__ wpre,
                                               int n_traj, int total, const int* __restrict__ step, int mode,
                                               int fixed_step) {
  pdl_wait();
  pdl_trigger();
  const Unit U = unit_of(wpre, n_traj, total);
  if (!U.active) return;
  const int lane = threadIdx.x & 15;
  const DevTraj& T = trj[U.t];
  const DevSys& S = sysv[T.sys];
  const int n = fixed_step >= 0 ? fixed_step : *step;
  double A0 = 0.0, A1 = 0.0, A2 = 0.0;
  if (T.A) {
    A0 = T.A[3 * n];
    A1 = T.A[3 * n + 1];
    A2 = T.A[3 * n + 2];
    if (mode == PH_FP64_CN) {  // A(t_{n+1/2}) = (A_n + A_{n+1}) / 2
      A0 = 0.5 * (A0 + T.A[3 * n + 3]);
      A1 = 0.5 * (A1 + T.A[3 * n + 4]);
      A2 = 0.5 * (A2 + T.A[3 * n + 5]);
    }
  }
  const double ic = 1.0 / kLight;
  const double alpha = (A0 * A0 + A1 * A1 + A2 * A2) * 0.5 * ic * ic;
  const int I = S.tgt_I[U.tg], J = S.tgt_J[U.tg];
  const int oi = S.orb_off[I], ni = S.orb_off[I + 1] - oi;
  const int oj = S.orb_off[J], nj = S.orb_off[J + 1] - oj;
  const int nel = ni * nj;
  const int g0 = S.tgt_img0[U.tg], g1 = S.tgt_img0[U.tg + 1];
  double eI = T.eps[I], eJ = T.eps[J];
  if (mode == PH_FP64_CN && n > 0) {  // eps(t_{n+1/2}) = (3 eps_n - eps_{n-1}) / 2
    const double* cur = T.eps_lv + (long long)(n & 1) * S.nat;
    const double* prv = T.eps_lv + (long long)((n - 1) & 1) * S.nat;
    eI = 1.5 * cur[I] - 0.5 * prv[I];
    eJ = 1.5 * cur[J] - 0.5 * prv[J];
  }
  const double ebar = 0.5 * (eI + eJ);
  const double beta = (mode == PH_FP64_PLAIN) ? alpha + ebar : ebar;
  const double dbeta = (mode == PH_FP64_PLAIN) ? 0.0 : 0.5 * ((T.eps[I] - S.eps0[I]) + (T.eps[J] - S.eps0[J]));
  for (int k = 0; k < S.nk; ++k) {
    const DevItem& it = items[T.item0 + k];
    for (int e = lane; e < nel; e += 16) {
      const int a = e / nj, b = e - a * nj;
      const long long idx = (long long)(oi + a) * S.Np + (oj + b);
      double hr = 0.0, hi = 0.0, dr = 0.0, di = 0.0;
      for (int g = g0; g < g1; ++g) {
        const long long off = S.img_off[g] + e;
        const double sv = S.s[off], hv = S.h0[off];
        const double adS = (A0 * S.ds[off] + A1 * S.ds[S.ds_stride + off] + A2 * S.ds[2 * S.ds_stride + off]) * ic;
        const double2 ph = S.phase[(long long)k * S.n_blk + S.img_blk[g]];
        const double vr = hv + beta * sv;  // v = vr + i adS
        hr += ph.x * vr - ph.y * adS;
        hi += ph.x * adS + ph.y * vr;
        const double wr = dbeta * sv;       // dv = wr + i adS
        dr += ph.x * wr - ph.y * adS;
        di += ph.x * adS + ph.y * wr;
      }
      if (it.kH) {
        // block-sparse first product: the target's elements, in target order
        const long long ce = S.tgt_el0[U.tg] + e;
        reinterpret_cast<double2*>(it.kH)[ce] = make_double2(hr, hi);
        if (mode == PH_FP64_DELTA) reinterpret_cast<double2*>(it.kdH)[ce] = make_double2(dr, di);
      } else {
        it.H[idx] = make_double2(hr, hi);
        if (mode == PH_FP64_DELTA) it.dH[idx] = make_double2(dr, di);
      }
    }
  }
}

void launch_phase(const DevSys* sys, const DevTraj* trj, const DevItem* items, const int* warp_prefix,
                  int n_traj, int total_units, const int* step, int mode, int fixed_step, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (total_units * 16 + threads - 1) / threads;
  launch_pdl(k_phase, blocks, threads, 0, st, sys, trj, items, warp_prefix, n_traj, total_units, step, mode,
             fixed_step);
}

// ---------------------------------------------------------------------------
// Phase build, split form: the delta-form H and dH summed in FP32 and stored
// either at the target elements in FP32 (block-sparse first product) or as the
// embedded real matrix [[Re, Im], [-Im, Re]] in BF16 hi/lo pieces (the B
// operand of the tcgen05 first product), whose rows the first product takes
// interleaved in blocks of four: row r of [Re, Im] is stored as row
// emb_row_re(r) = 8 (r / 4) + r % 4 and row r of [-Im, Re] as emb_row_re(r) + 4.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long emb_row_re(int r) { return 8LL * (r >> 2) + (r & 3); }

__device__ __forceinline__ void store_emb_f(__nv_bfloat16* base, int Np, int r, int c, float re, float im) {
  const long long P = 4LL * Np * Np;
  const long long ld = 2LL * Np;
  const __nv_bfloat16 rh = __float2bfloat16_rn(re), ih = __float2bfloat16_rn(im);
  const __nv_bfloat16 rl = __float2bfloat16_rn(re - __bfloat162float(rh));
  const __nv_bfloat16 il = __float2bfloat16_rn(im - __bfloat162float(ih));
  const long long i00 = emb_row_re(r) * ld + c;
  const long long i01 = emb_row_re(r) * ld + Np + c;
  const long long i10 = (emb_row_re(r) + 4) * ld + c;
  const long long i11 = (emb_row_re(r) + 4) * ld + Np + c;
  base[i00] = rh;
  base[P + i00] = rl;
  base[i01] = ih;
  base[P + i01] = il;
  base[i10] = __hneg(ih);
  base[P + i10] = __hneg(il);
  base[i11] = rh;
  base[P + i11] = rl;
}

// unit = (trajectory, target), one per 4 lanes (vectorised phase build)
__device__ __forceinline__ Unit unit_of_q(const int* wpre, int n_traj, int total) {
  const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  Unit r;
  r.active = u < total;
  r.t = r.active ? find_traj(wpre, n_traj, u) : 0;
  r.tg = r.active ? u - wpre[r.t] : 0;
  return r;
}

__device__ __forceinline__ uint2 pack_bf16x4(const __nv_bfloat16 (&v)[4]) {
  uint2 o;
  o.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
  o.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
  return o;
}

// four consecutive columns c..c+3 of row r (c a multiple of 4): one 8-byte store per
// quadrant of [[Re, Im], [-Im, Re]] and per piece (rows interleaved as above)
__device__ __forceinline__ void store_emb_f4(__nv_bfloat16* base, int Np, int r, int c, const float (&re)[4],
                                             const float (&im)[4]) {
  const long long P = 4LL * Np * Np;
  const long long ld = 2LL * Np;
  __nv_bfloat16 rh[4], rl[4], ih[4], il[4], nh[4], nl[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    rh[j] = __float2bfloat16_rn(re[j]);
    ih[j] = __float2bfloat16_rn(im[j]);
    rl[j] = __float2bfloat16_rn(re[j] - __bfloat162float(rh[j]));
    il[j] = __float2bfloat16_rn(im[j] - __bfloat162float(ih[j]));
    nh[j] = __hneg(ih[j]);
    nl[j] = __hneg(il[j]);
  }
  const long long i00 = emb_row_re(r) * ld + c;
  const long long i01 = emb_row_re(r) * ld + Np + c;
  const long long i10 = (emb_row_re(r) + 4) * ld + c;
  const long long i11 = (emb_row_re(r) + 4) * ld + Np + c;
  const uint2 prh = pack_bf16x4(rh), prl = pack_bf16x4(rl);
  *reinterpret_cast<uint2*>(base + i00) = prh;
  *reinterpret_cast<uint2*>(base + P + i00) = prl;
  *reinterpret_cast<uint2*>(base + i01) = pack_bf16x4(ih);
  *reinterpret_cast<uint2*>(base + P + i01) = pack_bf16x4(il);
  *reinterpret_cast<uint2*>(base + i10) = pack_bf16x4(nh);
  *reinterpret_cast<uint2*>(base + P + i10) = pack_bf16x4(nl);
  *reinterpret_cast<uint2*>(base + i11) = prh;
  *reinterpret_cast<uint2*>(base + P + i11) = prl;
}

// Four lanes per target.  Targets whose blocks have 4 columns and 16-byte aligned
// values (tgt_vec: every sp3-sp3 pair) read each block row with float4 loads and
// write 4 columns per store; other shapes take the element loop.
// CTAs from `fin0` on (grid row 0 only, one per trajectory) are finishers: they add
// up k_scc_eps's partials of the level (scc_finish), in parallel with the build.
__global__ void __launch_bounds__(256, 4) k_phase_split(const DevSys* __restrict__ sysv,
                                                     DevTraj* __restrict__ trj,
                                                     const DevItem* __restrict__ items,
                                                     const int* __restrict__ wpre, int n_traj, int total,
                                                     int fin0, const int* __restrict__ step) {
  pdl_wait();
  pdl_trigger();
  if (fin0 >= 0 && (int)blockIdx.x >= fin0) {
    const int t = (int)blockIdx.x - fin0;
    if (blockIdx.y != 0 || t >= n_traj || threadIdx.x >= 32) return;
    scc_finish(trj[t], sysv[trj[t].sys], *step, 1, threadIdx.x);
    return;
  }
  const Unit U = unit_of_q(wpre, n_traj, total);
  if (!U.active) return;
  const int sub = threadIdx.x & 3;
  const DevTraj& T = trj[U.t];
  const DevSys& S = sysv[T.sys];
  // A(t_n)/c and the shifts as FP32, prepared once per step by k_scc_eps: the
  // kernel issues no FP64 instruction (each costs a warp many FP32 issue slots)
  const float a0 = T.af[0], a1 = T.af[1], a2 = T.af[2];
  // the target's constants in two 16-byte records (one load each, no lookups)
  const int4 t0 = S.tgt_p0[U.tg], t1 = S.tgt_p1[U.tg];
  const int I = t0.x, J = t0.y, g0 = t0.z, g1 = t0.w;
  const int oi = t1.x, oj = t1.y, ni = t1.z & 0xffff, nj = t1.w & 0xffff;
  const bool vec = (t1.z >> 16) != 0;
  const int nel = ni * nj;
  const float beta = 0.5f * (T.epsf[I] + T.epsf[J]);
  const float dbeta = 0.5f * (T.depsf[I] + T.depsf[J]);
  const long long dss = S.ds_stride;
  // one k-point per grid row (blockIdx.y): the k-points of a target run in parallel
  for (int k = blockIdx.y; k < S.nk; k += gridDim.y) {
    const DevItem& it = items[T.item0 + k];
    if (vec) {
      for (int r = sub; r < ni; r += 4) {
        float hr[4] = {0.f, 0.f, 0.f, 0.f}, hi[4] = {0.f, 0.f, 0.f, 0.f};
        float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
        for (int g = g0; g < g1; ++g) {
          const long long off = S.img_off[g] + 4LL * r;
          const float4 sv = *reinterpret_cast<const float4*>(S.sf + off);
          const float4 hv = *reinterpret_cast<const float4*>(S.h0f + off);
          const float4 dx = *reinterpret_cast<const float4*>(S.dsf + off);
          const float4 dy = *reinterpret_cast<const float4*>(S.dsf + dss + off);
          const float4 dz = *reinterpret_cast<const float4*>(S.dsf + 2 * dss + off);
          const float2 ph = S.phase_img[(long long)k * S.n_img + g];  // e^{-i 2 pi k.n} of image g
          const float s4[4] = {sv.x, sv.y, sv.z, sv.w}, h4[4] = {hv.x, hv.y, hv.z, hv.w};
          const float x4[4] = {dx.x, dx.y, dx.z, dx.w}, y4[4] = {dy.x, dy.y, dy.z, dy.w};
          const float z4[4] = {dz.x, dz.y, dz.z, dz.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float adS = a0 * x4[j] + a1 * y4[j] + a2 * z4[j];
            const float vr = h4[j] + beta * s4[j];
            hr[j] += ph.x * vr - ph.y * adS;
            hi[j] += ph.x * adS + ph.y * vr;
            const float wr = dbeta * s4[j];
            dr[j] += ph.x * wr - ph.y * adS;
            di[j] += ph.x * adS + ph.y * wr;
          }
        }
        if (it.kH) {
          // block-sparse first product: row r of the target's 4 x 4 block (every
          // atom has 4 orbitals there, so the element index is a multiple of 4)
          const long long ce = S.tgt_el0[U.tg] + 4LL * r;
          float4* h4 = reinterpret_cast<float4*>(reinterpret_cast<float2*>(it.kH) + ce);
          float4* d4 = reinterpret_cast<float4*>(reinterpret_cast<float2*>(it.kdH) + ce);
          h4[0] = make_float4(hr[0], hi[0], hr[1], hi[1]);
          h4[1] = make_float4(hr[2], hi[2], hr[3], hi[3]);
          d4[0] = make_float4(dr[0], di[0], dr[1], di[1]);
          d4[1] = make_float4(dr[2], di[2], dr[3], di[3]);
        } else {
          store_emb_f4(it.Hemb_p, S.Np, oi + r, oj, hr, hi);
          store_emb_f4(it.dHemb_p, S.Np, oi + r, oj, dr, di);
        }
      }
    } else {
      for (int e = sub; e < nel; e += 4) {
        const int a = e / nj, b = e - a * nj;
        float hr = 0.f, hi = 0.f, dr = 0.f, di = 0.f;
        for (int g = g0; g < g1; ++g) {
          const long long off = S.img_off[g] + e;
          const float sv = S.sf[off], hv = S.h0f[off];
          const float adS = a0 * S.dsf[off] + a1 * S.dsf[dss + off] + a2 * S.dsf[2 * dss + off];
          const float2 ph = S.phase_img[(long long)k * S.n_img + g];  // e^{-i 2 pi k.n} of image g
          const float vr = hv + beta * sv;
          hr += ph.x * vr - ph.y * adS;
          hi += ph.x * adS + ph.y * vr;
          const float wr = dbeta * sv;
          dr += ph.x * wr - ph.y * adS;
          di += ph.x * adS + ph.y * wr;
        }
        if (it.kH) {
          const long long ce = S.tgt_el0[U.tg] + e;
          reinterpret_cast<float2*>(it.kH)[ce] = make_float2(hr, hi);
          reinterpret_cast<float2*>(it.kdH)[ce] = make_float2(dr, di);
        } else {
          store_emb_f(it.Hemb_p, S.Np, oi + a, oj + b, hr, hi);
          store_emb_f(it.dHemb_p, S.Np, oi + a, oj + b, dr, di);
        }
      }
    }
  }
}

void launch_phase_split(const DevSys* sys, DevTraj* trj, const DevItem* items, const int* warp_prefix,
                        int n_traj, int total_units, int max_nk, const int* step, int finish, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (total_units * 4 + threads - 1) / threads;
  launch_pdl(k_phase_split, dim3(blocks + (finish ? n_traj : 0), max_nk), threads, 0, st, sys, trj, items,
             warp_prefix, n_traj, total_units, finish ? blocks : -1, step);
}

// ---------------------------------------------------------------------------
// Setup kernels for one system and one k (warp per target):
//   mode 0: S_k (Eq. 7);  mode 1: H_k at A = 0 = H0_k + (eps_I + eps_J)/2 S_k
// written densely into out (Np x Np, zeros elsewhere set by the caller), and
// the Mulliken partial sum per target of a density set D (all k, weighted).
// ---------------------------------------------------------------------------
__global__ void k_bloch_setup(const DevSys* __restrict__ sysv, int s_idx, int k, int mode,
                              const double* __restrict__ eps, double2* out) {
  const int tg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const DevSys& S = sysv[s_idx];
  if (tg >= S.n_tgt) return;
  const int I = S.tgt_I[tg], J = S.tgt_J[tg];
  const int oi = S.orb_off[I], ni = S.orb_off[I + 1] - oi;
  const int oj = S.orb_off[J], nj = S.orb_off[J + 1] - oj;
  const double beta = mode == 1 ? 0.5 * (eps[I] + eps[J]) : 0.0;
  for (int e = lane; e < ni * nj; e += 32) {
    const int a = e / nj, b = e - a * nj;
    double xr = 0.0, xi = 0.0;
    for (int g = S.tgt_img0[tg]; g < S.tgt_img0[tg + 1]; ++g) {
      const int blk = S.img_blk[g];
      const long long off = S.img_off[g] + e;
      const double v = mode == 1 ? S.h0[off] + beta * S.s[off] : S.s[off];
      const double2 ph = S.phase[(long long)k * S.n_blk + blk];
      xr += ph.x * v;
      xi += ph.y * v;
    }
    out[(long long)(oi + a) * S.Np + (oj + b)] = make_double2(xr, xi);
  }
}

__global__ void k_mulliken_setup(const DevSys* __restrict__ sysv, int s_idx, const double2* __restrict__ D,
                                 double* part) {
  const int tg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const DevSys& S = sysv[s_idx];
  if (tg >= S.n_tgt) return;
  const int I = S.tgt_I[tg], J = S.tgt_J[tg];
  const int oi = S.orb_off[I], ni = S.orb_off[I + 1] - oi;
  const int oj = S.orb_off[J], nj = S.orb_off[J + 1] - oj;
  const long long NN = (long long)S.Np * S.Np;
  double acc = 0.0;
  for (int e = lane; e < ni * nj; e += 32) {
    const int a = e / nj, b = e - a * nj;
    const long long idx = (long long)(oi + a) * S.Np + (oj + b);
    for (int k = 0; k < S.nk; ++k) {
      const double2 d = D[k * NN + idx];
      double l = 0.0;
      for (int g = S.tgt_img0[tg]; g < S.tgt_img0[tg + 1]; ++g) {
        const double2 ph = S.phase[(long long)k * S.n_blk + S.img_blk[g]];
        l += S.s[S.img_off[g] + e] * (d.x * ph.x + d.y * ph.y);
      }
      acc += S.wk[k] * l;
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) part[tg] = acc;
}

void launch_bloch_setup(const DevSys* sys, int s_idx, int n_tgt, int k, int mode, const double* eps,
                        double2* out, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (n_tgt * 32 + threads - 1) / threads;
  k_bloch_setup<<<blocks, threads, 0, st>>>(sys, s_idx, k, mode, eps, out);
}

void launch_mulliken_setup(const DevSys* sys, int s_idx, int n_tgt, const double2* D, double* part,
                           cudaStream_t st) {
  const int threads = 256;
  const int blocks = (n_tgt * 32 + threads - 1) / threads;
  k_mulliken_setup<<<blocks, threads, 0, st>>>(sys, s_idx, D, part);
}

}  // namespace vgtb
