// Internal data structures and kernel launchers of libvgtb.
//
// Layout in HBM (per system s with N orbitals, Np = N rounded up to 128):
//   * real-space blocks: h0, s, ds values as given (n_I x n_J row-major
//     blocks, concatenated), plus targets = distinct (I, J) pairs sorted by I
//     with the list of their images (blocks with different L); the Bloch
//     phase e^{-i 2 pi k.n} of every (k, block) is tabulated once.
//   * per (s, k): S_k^-1, D_k(0) and (delta forms) R0 as Np x Np complex128
//     row-major; for the split-precision form also their BF16 hi/lo pieces in
//     "planar" rows [Re(row) | Im(row)] (Np x 2Np per piece).
//   * per item = (trajectory, k): the two leapfrog levels as Np x Np
//     complex128, plus the working operands of the commutator products.
// Padding rows / columns (N <= i < Np) hold zeros and stay zero.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace vgtb {

// Programmatic dependent launch: the step kernels are launched with
// programmatic stream serialization, so a kernel's CTAs may be scheduled while
// its predecessor drains.  Every CTA calls pdl_wait() before its first access
// to memory that an earlier kernel writes (and before any early return, so
// that a grid never completes ahead of its predecessor); pdl_wait() returns
// once the preceding grid has completed and its writes are visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

constexpr double kLight = 137.035999084;

// status bits written by kernels
enum : int {
  ST_NONFINITE = 1,      // non-finite J / E / charges
  ST_DRIFT = 2,          // electron count drifted
  ST_TIMEOUT = 4,        // a bounded device wait gave up
  ST_BADSHAPE = 8,       // a kernel saw an impossible shape
  ST_CN_NOCONV = 16,     // Crank-Nicolson fixed point still moving after the last sweep
};

// ---------------------------------------------------------------------------
// IEEE-754 float <-> double conversions done with integer bit operations.
// GB300 runs FP64 instructions, conversions included, at a small fraction of
// the integer rate, so the split-form kernels convert with these and keep the
// FP64 pipe for the arithmetic that needs it.
//  * f2d_bits: exact for every normal float, infinities and NaNs (payload
//    kept); float subnormals (below 2^-126 = 1.2e-38) become signed zero.
//  * d2f_bits: round to nearest, ties to even, like __double2float_rn, for
//    every input of magnitude >= 2^-126; an input below 2^-126 becomes signed
//    zero (no float subnormals), magnitudes that round above the float range
//    become +-infinity, and a NaN becomes a quiet NaN of the same sign.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t sign = u & 0x80000000u;
  const uint32_t ee = (e == 255u) ? 2047u : e + 896u;  // exponent bias 1023 - 127
  const uint32_t hi = (e == 0u) ? sign : (sign | (ee << 20) | ((u >> 3) & 0xfffffu));
  const uint32_t lo = (e == 0u) ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_bits(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const uint32_t mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu;
  uint32_t f = sign | ((uint32_t)e << 23) | mant;
  f += (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ? 1u : 0u;
  f = (e <= 0) ? sign : f;
  f = (e >= 255) ? (sign | 0x7f800000u) : f;
  const uint32_t ah = hi & 0x7fffffffu;
  f = (ah > 0x7ff00000u || (ah == 0x7ff00000u && lo != 0u)) ? (sign | 0x7fc00000u) : f;
  return __uint_as_float(f);
}

constexpr int kSccRowsPerCta = 4;  // rows of gamma per CTA of k_scc_eps (one warp each)

struct DevSys {
  int N, Np, nat, nk, n_tgt, n_blk;
  int scc_frozen;          // 1: H keeps the shift eps0 of D(0) (VGTB_SCC_FROZEN)
  double omega, nel, dt;
  double inv_omega;        // 1 / omega (an FP64 division is a long sequence on GB300)
  const int* orb_off;      // [nat+1]
  const double* z;         // [nat]
  const double* gamma;     // [nat*nat]
  const int* tgt_I;        // [n_tgt]
  const int* tgt_J;        // [n_tgt]
  const int* tgt_img0;     // [n_tgt+1] range into img_blk
  const int* img_blk;      // [n_img] block index of each image
  const long long* img_off;// [n_img] value offset of each image's block
  const long long* blk_off;// [n_blk] offset of each block's values
  const double* h0;        // values
  const double* s;
  const double* ds;        // [3][ds_stride]
  long long ds_stride;
  const double2* phase;    // [nk][n_blk] = e^{-i 2 pi k.n}
  const double* wk;        // [nk]
  const int* atom_tgt0;    // [nat+1] targets of row atom I are atom_tgt0[I]..atom_tgt0[I+1]-1
  int n_el;                // elements over all targets (sum of n_I n_J)
  const int* tgt_el0;      // [n_tgt+1] first element of each target
  const int* tgt_vec;      // [n_tgt] 1: 4-column blocks with 16-byte aligned values (vector phase build)
  const int* el_off;       // [n_el] offset (row * Np + column) of each nonzero in an Np x Np matrix
  const int* el_atom0;     // [nat+1] first nonzero of each row atom (= tgt_el0[atom_tgt0[I]])
  double2* kS;             // [nk][n_el] Bloch-summed S_k at the target elements (Eq. 7)
  double2* kP;             // [3][nk][n_el] momentum P_k = sum e^{-ik.L} i dS/dR_J (Eq. 12)
  double2* kH0;            // [nk][n_el] H0_k
  double* obs0;            // [n_tgt][5] delta forms: the D0 part of the k_obs sums
  double* obs0a;           // [nat][5] split form: obs0 summed over the targets of each row atom
  double2* Sinv;           // [nk][Np*Np]
  double2* D0;             // [nk][Np*Np]
  double2* R0;             // [nk][Np*Np] (delta forms), else null
  double* dq0;             // [nat] charges of D(0)
  double* eps0;            // [nat] shift of D(0)
  __nv_bfloat16* Sinv_p;   // [nk][2][Np][2Np] split pieces (split form)
  __nv_bfloat16* D0_p;     // [nk][2][Np][2Np]
  // split form only: FP32 copies for the phase build and the leapfrog derivative
  const float* h0f;        // values as float
  const float* sf;
  const float* dsf;        // [3][ds_stride]
  const float2* phasef;    // [nk][n_blk]
  float* R0f;              // [nk][Np][2Np] planar
  float2* D0f;             // [nk][Np][Np] FP32 copy of D0 (split form, block-sparse first product)
  // split-form phase build: per target {I, J, first image, end image} and
  // {o_I, o_J, n_I | vec << 16, n_J}; the FP32 phase of every (k, image)
  const int4* tgt_p0;      // [n_tgt]
  const int4* tgt_p1;      // [n_tgt]
  const float2* phase_img; // [nk][n_img]
  int n_img;
};

struct DevTraj {
  int sys;
  int item0;               // item index of (this trajectory, k = 0)
  int sys_traj;            // index among the trajectories of its system
  int n_times;             // length of the A table
  const double* A;         // [n_times][3]
  double* J;               // [n_times][3]
  double* E;               // [n_times]
  double* q;               // [(n_times-1)/stride+1][nat]
  double* dq;              // [nat] current dq
  double* eps;             // [nat] current eps
  double* eps_lv;          // [2][nat] eps of the two latest levels by parity (Crank-Nicolson), or null
  // split form: FP32 operands of the phase build, written by k_scc_eps at level n
  float* epsf;             // [nat] eps_I
  float* depsf;            // [nat] eps_I - eps0_I
  float* af;               // [3] A(t_n) / c
  double* part;            // [n_tgt][5] per-target partial sums
  double* cpart;           // [ceil(nat / kSccRowsPerCta)][6] per-CTA partial sums of k_scc_eps
  double* apart;           // [nat][4] per-atom shares of T_x, T_y, T_z and the band energy
  int* ticket;             // [1] CTA arrival counter of k_scc (reset by the last CTA)
  int* status;
};

struct DevItem {
  int sys, traj, k;
  double2* D[2];           // leapfrog levels (delta forms: dD = D - D0)
  double2* H;              // FP64 H_k(t) (delta form: H without the |A|^2 term)
  double2* dH;             // FP64 delta form: H_k(t) - H_ref
  double2* W;              // FP64 first product
  double2* X;              // FP64 second product
  __nv_bfloat16* dD_p;     // split form: [2][Np][2Np] pieces of dD
  __nv_bfloat16* Hemb_p;   // split form: [2][2Np][2Np] embedded H
  __nv_bfloat16* dHemb_p;  // split form: [2][2Np][2Np] embedded dH
  __nv_bfloat16* Wemb_p;   // split form: [2][2Np][2Np] embedded W
  float* Xf;               // split form: [Np][2Np] planar X
  double2* Cd;             // Crank-Nicolson: occupied states as rows, C^dagger [nocc][Np]
  double2* Y[2];           // Crank-Nicolson: fixed-point iterates [nocc][Np]
  // block-sparse first product: H_k(t) and dH_k(t) at the target elements only
  // ([n_el], complex; double2 on the FP64 path, float2 in the split form), and in
  // the split form the FP32 copy of the current dD level ([Np][Np] float2)
  void* kH;
  void* kdH;
  float2* dDf;
};

// ---------------------------------------------------------------------------
// Block-sparse first product (k_bsr.cu): W = sum_seg A_seg R_seg^dagger with R
// on the target pattern (every atom 4 orbitals), A dense and Hermitian.
// ---------------------------------------------------------------------------
constexpr int kBsrThreads = 128;   // output rows (columns of A) per CTA
constexpr int kBsrGroupF32 = 8;    // atoms per group (output columns / 4), split form
constexpr int kBsrGroupF64 = 4;    // atoms per group, FP64 path

struct BsrSys {
  int Np, nat, n_grp;
  const int* grp_t0;       // [n_grp+1] first target of each group (targets sorted by row atom)
  const int* grp_e0;       // [n_grp+1] first union entry of each group
  const int* ent_K;        // [n_ent] column atom K of each entry
  const short* ent_slot;   // [n_ent][G] target index of (J_j, K) minus grp_t0, or -1
  const short* tgt_ent;    // [n_tgt] 1024 x (row atom - first atom of its group) + position of the
                           // column atom K in the group's union list
};

struct BsrItem {
  int sys, nseg;
  const void* A[2];        // [Np][Np] complex (double2 / float2), Hermitian
  long long a_par;         // segment 0 reads A[0] + ((*step) & 1) * a_par (leapfrog level)
  const void* R[2];        // [n_el] complex target blocks (4 x 4 row-major each)
  void* W;                 // FP64: [Np][Np] double2; split: embedded BF16 pieces [2][2Np][2Np]
};
int bsr_group(int fp64);
size_t bsr_smem_bytes(int fp64, int max_grp_targets);
int bsr_configure(int fp64, int max_grp_targets);
int bsr_units(int fp64, int n_grp, int Np);  // CTAs per item

// Crank-Nicolson: D_k = 2 C C^dagger at the nonzero pattern of H_k only (what
// the charge, current and energy sums read), from C^dagger [nocc][Np] of every
// item; uses the FP64 group tables of the block-sparse product.  D entries off
// the pattern are left as they are.
struct CnDensItem {
  int sys;
  const double2* Cd;       // [nocc][Np] occupied states as rows (C^dagger)
  double2* D;              // [Np][Np]
  int nocc;
};
int cn_density_configure(int max_ent);
int cn_density_max_targets();  // most targets per atom group the kernel takes
void launch_cn_density_pattern(const CnDensItem* items, const BsrSys* sys, int n_items, int max_groups, int max_ent,
                               cudaStream_t st);
// FP64: grid (max_units, n_items); split form: persistent CTAs taking units
// 0..total_units-1 (item it owns item_u0[it] .. item_u0[it+1]-1) from the
// counter pair ctr[2] (zero before the first launch; reset by each launch)
void launch_bsr(const BsrItem* items, const BsrSys* sys, int n_items, int max_units, int total_units,
                const int* item_u0, int* ctr, int fp64, int max_grp_targets, const int* step, cudaStream_t st);

// Crank-Nicolson convergence check of one item: max |Y[a] - Y[b]| over nocc x N
struct CnCheckItem {
  const double2* a;
  const double2* b;
  int rows, cols, ld, traj;
};
void launch_cn_check(const CnCheckItem* items, int n_items, int max_elems, const DevTraj* trj, double tol,
                     cudaStream_t st);
// dst[r][c] = conj(src[c][r]) for r < rows, c < cols (dst row stride ldd, src row stride lds)
void launch_conj_transpose(const double2* src, int lds, double2* dst, int ldd, int rows, int cols, cudaStream_t st);

// What the phase-build kernel writes.
enum PhaseMode : int {
  PH_FP64_PLAIN = 0,   // H = H0 + (alpha + (eps_I+eps_J)/2) S + (i/c) A.dS  -> item.H
  PH_FP64_DELTA = 1,   // H without alpha -> item.H ; dH = ((deps_I+deps_J)/2) S + (i/c) A.dS -> item.dH
  PH_FP64_CN = 2,      // H at t_{n+1/2} without alpha: midpoint A, extrapolated eps -> item.H
};

// Launchers (all enqueue on `st`)
// delta: 0 = D itself (FP64), 1 = dD with the D0 part from obs0 (FP64)
void launch_obs(const DevSys* sys, const DevTraj* trj, const DevItem* items, const int* warp_prefix,
                int n_traj, int total_warps, const int* step, int delta, int fixed_step, cudaStream_t st);
// atoms_done = 1: the per-atom sums were made by k_obs_atoms_split (split form);
// finish = 0: J, E and the checks of the level are left to launch_phase_split's
// finisher CTAs (the split form's step), else the last CTA of k_scc_eps does them
void launch_scc(const DevSys* sys, DevTraj* trj, int n_traj, const int* step, int stride,
                int fixed_step, int record, int max_nat, int atoms_done, cudaStream_t st, int finish = 1);
void launch_obs_atoms_split(const DevSys* sys, DevTraj* trj, const DevItem* items, int n_traj, int max_nat,
                            const int* step, int stride, int fixed_step, int record, cudaStream_t st);
// grid rows = max_nk: row y builds k-points y, y + max_nk, ... of every target;
// finish = 1 adds one CTA per trajectory that finishes the level's J, E and
// checks from k_scc_eps's partials (launched with finish = 0)
void launch_phase_split(const DevSys* sys, DevTraj* trj, const DevItem* items, const int* warp_prefix,
                        int n_traj, int total_units, int max_nk, const int* step, int finish, cudaStream_t st);
void launch_to_planar_f32(const double2* src, float* dst, int Np, cudaStream_t st);
void launch_phase(const DevSys* sys, const DevTraj* trj, const DevItem* items, const int* warp_prefix,
                  int n_traj, int total_warps, const int* step, int mode, int fixed_step, cudaStream_t st);
int scc_configure(int max_nat);
void launch_kblocks(const DevSys* sys, int s_idx, int n_tgt, int k, cudaStream_t st);
void launch_obs0(const DevSys* sys, int s_idx, int n_tgt, int nat, int split, cudaStream_t st);
void launch_bloch_setup(const DevSys* sys, int s_idx, int n_tgt, int k, int mode, const double* eps,
                        double2* out, cudaStream_t st);
void launch_mulliken_setup(const DevSys* sys, int s_idx, int n_tgt, const double2* D, double* part,
                           cudaStream_t st);

struct GemmF64Item {
  const double2* A[2];
  const double2* R[2];
  long long a_par[2];      // A += ((*step) & 1) * a_par  (leapfrog level selection)
  double2* C;
  int K[2];
  int lda[2], ldr[2];
  int nseg, M, N, ldc;
  int conj_t;              // bit 0: A(m, k) = conj(A[k * lda + m]); bit 1: the same for R
  int epi;                 // 0: C = acc;  1: C = coef * acc (+ base when base != null)
  double2 coef;
  const double2* base;     // may alias C (element-wise read-before-write by one thread)
  int ldb;
};
void launch_gemm_f64(const GemmF64Item* items, int n_items, int max_m, int max_n, const int* step,
                     cudaStream_t st);

struct LeapItem {
  const void* X;           // FP64 interleaved (double2) or FP32 planar
  const double2* R0;       // optional (FP64 path)
  const float* R0f;        // optional (split path, FP32 planar)
  double2* D[2];
  __nv_bfloat16* pieces;   // optional [2][Np][2Np]
  float2* f32;             // optional [Np][Np]: FP32 copy of the new level (split form)
  int Np;
  int mode;                // 0 = leapfrog, 1 = write the derivative only into out
  double2* out;            // mode 1 target
};
void launch_leap(const LeapItem* items, int n_items, int Np_max, int x_f32, const int* step, double dt,
                 int* counter, int* step_rw, cudaStream_t st);
void launch_leap_split(const LeapItem* items, int n_items, int Np_max, const int* step, double dt, int* counter,
                       int* step_rw, cudaStream_t st);

// helpers
void launch_fill_hermitian_lower(double2* a, int n, int ld, cudaStream_t st);
void launch_vt_from_evecs(const double2* evec, double2* vt, int n, int nocc, int ld, cudaStream_t st);
void launch_scale(double2* a, long long n, double s, cudaStream_t st);
void launch_split_planar(const double2* src, __nv_bfloat16* dst, int N, int Np, cudaStream_t st);
void launch_increment(int* step, cudaStream_t st);
void launch_hermitize(double2* a, int n, int ld, cudaStream_t st);
void launch_split_embedded(const double2* src, __nv_bfloat16* dst, int Np, cudaStream_t st);
void launch_to_f32(const double2* src, float2* dst, long long n, cudaStream_t st);

// post-propagation reductions (k_spectrum.cu)
void launch_conductivity(const double* J, int n0, int n1, double dt, double e0, double tau0, const double* omega,
                         int n_omega, double* sigma, double* eps, cudaStream_t st);
void launch_group_charge(const double* q, int nat, const int* group, int n_groups, int n_levels, double* out,
                         cudaStream_t st);

// tcgen05 split-precision complex GEMM (k_gemm_tc.cu)
struct TcGemmPlan;   // opaque, built on the host
int tc_gemm_supported();

}  // namespace vgtb
