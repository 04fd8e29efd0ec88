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

constexpr double kLight = 137.035999084;

// status bits written by kernels
enum : int {
  ST_NONFINITE = 1,      // non-finite J / E / charges
  ST_DRIFT = 2,          // electron count drifted
  ST_TIMEOUT = 4,        // a bounded device wait gave up
  ST_BADSHAPE = 8,       // a kernel saw an impossible shape
};

struct DevSys {
  int N, Np, nat, nk, n_tgt, n_blk;
  double omega, nel, dt;
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
  double2* kS;             // [nk][n_el] Bloch-summed S_k at the target elements (Eq. 7)
  double2* kP;             // [3][nk][n_el] momentum P_k = sum e^{-ik.L} i dS/dR_J (Eq. 12)
  double2* kH0;            // [nk][n_el] H0_k
  double* obs0;            // [n_tgt][5] delta forms: the D0 part of the k_obs sums
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
  double* part;            // [n_tgt][5] per-target partial sums
  double* erow;            // [nat] dq_I eps_I (energy of the SCC term, per row)
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
};

// What the phase-build kernel writes.
enum PhaseMode : int {
  PH_FP64_PLAIN = 0,   // H = H0 + (alpha + (eps_I+eps_J)/2) S + (i/c) A.dS  -> item.H
  PH_FP64_DELTA = 1,   // H without alpha -> item.H ; dH = ((deps_I+deps_J)/2) S + (i/c) A.dS -> item.dH
};

// Launchers (all enqueue on `st`)
void launch_obs(const DevSys* sys, const DevTraj* trj, const DevItem* items, const int* warp_prefix,
                int n_traj, int total_warps, const int* step, int delta, int fixed_step, cudaStream_t st);
void launch_scc(const DevSys* sys, DevTraj* trj, int n_traj, const int* step, int stride,
                int fixed_step, int record, int max_nat, cudaStream_t st);
void launch_phase_split(const DevSys* sys, const DevTraj* trj, const DevItem* items, const int* warp_prefix,
                        int n_traj, int total_units, const int* step, cudaStream_t st);
void launch_to_planar_f32(const double2* src, float* dst, int Np, cudaStream_t st);
void launch_phase(const DevSys* sys, const DevTraj* trj, const DevItem* items, const int* warp_prefix,
                  int n_traj, int total_warps, const int* step, int mode, int fixed_step, cudaStream_t st);
int scc_configure(int max_nat);
void launch_kblocks(const DevSys* sys, int s_idx, int n_tgt, int k, cudaStream_t st);
void launch_obs0(const DevSys* sys, int s_idx, int n_tgt, cudaStream_t st);
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
};
void launch_gemm_f64(const GemmF64Item* items, int n_items, int max_m, int max_n, const int* step,
                     cudaStream_t st);

struct LeapItem {
  const void* X;           // FP64 interleaved (double2) or FP32 planar
  const double2* R0;       // optional (FP64 path)
  const float* R0f;        // optional (split path, FP32 planar)
  double2* D[2];
  __nv_bfloat16* pieces;   // optional [2][Np][2Np]
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

// post-propagation reductions (k_spectrum.cu)
void launch_conductivity(const double* J, int n0, int n1, double dt, double e0, double tau0, const double* omega,
                         int n_omega, double* sigma, double* eps, cudaStream_t st);
void launch_group_charge(const double* q, int nat, const int* group, int n_groups, int n_levels, double* out,
                         cudaStream_t st);

// tcgen05 split-precision complex GEMM (k_gemm_tc.cu)
struct TcGemmPlan;   // opaque, built on the host
int tc_gemm_supported();

}  // namespace vgtb
