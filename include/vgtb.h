/*
 * vgtb.h - C-ABI of the GB300 velocity-gauge real-time TDDFTB propagator.
 *
 * The library advances k-resolved density matrices D_k(t) of a periodic
 * system in a non-orthogonal tight-binding basis under a time-dependent
 * vector potential A(t) (Xu et al., "Velocity-gauge real-time TDDFTB for
 * large-scale condensed matter systems", Sec. 2):
 *
 *   i dD_k/dt = S_k^-1 H_k D_k - D_k H_k S_k^-1                     (Eq. 6)
 *   S_k = sum_L e^{-ik.L} S(L),  H_k = sum_L e^{-ik.L} H(L)         (Eqs. 7, 8)
 *   H(L) = H0(L) + 1/2 S(L)(eps_I + eps_J) + (1/c) A.P(L)
 *          + |A|^2/(2c^2) S(L),  eps = gamma dq,  P(L) = i dS(L)/dR_J (Eqs. 9-12)
 *   q_I = sum_k w_k sum_{mu in I} Re[D_k S_k]_{mu mu}, dq = q - Z  (Eq. 10)
 *   D_k(t+dt) = D_k(t-dt) + 2 dt dD_k/dt(t)                         (Eq. 13)
 *   J(t) = -(1/Omega) sum_k w_k Re Tr[D_k (P_k + (A/c) S_k)]         (Eq. 14)
 *
 * Readings of points the paper leaves open: the leapfrog starts with one
 * forward-Euler step; D_k carries occupations f in {0, 2} so Tr(D_k S_k) =
 * N_el; the SCC shift at t_n comes from D(t_n); the energy is
 * E = sum_k w_k Re Tr[D_k(H0_k + (A/c).P_k + |A|^2/(2c^2) S_k)] + 1/2 dq.gamma.dq.
 *
 * Conventions for every call:
 *  - Return value 0 (VGTB_OK) on success, a negative VGTB_E_* code otherwise;
 *    no C++ exception crosses the ABI.  vgtb_last_error() gives a message.
 *  - All pointers in vgtb_system and all input/output arrays of the calls are
 *    HOST pointers, row-major, owned by the caller.  Inputs are copied before
 *    the call returns; outputs are caller-allocated.  Complex matrices are
 *    N x N row-major with interleaved (re, im) doubles.
 *  - A context owns all device memory it allocates and is used from one host
 *    thread at a time.  Work is enqueued on the context's CUDA stream
 *    (vgtb_options.cuda_stream, or a stream the context creates); every call
 *    synchronises that stream before it returns.
 *  - Units: Hartree atomic units; c = 137.035999084.
 */
#ifndef VGTB_H
#define VGTB_H

#ifdef __cplusplus
extern "C" {
#endif

#define VGTB_OK             0
#define VGTB_E_INVALID     -1  /* bad argument: shape, NaN/Inf input, asymmetric gamma,
                                  missing mirror block, index out of range */
#define VGTB_E_NOT_PD      -2  /* S_k is not positive definite */
#define VGTB_E_NO_GAP      -3  /* ground state: no gap at N_el/2 at some k */
#define VGTB_E_CUDA        -4  /* a CUDA / cuSOLVER call failed */
#define VGTB_E_NOMEM       -5  /* device allocation failed */
#define VGTB_E_STATE       -6  /* call out of order (no density, no field, field too short) */
#define VGTB_E_UNSTABLE    -7  /* non-finite J/E/charges or electron-count drift */
#define VGTB_E_TIMEOUT     -8  /* a bounded device wait expired */
#define VGTB_E_NO_CONVERGE -9  /* SCC ground state did not converge */
#define VGTB_E_UNSUPPORTED -10 /* option not available for these shapes */

/* precision forms of the commutator products */
#define VGTB_FP64          0   /* complex FP64 everywhere (Eq. 6 evaluated directly) */
#define VGTB_SPLIT_BF16X3  1   /* delta form, tcgen05 BF16 hi/lo 3-product GEMMs, FP32 accumulate */

#define VGTB_INIT_GROUND   0   /* create() computes the SCC ground state D_k(0) */
#define VGTB_INIT_USER     1   /* caller sets D_k(0) with vgtb_set_density() (leapfrog) or the
                                  occupied states with vgtb_set_coefficients() (Crank-Nicolson) */

#define VGTB_LEAPFROG       0  /* density matrices by Eq. 6 and the leapfrog of Eq. 13 */
#define VGTB_CRANK_NICOLSON 1  /* occupied coefficient vectors by Eq. 5 with the unitary
                                  Crank-Nicolson scheme named in Sec. 2:
                                  (S + i dt/2 H(t+dt/2)) C(t+dt) = (S - i dt/2 H(t+dt/2)) C(t),
                                  H(t+dt/2) from A((t_n + t_{n+1})/2) and the SCC shift
                                  extrapolated as (3 eps_n - eps_{n-1})/2, without the |A|^2 S
                                  term (an overall phase, remark after Eq. 3); the linear
                                  system is solved by cn_iter fixed-point sweeps
                                  Y <- C - i dt/2 S^-1 H Y, C(t+dt) = 2Y - C.  FP64 only. */

typedef struct vgtb_ctx vgtb_ctx;  /* opaque; owned by the library */

/* One periodic system (Sec. 2).  Every pointer is a host pointer, read during
 * vgtb_create*(); the caller keeps ownership. */
typedef struct {
  double lattice[9];        /* rows a1, a2, a3 in bohr; Omega = |det| (Eq. 14) */
  int n_atoms;
  const double* pos;        /* [n_atoms][3] cartesian bohr (R_I of Eq. 4) */
  const int* orb_offset;    /* [n_atoms+1] orbital ranges of mu = (I,l,m); N = orb_offset[n_atoms] */
  const double* z_ref;      /* [n_atoms] Z_I of dq = q - Z (Eq. 10) */
  int n_blocks;
  const int* blk_ijl;       /* [n_blocks][5]: I, J, n1, n2, n3 with L = n1 a1 + n2 a2 + n3 a3.
                               Block (I,J,L) = <phi_mu(r-R_I-L)| . |phi_nu(r-R_J)> (Eq. 7);
                               the mirror block (J,I,-L) must be present. */
  const double* h0;         /* block values, each n_I x n_J row-major, concatenated (Eq. 9 H0) */
  const double* s;          /* same layout: overlap S(L) (Eq. 7) */
  const double* ds;         /* [3][total]: dS(L)/dR_J per cartesian component (Eq. 12) */
  const double* gamma;      /* [n_atoms][n_atoms] symmetric (Eqs. 10, 11) */
  int n_k;
  const double* kpt;        /* [n_k][3] reduced coordinates: k.L = 2 pi k_red.n */
  const double* wk;         /* [n_k] weights summing to 1 (1/N_k of Eq. 10) */
  double n_electrons;       /* N_el; N_el/2 states per k are doubly occupied */
  double dt;                /* time step in a.u. (Eq. 13) */
} vgtb_system;

typedef struct {
  int precision;            /* VGTB_FP64 or VGTB_SPLIT_BF16X3 */
  int delta_form;           /* FP64 only: 1 = propagate dD = D - D(0) with the exact delta form
                               dD/dt = R0 - i[S^-1(H dD + dH D0) - h.c.] (same result as Eq. 6) */
  int init;                 /* VGTB_INIT_GROUND or VGTB_INIT_USER */
  void* cuda_stream;        /* cudaStream_t to enqueue on; NULL = the context creates one */
  long long timeout_ns;     /* limit of every device-side wait (0 = 2e9 ns) */
  int obs_stride;           /* charges q(t_n) are stored every obs_stride steps (0 = 1) */
  int graph_steps;          /* steps captured per CUDA graph replay (0 = 32; 1 = no graph) */
  int autotune;             /* 1 = time the GEMM tile candidates at create and keep the fastest */
  double scc_tol;           /* ground state: stop when max|dq_out - dq_in| < scc_tol (0 = 1e-11) */
  int scc_max_iter;         /* ground state iteration limit (0 = 200) */
  int integrator;           /* VGTB_LEAPFROG (default) or VGTB_CRANK_NICOLSON */
  int cn_iter;              /* Crank-Nicolson fixed-point sweeps per step, >= 2 (0 = 12); the
                               sweeps contract by dt/2 max|eig(S^-1 H)| each */
  double cn_tol;            /* Crank-Nicolson: propagate() fails with E_UNSTABLE when the last
                               two iterates differ by more than cn_tol in any entry (0 = 1e-10) */
  int tile_variant[2];      /* split form: tile variant of product 1 / product 2 (see
                               vgtb_tile_config; -1 = variant 0, or the autotuner's choice) */
  int product1;             /* form of the first product W = D H of Eq. 6 (VGTB_P1_*):
                               AUTO (0, default): the FP64 path runs it block-sparse (below), and
                               so does the Crank-Nicolson integrator its product M = S^-1 H; the
                               split form runs the tcgen05 GEMM and skips the 64-wide k-panels in
                               which a tile's rows of H_k and dH_k are zero;
                               DENSE: a dense GEMM over all of H_k (8 N^3 flops; FP64 DFMA or
                               tcgen05 BF16x3, no panel skipped); BLOCKS: block-sparse over the
                               nonzero atom blocks of H_k on the CUDA cores (8 nnz(H) N flops;
                               FP64, or FP32 in the split form), which needs every atom to carry
                               4 orbitals (the FP64 AUTO falls back to DENSE otherwise, BLOCKS
                               fails with E_UNSUPPORTED) */
  int scc;                  /* VGTB_SCC_ON (0, default): the shift eps = gamma dq of Eq. 10 follows
                               the charges at every step; VGTB_SCC_FROZEN: H keeps the shift of
                               D_k(0) at every step (non-self-consistent propagation); charges,
                               current and energy are still evaluated from D_k(t_n) */
  int chain;                /* split form, both products on the tcgen05 kernel: VGTB_CHAIN_AUTO (0,
                               default) runs them as one launch, with a product-2 tile starting
                               as soon as the rows of W it reads are stored (Eq. 6: X = S^-1 W^dagger
                               needs W only), when that is faster at create than the two fastest
                               separate launches (with autotune, the one launch runs on the
                               fastest chainable variants, which may differ from the separate
                               picks); VGTB_CHAIN_OFF: two launches; VGTB_CHAIN_ON: one launch
                               whenever the tile variants allow it (2-SM pairs, classic
                               schedules, 64-column stages) */
} vgtb_options;

#define VGTB_P1_AUTO     0
#define VGTB_P1_DENSE    1
#define VGTB_P1_BLOCKS   2
#define VGTB_SCC_ON      0
#define VGTB_SCC_FROZEN  1
#define VGTB_CHAIN_AUTO  0
#define VGTB_CHAIN_OFF   1
#define VGTB_CHAIN_ON    2

/* Fill *opt with the defaults above (precision FP64, ground-state init, leapfrog). */
void vgtb_default_options(vgtb_options* opt);

/* Create a context for one system and one trajectory (Sec. 2 problem statement).
 * Builds S_k (Eq. 7) and S_k^-1 (Cholesky, FP64), and with VGTB_INIT_GROUND the
 * SCC ground state (Sec. 3.1).  Errors: E_INVALID, E_NOT_PD, E_NO_GAP,
 * E_NO_CONVERGE, E_NOMEM, E_CUDA.  On error *out is NULL. */
int vgtb_create(vgtb_ctx** out, const vgtb_system* sys, const vgtb_options* opt);

/* Batched form: n_sys systems (orbital counts may differ) and n_traj
 * trajectories; trajectory t propagates system traj_sys[t] under its own A(t)
 * table.  All k-points of all trajectories advance together in each step. */
int vgtb_create_batch(vgtb_ctx** out, int n_sys, const vgtb_system* sys,
                      int n_traj, const int* traj_sys, const vgtb_options* opt);

/* Set D_k(0) of system `sys_index` at k-point k (N x N complex, interleaved,
 * Hermitian; the library keeps its exact Hermitian part (D + D^dagger)/2 so
 * that the propagation preserves Hermiticity bit for bit).  Once every k of
 * the system is set, every trajectory of that system restarts from step 0.
 * Errors: E_INVALID (index, non-finite entries). */
int vgtb_set_density(vgtb_ctx* ctx, int sys_index, int k, const double* d0);

/* Crank-Nicolson integrator: set the occupied states C_k(0) of system
 * `sys_index` at k-point k.  c: host array [N][n_occ] complex interleaved,
 * column n = state n (coefficients of Eq. 4), each occupied twice; n_occ must
 * be N_el/2.  D_k(0) = 2 C C^dagger is formed on the device.  Once every k of
 * the system is set, every trajectory of that system restarts from step 0.
 * Errors: E_INVALID (not a Crank-Nicolson context, index, n_occ, non-finite). */
int vgtb_set_coefficients(vgtb_ctx* ctx, int sys_index, int k, int n_occ, const double* c);

/* Crank-Nicolson integrator: copy C_k(t_n) of trajectory `traj` into c_out
 * ([N][n_occ] complex interleaved, caller-owned).  Errors: E_INVALID. */
int vgtb_get_coefficients(vgtb_ctx* ctx, int traj, int k, double* c_out);

/* Set the vector potential of trajectory `traj`: A[n][3] = A(t_n), n = 0 ..
 * n_times-1 (Eq. 3; a delta kick is A(t_n) = A0 for all n).  Restarts the
 * trajectory clock at step 0.  Errors: E_INVALID. */
int vgtb_set_field(vgtb_ctx* ctx, int traj, int n_times, const double* A);

/* Advance every trajectory by nsteps steps of the context's integrator
 * (leapfrog: Eqs. 6, 10, 13, 14; Crank-Nicolson: Eq. 5 with the same
 * observables from D_k = 2 C C^dagger).
 * Observables of every visited time level are stored on the device.
 * Errors: E_STATE (no density / field, or the field table ends before step
 * n+nsteps), E_UNSTABLE, E_TIMEOUT, E_CUDA. */
int vgtb_propagate(vgtb_ctx* ctx, int nsteps);

/* Number of completed steps n (the current time level is t_n = n dt). */
int vgtb_steps_done(const vgtb_ctx* ctx);

/* Copy the observables of trajectory `traj` for levels 0..n: J[(n+1)][3],
 * E[n+1], and (if q != NULL) q[(n/obs_stride)+1][n_atoms].  Levels are the
 * ones visited so far; J/E of level n are computed when propagate() reaches
 * it (level 0 after the first call, or after vgtb_propagate(ctx, 0)). */
int vgtb_observables(vgtb_ctx* ctx, int traj, double* J, double* E, double* q);

/* Copy D_k(t_n) of trajectory `traj` (N x N complex interleaved). */
int vgtb_get_density(vgtb_ctx* ctx, int traj, int k, double* d_out);

/* Copy D_k(0) of system `sys_index`: the SCC ground state (VGTB_INIT_GROUND)
 * or the Hermitian part of the density given to vgtb_set_density().
 * Errors: E_INVALID (index), E_STATE (no density yet). */
int vgtb_get_initial_density(vgtb_ctx* ctx, int sys_index, int k, double* d_out);

/* Conductivity and dielectric function from the current of a kick (Eqs. 15,
 * 16) of trajectory `traj`, over its stored levels n0..n1 (0 <= n0 < n1 <=
 * steps done):  sigma_i(w) = (1/e0) int_0^T e^{iwt} J_i(t) exp(-t/tau0) dt with
 * t = (n - n0) dt (trapezoid rule), eps_i(w) = 1 + 4 pi i sigma_i(w) / w.
 * e0 is the kick strength, E(t) = e0 delta(t) along the kick direction (a kick
 * A(t) = A0 for t >= 0 has e0 = -A0/c, Eq. 3); tau0 = 200 a.u. in the paper.
 * omega: [n_omega] host array of frequencies > 0.  sigma, eps: caller-owned
 * host arrays [n_omega][3] complex (interleaved doubles), component i = x,y,z.
 * Errors: E_INVALID, E_STATE (levels not yet propagated). */
int vgtb_spectrum(vgtb_ctx* ctx, int traj, int n0, int n1, double e0, double tau0, int n_omega,
                  const double* omega, double* sigma, double* eps);

/* Charge transfer between atom groups (the per-class Mulliken analysis of
 * Sec. 3.3): dQ_g(t_n) = sum_{I in g} (Q_I(t_n) - Q_I(t_0)) with atomic charge
 * Q_I = -(q_I - Z_I), for every stored charge level (every obs_stride steps up
 * to the current step).  group: [n_atoms] host array, group index of each atom
 * in 0..n_groups-1 or negative for none.  out: caller-owned host array
 * [n_levels][n_groups], n_levels = steps_done / obs_stride + 1.
 * Errors: E_INVALID, E_STATE (no field set). */
int vgtb_group_charges(vgtb_ctx* ctx, int traj, int n_groups, const int* group, double* out);

/* Checkpoint: the state is D_k(t_n), D_k(t_{n-1}) of every trajectory and k,
 * plus n (Crank-Nicolson: C_k(t_n) and the SCC shifts of levels n, n-1).
 * vgtb_state_size() gives the byte size of the host buffer. */
long long vgtb_state_size(const vgtb_ctx* ctx);
int vgtb_get_state(vgtb_ctx* ctx, void* buf, long long bytes);
int vgtb_set_state(vgtb_ctx* ctx, const void* buf, long long bytes);

/* Kernel timing: with enable = 1, propagate() records CUDA events around the
 * hot kernels on the context stream and accumulates their device time.
 * vgtb_kernel_stats() copies, for kernel classes 0..n-1 (see VGTB_K_*),
 * launches[i] and total milliseconds ms[i], and returns the class count.
 * Crank-Nicolson contexts use the same classes for: OBS = D = 2 C C^dagger and
 * the sums, GEMM1 = S^-1 H(t+dt/2), GEMM2 = the fixed-point sweeps, LEAP = the
 * convergence check and the step counter. */
#define VGTB_K_OBS     0   /* charges / current / energy sums (Eqs. 10, 14); split form: per atom, with dq */
#define VGTB_K_SCC     1   /* (FP64 forms: dq), eps = gamma dq, finalised observables */
#define VGTB_K_PHASE   2   /* Bloch sum of H_k(t) with A(t) (Eqs. 7-12) */
#define VGTB_K_GEMM1   3   /* first commutator product */
#define VGTB_K_GEMM2   4   /* second commutator product (S^-1 applied) */
#define VGTB_K_LEAP    5   /* leapfrog update (Eq. 13) */
#define VGTB_K_COUNT   6
int vgtb_profile(vgtb_ctx* ctx, int enable);
int vgtb_kernel_stats(vgtb_ctx* ctx, long long* launches, double* ms, int n);

/* Text of the last error on this context (or of the last failed create when
 * ctx is NULL).  Valid until the next call on the same context. */
/* Split-precision contexts: the tile variant each tcgen05 product runs with
 * (product 1 = [dD|D0][H|dH]^dagger, product 2 = S^-1 W^dagger), chosen at
 * create (variant 0, or the autotuner's fastest).  cfg[4] = {tile width,
 * pipeline stages, schedule (0 classic, 1 stream-K, 2 whole waves classic and
 * stream-K over the rest; + 4: the k-panels skipped in which the tile's rows
 * of H_k and dH_k are zero, product 1 only; + 8: classic over column tiles of
 * planned widths, multiples of 16, the tile width being the widest; + 16: both
 * products run as one launch, VGTB_CHAIN_*), 1 if the tile spans a 2-SM CTA pair}.  When the first product runs block-sparse
 * (VGTB_P1_BLOCKS), product 1 reports {atoms per group, output rows per CTA, 3, 0}.
 * Errors: E_INVALID (product not 1 or 2, NULL), E_STATE (FP64 context). */
int vgtb_tile_config(const vgtb_ctx* ctx, int product, int* cfg);

const char* vgtb_last_error(const vgtb_ctx* ctx);

/* Release the context and all its device memory.  NULL-safe. */
void vgtb_destroy(vgtb_ctx* ctx);

/* Complex product C = A R^dagger with the split-precision tcgen05 kernel of
 * the propagation (BF16 hi/lo pieces, three products, FP32 accumulation), for
 * callers that must not allocate device memory: code whose device memory is
 * owned by another allocator (a framework caching allocator or a pool that has
 * reserved the HBM, where a cudaMalloc fails or fragments it) and loops that
 * cannot take the implicit device synchronisation of cudaMalloc/cudaFree.
 * The paper has no counterpart; it is a library-level variant.
 *
 * a, r, c: DEVICE pointers to n x n complex matrices, row-major, interleaved
 * (re, im) doubles, owned by the caller; c is written.  1 <= n <= 256.
 * stream: cudaStream_t to run on (NULL = the legacy default stream); the call
 * synchronises that stream before it returns.
 * The call allocates nothing: its scratch (BF16 pieces, the FP32 product, a
 * problem table and an error word, 2 MiB + 512 B) is one static device array
 * that every GPU which loads the library holds until the process exits.  The
 * first call on a device (and the first call after that device's context was
 * replaced, e.g. by cudaDeviceReset) looks up the array's device address and
 * raises the kernel's shared-memory limit; make that first call before any
 * stream capture.  First calls from several host threads are serialised by a
 * lock inside the library.  All calls share the array and it keeps the last call's contents
 * (each call rewrites, zero padding included, everything it reads), so calls
 * whose work overlaps on the GPU (other streams or host threads) race.
 * Returns VGTB_OK; VGTB_E_INVALID for n outside 1..256 or a NULL pointer;
 * VGTB_E_UNSUPPORTED without an sm_103a device; VGTB_E_TIMEOUT when a bounded
 * device wait expired (c is then left unwritten); VGTB_E_CUDA for a failed
 * CUDA call (the contents of c are then unspecified). */
int vgtb_split_cgemm_noalloc(int n, const double* a, const double* r, double* c, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* VGTB_H */
