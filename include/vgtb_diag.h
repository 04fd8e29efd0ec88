/*
 * vgtb_diag.h - diagnostic entry point of libvgtb (kernel unit tests).
 *
 * Runs the two tcgen05 split-precision products of the commutator of Eq. 6
 * in isolation, on caller matrices, exactly as vgtb_propagate() does:
 *   W = A R^dagger   (product 1; its output is stored as embedded BF16 pieces)
 *   X = S W^dagger   (product 2; FP32 output)
 * The inputs are N x N complex matrices (host pointers, row-major, interleaved
 * re/im doubles); none of them needs to be Hermitian.
 * Outputs (caller-allocated, N x N complex): W read back from its hi + lo
 * pieces, and X.  Returns VGTB_OK or a VGTB_E_* code (VGTB_E_UNSUPPORTED
 * without an sm_103a device).  Allocates and frees its own device memory.
 */
#ifndef VGTB_DIAG_H
#define VGTB_DIAG_H
#ifdef __cplusplus
extern "C" {
#endif

int vgtb_diag_split_chain(int n, const double* a, const double* r, const double* s, double* w_out,
                          double* x_out);

/* The same with both products forced to tile variant `variant` (0 ..
 * vgtb_diag_num_variants()-1; -1 = the default), so that every schedule the
 * autotuner may pick (classic, stream-K, classic waves + stream-K; single CTA
 * or 2-SM pair) can be checked on its own.  E_INVALID for an index out of range. */
int vgtb_diag_split_chain_variant(int n, const double* a, const double* r, const double* s, int variant,
                                  double* w_out, double* x_out);
int vgtb_diag_num_variants(void);

/* The library's integer-bit float <-> double conversions (used by the
 * split-precision kernels on their hot path) run on the device beside the CUDA
 * conversions, for unit tests.  The paper has no counterpart.
 * d_in [n] doubles -> f_bits[n] (d2f_bits) and f_ref[n] (__double2float_rn);
 * f_in [n] floats  -> d_bits[n] (f2d_bits) and d_ref[n] (the exact widening).
 * All host pointers, caller-owned; n >= 0.  Returns VGTB_OK, VGTB_E_INVALID
 * (negative n or a NULL pointer with n > 0) or VGTB_E_CUDA.  Allocates and
 * frees its own device memory. */
int vgtb_diag_convert(int n, const double* d_in, const float* f_in, float* f_bits, float* f_ref, double* d_bits,
                      double* d_ref);

/* The bounded device waits of the tcgen05 product kernels, made to run out: one
 * thread waits, with the kernels' own wait routine, for an mbarrier phase that no
 * thread completes (which = 0) or for a stream-K partial flag that no CTA sets
 * (which = 1), limited to limit_ns (1 .. 10^10 ns).  The wait gives up, records
 * the expiry in an error word and the kernel returns; the call then returns
 * VGTB_E_TIMEOUT.  VGTB_OK would mean the wait ended without its event (a
 * defect).  The paper has no counterpart.  Errors: VGTB_E_INVALID (which or
 * limit out of range), VGTB_E_UNSUPPORTED (no sm_103a device), VGTB_E_CUDA. */
int vgtb_diag_bounded_wait(long long limit_ns, int which);

#ifdef __cplusplus
}
#endif
#endif
