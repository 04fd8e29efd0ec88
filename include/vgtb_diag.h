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

#ifdef __cplusplus
}
#endif
#endif
