// Host interface of the tcgen05 split-precision complex products (k_gemm_tc.cu).
#pragma once
#include <string>
#include <vector>

#include "vgtb_internal.h"

namespace vgtb {

struct TcPlan;  // tensor maps, problem table and launch shape of one product

// Operand families of one system, each contiguous over that system's items
// (items in creation order: trajectory-major, k-minor).
struct TcSysView {
  int Np, nk, n_items;
  __nv_bfloat16* Sinv_p;   // [nk][2][Np][2Np]
  __nv_bfloat16* D0_p;     // [nk][2][Np][2Np]
  __nv_bfloat16* dD_p;     // [n_items][2][Np][2Np]
  __nv_bfloat16* Hemb_p;   // [n_items][2][2Np][2Np]
  __nv_bfloat16* dHemb_p;  // [n_items][2][2Np][2Np]
  __nv_bfloat16* Wemb_p;   // [n_items][2][2Np][2Np]
  // nonzero pattern of H_k (host data, may be null): orbital offsets of the
  // atoms and the atom pairs (I, J) of the targets.  With it, the classic
  // schedules of product 1 skip the k-panels in which a tile's rows of H and dH
  // are zero.
  const std::vector<int>* orb_off = nullptr;
  const std::vector<int>* tgt_I = nullptr;
  const std::vector<int>* tgt_J = nullptr;
};

// Plans for the two products of the split form, over every item:
//   product 1: W = [dD | D0] [H | dH]^dagger  -> embedded BF16 hi/lo pieces of W
//   product 2: X = S^-1 W^dagger               -> FP32 planar X
// force_variant[p] >= 0 uses that tile variant for product p+1; otherwise variant
// 0, or with autotune the fastest candidate (median of 9 timed launches).
// p1 == nullptr builds product 2 only (the first product runs block-sparse).
// When autotuning, *alt1 / *alt2 (if given) receive the fastest chainable plan
// of each product (tc_chainable) when that is not already the chosen plan, else
// nullptr; the caller owns them.  ms_best[2] (if given) receives the median
// times of the chosen plans (0 without autotuning).
// Returns 0 on success, else fills *msg.
int tc_build_plans(const std::vector<TcSysView>& sys, const std::vector<DevItem>& items, long long timeout_ns,
                   int autotune, const int force_variant[2], cudaStream_t st, TcPlan** p1, TcPlan** p2,
                   std::string* msg, TcPlan** alt1 = nullptr, TcPlan** alt2 = nullptr, double* ms_best = nullptr);
int tc_num_variants();
// {tile width, pipeline stages, schedule (0 classic, 1 stream-K, 2 classic waves + stream-K rest), 2-SM pair}
int tc_variant_info(int v, int* out4);
// tc_variant_info of the plan, with schedule 4 for a classic schedule that skips zero k-panels
int tc_plan_info(const TcPlan* p, int* out4);
int tc_launch(TcPlan* p, cudaStream_t st);
int tc_status(TcPlan* p, cudaStream_t st);  // 0 or the plan's device error word
void tc_destroy_plan(TcPlan* p);
int tc_plan_variant(const TcPlan* p);  // index of the tile variant the plan uses
void tc_clear_error(TcPlan* p);        // zero the plan's device error word

// Chained schedule: both products in one launch (tc_chain.cuh), over the
// tables of two plans that it does not own (2-SM pair, classic schedule,
// 64-column stages: tc_chainable).  tc_time_chain times it against two
// separate launches of p1 and p2, which may be other plans than the chain's
// (median of 9 each; -1 if a launch failed or timed out).
struct TcChain;
bool tc_chainable(const TcPlan* p1, const TcPlan* p2);
int tc_build_chain(const TcPlan* p1, const TcPlan* p2, TcChain** out, std::string* msg);
int tc_launch_chain(TcChain* c, cudaStream_t st);
int tc_time_chain(TcChain* c, TcPlan* p1, TcPlan* p2, cudaStream_t st, double* ms_chain, double* ms_sep);
void tc_reset_chain(TcChain* c, cudaStream_t st);  // zero the block counts and the launch count
void tc_destroy_chain(TcChain* c);

}  // namespace vgtb
