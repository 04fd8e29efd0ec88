// Host side of the tcgen05 split-precision complex products (Eq. 6): tensor
// maps, problem tables over all items, variant autotuner and launches.  The
// device code is in tc_kernel.cuh.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "tc_chain.cuh"

namespace vgtb {

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 4-D BF16 map: (cols, rows, 2 pieces, batch), box (64 / kh, box_rows, 1, 1),
// 128-byte swizzle (kh = 1) or 64-byte swizzle (kh = 2)
bool encode_map(CUtensorMap* m, const void* base, int cols, int rows, int batch, int box_rows, std::string* msg,
                int kh = 1) {
  auto enc = get_encode();
  if (!enc) {
    *msg = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)rows, 2, (cuuint64_t)batch};
  cuuint64_t strides[3] = {(cuuint64_t)cols * 2, (cuuint64_t)cols * rows * 2, (cuuint64_t)cols * rows * 4};
  cuuint32_t box[4] = {(cuuint32_t)(BK / kh), (cuuint32_t)box_rows, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, kh == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char b[128];
    snprintf(b, sizeof(b), "cuTensorMapEncodeTiled failed (%d) for %dx%dx2x%d box %d", (int)r, cols, rows, batch,
             box_rows);
    *msg = b;
    return false;
  }
  return true;
}

struct Variant {
  int bn, st, streamk, pair, widths, kh;
};
// tile width (per CTA, or per pair for the 2-SM variant; the largest width
// with planned widths), pipeline stages, schedule (0 classic, 1 stream-K over
// all tiles, 2 whole waves classic and stream-K over the rest), 2-SM pair,
// column tiles (0: all bn wide; 1: the split of the 2 Np B rows into tiles of
// near-equal widths, multiples of 16, with the shortest modelled time of the
// longest worker, see plan_columns; 2: the same among splits into tiles at
// least 192 wide, which re-read the A operand less often), k-slices per 64-wide
// panel (1: stages of 64 columns; 2: stages of 32 columns, 7 of them, for the
// pair kernel).  Variant 0 is the default; all are
// autotune candidates.
constexpr Variant kVariants[] = {{256, 3, 0, 1, 0, 1}, {256, 3, 1, 1, 0, 1}, {256, 3, 2, 1, 0, 1},
                                 {256, 2, 0, 0, 0, 1}, {256, 2, 1, 0, 0, 1}, {128, 3, 0, 0, 0, 1},
                                 {128, 3, 1, 0, 0, 1}, {256, 3, 0, 1, 1, 1}, {256, 3, 0, 1, 2, 1},
                                 {256, 7, 0, 1, 0, 2}, {256, 7, 0, 1, 1, 2}, {256, 7, 1, 1, 0, 2}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

template <int BN, int ST, int EPI>
int smem_bytes() {
  return ST * (2 * BM * BK * 2 + 2 * BN * BK * 2) + 1024 + 256;
}

template <int BN, int ST, int EPI>
cudaError_t launch_t(const TcPlan* p, cudaStream_t st) {
  return launch_pdl(k_tc_gemm<BN, ST, EPI>, p->grid, 192, p->smem, st, p->P);
}

template <int ST, int KH>
int smem_pair() {
  return ST * (2 * BM * (BK / KH) * 2 + 2 * 128 * (BK / KH) * 2) + 1024 + 256;
}

template <int ST, int EPI, int KH>
cudaError_t launch_pair(const TcPlan* p, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p->grid, 1, 1);
  cfg.blockDim = dim3(192, 1, 1);
  cfg.dynamicSmemBytes = p->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_tc_gemm2<ST, EPI, KH>, p->P);
}

template <int BN, int ST, int EPI>
cudaError_t configure_t() {
  return cudaFuncSetAttribute(k_tc_gemm<BN, ST, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_bytes<BN, ST, EPI>());
}

cudaError_t launch_variant(const TcPlan* p, cudaStream_t st) {
  if (kVariants[p->variant].pair) {
    if (kVariants[p->variant].kh == 2)
      return p->epi == 0 ? launch_pair<7, 0, 2>(p, st) : launch_pair<7, 1, 2>(p, st);
    return p->epi == 0 ? launch_pair<3, 0, 1>(p, st) : launch_pair<3, 1, 1>(p, st);
  }
  const bool wide = kVariants[p->variant].bn == 256;
  if (p->epi == 0) return wide ? launch_t<256, 2, 0>(p, st) : launch_t<128, 3, 0>(p, st);
  return wide ? launch_t<256, 2, 1>(p, st) : launch_t<128, 3, 1>(p, st);
}

int variant_smem(int v) {
  if (kVariants[v].pair) return kVariants[v].kh == 2 ? smem_pair<7, 2>() : smem_pair<3, 1>();
  return kVariants[v].bn == 256 ? smem_bytes<256, 2, 0>() : smem_bytes<128, 3, 0>();
}

cudaError_t configure_all() {
  cudaError_t e;
  if ((e = configure_t<256, 2, 0>()) != cudaSuccess) return e;
  if ((e = configure_t<128, 3, 0>()) != cudaSuccess) return e;
  if ((e = configure_t<256, 2, 1>()) != cudaSuccess) return e;
  if ((e = configure_t<128, 3, 1>()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_tc_gemm2<3, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_pair<3, 1>())) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_tc_gemm2<3, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_pair<3, 1>())) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_tc_gemm2<7, 0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_pair<7, 2>())) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_tc_gemm2<7, 1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_pair<7, 2>())) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_tc_chain<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_pair<3, 1>());
}

}  // namespace

int tc_gemm_supported() {
  int dev = 0, maj = 0, min = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
  return (maj == 10 && min == 3) ? 1 : 0;
}

// Nonzero k-panels of each B column tile of product 1 for system v (tile nt =
// B rows starts[nt] .. starts[nt+1]-1 of the embedded [[Re H, Im H], [-Im H, Re H]],
// rows interleaved in blocks of four: B row n' holds H row 4 (n' / 8) + n' % 4): a panel kt covers
// the 64 columns k' = 64 kt .. 64 kt + 63 of a segment, i.e. H columns k' (real
// half) or k' - Np (imaginary half); it is nonzero for the tile when some H row
// of the tile belongs to an atom I with a target (I, J) whose columns meet the
// panel.  H and dH share the pattern.
// uniform = true pads every tile's list with panels of zeros (in increasing
// order) to the longest list, so that all tiles take the same number of
// k-iterations, as the stream-K schedules need.
static void zero_panel_lists(const TcSysView& v, const std::vector<int>& starts, bool uniform,
                             std::vector<int>& kofs, std::vector<short>& kidx) {
  const std::vector<int>& off = *v.orb_off;
  const int nat = (int)off.size() - 1, N = off[nat], Np = v.Np;
  const int npan = 2 * Np / BK;
  std::vector<int> atom_of(N);
  for (int a = 0; a < nat; ++a)
    for (int o = off[a]; o < off[a + 1]; ++o) atom_of[o] = a;
  std::vector<std::vector<int>> nbr(nat);
  for (size_t t = 0; t < v.tgt_I->size(); ++t) nbr[(*v.tgt_I)[t]].push_back((*v.tgt_J)[t]);
  const int tiles_n = (int)starts.size() - 1;
  std::vector<std::vector<char>> pans(tiles_n);
  size_t longest = 1;
  for (int nt = 0; nt < tiles_n; ++nt) {
    std::vector<char> atoms(nat, 0), pan(npan, 0);
    for (int r = starts[nt]; r < starts[nt + 1]; ++r) {
      const int row = 4 * (r / 8) + (r % 4);
      if (row < N) atoms[atom_of[row]] = 1;
    }
    for (int a = 0; a < nat; ++a)
      if (atoms[a])
        for (int J : nbr[a])
          for (int c = off[J]; c < off[J + 1]; ++c) {
            pan[c / BK] = 1;
            pan[(Np + c) / BK] = 1;
          }
    size_t cnt = 0;
    for (int k = 0; k < npan; ++k) cnt += pan[k] ? 1 : 0;
    longest = std::max(longest, cnt);
    pans[nt] = pan;
  }
  kofs.assign(1, 0);
  kidx.clear();
  for (int nt = 0; nt < tiles_n; ++nt) {
    std::vector<char>& pan = pans[nt];
    size_t cnt = 0;
    for (int k = 0; k < npan; ++k) cnt += pan[k] ? 1 : 0;
    // a tile of padding rows only gets one panel of zeros, which clears its accumulator;
    // with uniform lists every tile is padded with zero panels to the longest list
    const size_t want = uniform ? longest : std::max<size_t>(cnt, 1);
    for (int k = 0; k < npan && cnt < want; ++k)
      if (!pan[k]) {
        pan[k] = 2;
        ++cnt;
      }
    for (int k = 0; k < npan; ++k)
      if (pan[k]) kidx.push_back((short)k);
    kofs.push_back(kofs.back() + (int)cnt);
  }
}

// Longest-processing-time assignment of tiles with costs cost[i] to G workers:
// each tile in decreasing cost goes to the worker with the least work so far.
// Returns the worker lists as the classic schedule's tile order (worker c takes
// tord[c], tord[c + G], ...; -1 ends a shorter list) and the modelled time of
// the longest worker in *span.
static std::vector<int> lpt_order(const std::vector<double>& cost, int G, double* span) {
  std::vector<int> idx(cost.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<int>> lists(G);
  std::vector<double> load(G, 0.0);
  for (int i : idx) {
    int c = 0;
    for (int g = 1; g < G; ++g)
      if (load[g] < load[c]) c = g;
    lists[c].push_back(i);
    load[c] += cost[i];
  }
  size_t depth = 0;
  for (auto& l : lists) depth = std::max(depth, l.size());
  std::vector<int> tord(depth * G, -1);
  for (int c = 0; c < G; ++c)
    for (size_t j = 0; j < lists[c].size(); ++j) tord[j * G + c] = lists[c][j];
  if (span) *span = *std::max_element(load.begin(), load.end());
  return tord;
}

// Modelled time of a tile in k-iterations of a 256-wide tile: its width share of
// its k-iterations, plus a fixed cost per tile (pipeline start, epilogue tail).
constexpr double kTileFixed = 2.0;
static double tile_model(int w, int kt) { return w / 256.0 * kt + kTileFixed; }

// 2 Np B rows split into n tiles of near-equal widths, multiples of 16
static std::vector<int> even_split(int total, int n) {
  const int units = total / 16, q = units / n, r = units % n;
  std::vector<int> st(1, 0);
  for (int i = 0; i < n; ++i) st.push_back(st.back() + 16 * (q + (i < r ? 1 : 0)));
  return st;
}

// Column tiles of the 2-SM pair kernel for system v: of the splits of its 2 Np
// B rows into n = 2Np/256 .. 2Np/96 tiles of near-equal widths (at most 256;
// mode 2: at least 192), the one with the shortest modelled time of the longest
// of G workers when all its tiles (n_items x tiles_m row tiles) are assigned
// longest first.  With the zero k-panels skipped a tile's k-iterations are its
// panel count.
static std::vector<int> plan_columns(const TcSysView& v, bool skip, int nseg, int tiles_m, int G, int mode) {
  const int total = 2 * v.Np, n0 = (total + 255) / 256;
  std::vector<std::pair<double, int>> score;
  for (int n = n0; n <= std::max(total / 96, n0); ++n) {
    const std::vector<int> st = even_split(total, n);
    if (mode == 2 && n > n0 && st[n] - st[n - 1] < 192) continue;
    std::vector<int> kt(n, nseg * total / BK);
    if (skip) {
      std::vector<int> kofs;
      std::vector<short> kidx;
      zero_panel_lists(v, st, false, kofs, kidx);
      for (int i = 0; i < n; ++i) kt[i] = nseg * (kofs[i + 1] - kofs[i]);
    }
    std::vector<double> cost;
    for (int it = 0; it < v.n_items; ++it)
      for (int i = 0; i < n; ++i)
        for (int m = 0; m < tiles_m; ++m) cost.push_back(tile_model(st[i + 1] - st[i], kt[i]));
    double span = 0;
    lpt_order(cost, G, &span);
    score.push_back({span, n});
  }
  std::stable_sort(score.begin(), score.end());
  return even_split(total, score[0].second);
}

static int build_one(const std::vector<TcSysView>& sys, const std::vector<DevItem>& items, int epi, int variant,
                     long long timeout_ns, TcPlan* plan, std::string* msg) {
  const Variant& var = kVariants[variant];
  const int BNv = var.bn;
  const bool pair = var.pair != 0;
  const int tm_rows = pair ? 2 * BM : BM;  // output rows of one tile
  const int nseg = epi == 0 ? 2 : 1;
  memset(&plan->P, 0, sizeof(plan->P));
  plan->epi = epi;
  plan->variant = variant;
  if ((int)sys.size() > kMaxSys) {
    *msg = "too many systems in one batch for the split form (max 4)";
    return -1;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int G_full = pair ? nsm / 2 : nsm;
  // zero-panel skipping: product 1, every system's pattern known; the stream-K
  // schedules get lists of one length per system (see zero_panel_lists)
  bool skip = epi == 0;
  const bool uniform = var.streamk != 0;
  for (const TcSysView& v : sys) skip = skip && v.orb_off && v.tgt_I && v.tgt_J;
  // column tiles of every system
  std::vector<std::vector<int>> starts(sys.size());
  int wmax = 0;
  for (size_t s = 0; s < sys.size(); ++s) {
    const int tiles_m = (sys[s].Np + tm_rows - 1) / tm_rows;
    starts[s] = var.widths ? plan_columns(sys[s], skip, nseg, tiles_m, G_full, var.widths)
                           : even_split(2 * sys[s].Np, 2 * sys[s].Np / BNv);
    for (size_t i = 0; i + 1 < starts[s].size(); ++i) wmax = std::max(wmax, starts[s][i + 1] - starts[s][i]);
  }
  const int bbox = pair ? wmax / 2 : BNv;  // B rows loaded by one CTA
  plan->wmax = wmax;
  plan->P.b_rows = pair ? bbox : 0;
  for (size_t s = 0; s < sys.size(); ++s) {
    const TcSysView& v = sys[s];
    const int Np = v.Np;
    if (epi == 0) {
      if (!encode_map(&plan->P.mA[s][0], v.dD_p, 2 * Np, Np, v.n_items, BM, msg, var.kh)) return -1;
      if (!encode_map(&plan->P.mA[s][1], v.D0_p, 2 * Np, Np, v.nk, BM, msg, var.kh)) return -1;
      if (!encode_map(&plan->P.mB[s][0], v.Hemb_p, 2 * Np, 2 * Np, v.n_items, bbox, msg, var.kh)) return -1;
      if (!encode_map(&plan->P.mB[s][1], v.dHemb_p, 2 * Np, 2 * Np, v.n_items, bbox, msg, var.kh)) return -1;
    } else {
      if (!encode_map(&plan->P.mA[s][0], v.Sinv_p, 2 * Np, Np, v.nk, BM, msg, var.kh)) return -1;
      if (!encode_map(&plan->P.mB[s][0], v.Wemb_p, 2 * Np, 2 * Np, v.n_items, bbox, msg, var.kh)) return -1;
    }
  }
  std::vector<int> sys_kofs0(sys.size(), 0), sys_kidx0(sys.size(), 0), sys_cofs0(sys.size(), 0), all_kofs, all_cofs;
  std::vector<short> all_kidx;
  std::vector<std::vector<int>> sys_cnt(sys.size());
  if (skip) {
    for (size_t s = 0; s < sys.size(); ++s) {
      std::vector<int> kofs;
      std::vector<short> kidx;
      zero_panel_lists(sys[s], starts[s], uniform, kofs, kidx);
      sys_kofs0[s] = (int)all_kofs.size();
      sys_kidx0[s] = (int)all_kidx.size();
      for (size_t i = 0; i + 1 < kofs.size(); ++i) sys_cnt[s].push_back(kofs[i + 1] - kofs[i]);
      all_kofs.insert(all_kofs.end(), kofs.begin(), kofs.end());
      all_kidx.insert(all_kidx.end(), kidx.begin(), kidx.end());
    }
    if (cudaMalloc(&plan->d_kofs, sizeof(int) * all_kofs.size()) != cudaSuccess ||
        cudaMalloc(&plan->d_kidx, sizeof(short) * all_kidx.size()) != cudaSuccess) {
      *msg = "cudaMalloc failed for the k-panel lists";
      return -1;
    }
    cudaMemcpy(plan->d_kofs, all_kofs.data(), sizeof(int) * all_kofs.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(plan->d_kidx, all_kidx.data(), sizeof(short) * all_kidx.size(), cudaMemcpyHostToDevice);
    plan->skip = true;
  }
  if (var.widths) {
    for (size_t s = 0; s < sys.size(); ++s) {
      sys_cofs0[s] = (int)all_cofs.size();
      all_cofs.insert(all_cofs.end(), starts[s].begin(), starts[s].end());
    }
    if (cudaMalloc(&plan->d_cofs, sizeof(int) * all_cofs.size()) != cudaSuccess) {
      *msg = "cudaMalloc failed for the column tiles";
      return -1;
    }
    cudaMemcpy(plan->d_cofs, all_cofs.data(), sizeof(int) * all_cofs.size(), cudaMemcpyHostToDevice);
  }
  std::vector<TcProb> probs;
  std::vector<int> local(sys.size(), 0);
  std::vector<double> tile_cost;  // modelled time of every tile, for the longest-first order
  int tiles = 0;
  long long iters = 0;
  for (const DevItem& it : items) {
    const TcSysView& v = sys[it.sys];
    const std::vector<int>& st = starts[it.sys];
    TcProb pr{};
    pr.sys = it.sys;
    const int li = local[it.sys]++;
    pr.Np = v.Np;
    pr.tiles_m = (v.Np + tm_rows - 1) / tm_rows;
    pr.tiles_n = (int)st.size() - 1;
    pr.tile0 = tiles;
    if (epi == 0) {
      pr.a_b[0] = li;
      pr.b_b[0] = li;
      pr.a_b[1] = it.k;
      pr.b_b[1] = li;
      pr.out = it.Wemb_p;
    } else {
      pr.a_b[0] = it.k;
      pr.b_b[0] = li;
      pr.out = it.Xf;
    }
    pr.kt = nseg * (2 * v.Np) / BK;
    pr.iter0 = (int)iters;
    if (skip) {
      pr.kofs = plan->d_kofs + sys_kofs0[it.sys];
      pr.kidx = plan->d_kidx + sys_kidx0[it.sys];
      pr.kt = nseg * sys_cnt[it.sys][0];  // every segment takes the panel list (uniform lists: one length)
    }
    if (var.widths) pr.cofs = plan->d_cofs + sys_cofs0[it.sys];
    for (int nt = 0; nt < pr.tiles_n; ++nt)
      for (int mt = 0; mt < pr.tiles_m; ++mt)
        tile_cost.push_back(tile_model(st[nt + 1] - st[nt], skip ? nseg * sys_cnt[it.sys][nt] : pr.kt));
    tiles += pr.tiles_m * pr.tiles_n;
    iters += (long long)pr.tiles_m * pr.tiles_n * pr.kt;
    probs.push_back(pr);
  }
  if (cudaMalloc(&plan->d_probs, sizeof(TcProb) * probs.size()) != cudaSuccess ||
      cudaMalloc(&plan->d_err, sizeof(int)) != cudaSuccess) {
    *msg = "cudaMalloc failed for the product plan";
    return -1;
  }
  cudaMemcpy(plan->d_probs, probs.data(), sizeof(TcProb) * probs.size(), cudaMemcpyHostToDevice);
  cudaMemset(plan->d_err, 0, sizeof(int));
  plan->probs_h = probs;
  plan->starts_h = starts;
  plan->cost_h = tile_cost;
  plan->P.probs = plan->d_probs;
  plan->P.n_prob = (int)probs.size();
  plan->P.total_tiles = tiles;
  plan->P.nseg = nseg;
  plan->P.err = plan->d_err;
  plan->P.timeout_ns = timeout_ns;
  plan->grid = std::min(tiles, nsm);
  plan->smem = variant_smem(variant);
  if (pair) plan->grid = 2 * std::min(tiles, nsm / 2);
  if (!var.streamk && ((skip && !uniform) || var.widths)) {
    // tiles of unequal cost: longest first, each to the least loaded worker
    const std::vector<int> tord = lpt_order(tile_cost, pair ? plan->grid / 2 : plan->grid, nullptr);
    if (cudaMalloc(&plan->d_tord, sizeof(int) * tord.size()) != cudaSuccess) {
      *msg = "cudaMalloc failed for the tile order";
      return -1;
    }
    cudaMemcpy(plan->d_tord, tord.data(), sizeof(int) * tord.size(), cudaMemcpyHostToDevice);
    plan->P.tord = plan->d_tord;
    plan->P.n_tord = (int)tord.size();
  }
  // stream-K needs every CTA to own at least one k-iteration; otherwise fall back
  if (var.streamk && iters >= 2LL * nsm) {
    plan->grid = pair ? (nsm & ~1) : nsm;  // pairs: workers are the nsm / 2 clusters
    plan->P.streamk = 1;
    plan->P.total_iters = iters;
    // schedule 2: whole waves of tiles first (classic order), stream-K over the
    // remainder; a remainder thinner than two k-iterations per worker is not
    // shared that way.  Schedule 1: stream-K over every tile.
    const int G = pair ? plan->grid / 2 : plan->grid;
    int t0 = 0;
    long long i0 = 0;
    if (var.streamk == 2) {
      t0 = (tiles / G) * G;
      i0 = iters;
      for (const TcProb& pr : probs)
        if (t0 >= pr.tile0 && t0 < pr.tile0 + pr.tiles_m * pr.tiles_n)
          i0 = pr.iter0 + (long long)(t0 - pr.tile0) * pr.kt;
      if (iters - i0 < 2LL * G) {
        t0 = 0;
        i0 = 0;
      }
    }
    plan->P.sk_tile0 = t0;
    plan->P.sk_iter0 = i0;
    if (cudaMalloc(&plan->d_ws, sizeof(float) * (size_t)nsm * BM * BNv) != cudaSuccess ||
        cudaMalloc(&plan->d_flags, sizeof(int) * nsm) != cudaSuccess) {
      *msg = "cudaMalloc failed for the stream-K workspace";
      return -1;
    }
    cudaMemset(plan->d_flags, 0, sizeof(int) * nsm);
    plan->P.ws = plan->d_ws;
    plan->P.flags = plan->d_flags;
  }
  return 0;
}

// median device time of 9 launches after 2 warm-up launches
static double time_plan(TcPlan* p, cudaStream_t st) {
  constexpr int R = 9;
  cudaEvent_t ev[R + 1];
  for (auto& e : ev) cudaEventCreate(&e);
  launch_variant(p, st);
  launch_variant(p, st);
  cudaEventRecord(ev[0], st);
  for (int i = 0; i < R; ++i) {
    launch_variant(p, st);
    cudaEventRecord(ev[i + 1], st);
  }
  cudaEventSynchronize(ev[R]);
  float ms[R];
  for (int i = 0; i < R; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  for (auto& e : ev) cudaEventDestroy(e);
  std::sort(ms, ms + R);
  return ms[R / 2];
}

int tc_num_variants() { return kNumVariants; }

int tc_variant_info(int v, int* out4) {
  if (v < 0 || v >= kNumVariants) return -1;
  out4[0] = kVariants[v].bn;
  out4[1] = kVariants[v].st;
  out4[2] = kVariants[v].streamk;
  out4[3] = kVariants[v].pair;
  return 0;
}

static bool variant_chainable(int v) {
  const Variant& a = kVariants[v];
  return a.pair && !a.streamk && a.kh == 1;
}

int tc_build_plans(const std::vector<TcSysView>& sys, const std::vector<DevItem>& items, long long timeout_ns,
                   int autotune, const int force_variant[2], cudaStream_t st, TcPlan** p1, TcPlan** p2,
                   std::string* msg, TcPlan** alt1, TcPlan** alt2, double* ms_best) {
  if (force_variant[0] >= kNumVariants || force_variant[1] >= kNumVariants) {
    *msg = "tile variant index out of range";
    return -1;
  }
  if (p1) *p1 = nullptr;
  *p2 = nullptr;
  if (alt1) *alt1 = nullptr;
  if (alt2) *alt2 = nullptr;
  if (ms_best) ms_best[0] = ms_best[1] = 0.0;
  if (configure_all() != cudaSuccess) {
    *msg = "cannot raise the shared-memory limit of the tcgen05 kernels";
    return -1;
  }
  for (int epi = p1 ? 0 : 1; epi < 2; ++epi) {
    // every variant that ran, with its median time; the fastest is the plan, and
    // the fastest chainable one (2-SM pair, classic, 64-column stages) is kept
    // beside it when it is another variant, for the one-launch schedule
    std::vector<std::pair<TcPlan*, double>> ran;
    // the pair kernel handles every Np (a multiple of 128), so variant 0 always applies
    const int fv = force_variant[epi];
    const int first = fv >= 0 ? fv : 0;
    const int nv = fv >= 0 ? first + 1 : (autotune ? kNumVariants : first + 1);
    for (int v = first; v < nv; ++v) {
      TcPlan* p = new TcPlan();
      if (build_one(sys, items, epi, v, timeout_ns, p, msg)) {
        tc_destroy_plan(p);
        for (auto& r : ran) tc_destroy_plan(r.first);
        return -1;
      }
      double ms = 0.0;
      if (nv - first > 1) {
        ms = time_plan(p, st);
        int err = 0;
        cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (cudaGetLastError() != cudaSuccess || err) {
          tc_destroy_plan(p);
          continue;
        }
      }
      ran.push_back({p, ms});
    }
    if (ran.empty()) {
      *msg = "no tcgen05 product variant ran";
      return -1;
    }
    int best = 0, bestc = -1;
    for (int i = 0; i < (int)ran.size(); ++i) {
      if (ran[i].second < ran[best].second) best = i;
      if (variant_chainable(ran[i].first->variant) && (bestc < 0 || ran[i].second < ran[bestc].second)) bestc = i;
    }
    TcPlan** alt = epi == 0 ? alt1 : alt2;
    const bool keep_alt = alt && bestc >= 0 && bestc != best;
    for (int i = 0; i < (int)ran.size(); ++i)
      if (i != best && !(keep_alt && i == bestc)) tc_destroy_plan(ran[i].first);
    cudaMemset(ran[best].first->d_err, 0, sizeof(int));
    (epi == 0 ? *p1 : *p2) = ran[best].first;
    if (ms_best) ms_best[epi] = ran[best].second;
    if (keep_alt) {
      cudaMemset(ran[bestc].first->d_err, 0, sizeof(int));
      *alt = ran[bestc].first;
    }
  }
  return 0;
}

int tc_launch(TcPlan* p, cudaStream_t st) {
  if (!p) return -1;
  return launch_variant(p, st) == cudaSuccess ? 0 : -1;
}

int tc_status(TcPlan* p, cudaStream_t st) {
  if (!p) return 0;
  int err = 0;
  cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return err;
}

void tc_destroy_plan(TcPlan* p) {
  if (!p) return;
  if (p->d_probs) cudaFree(p->d_probs);
  if (p->d_err) cudaFree(p->d_err);
  if (p->d_ws) cudaFree(p->d_ws);
  if (p->d_flags) cudaFree(p->d_flags);
  if (p->d_kofs) cudaFree(p->d_kofs);
  if (p->d_kidx) cudaFree(p->d_kidx);
  if (p->d_tord) cudaFree(p->d_tord);
  if (p->d_cofs) cudaFree(p->d_cofs);
  delete p;
}

int tc_plan_variant(const TcPlan* p) { return p ? p->variant : -1; }

void tc_clear_error(TcPlan* p) {
  if (p) cudaMemset(p->d_err, 0, sizeof(int));
}

int tc_plan_info(const TcPlan* p, int* out4) {
  if (!p || tc_variant_info(p->variant, out4)) return -1;
  if (p->skip) out4[2] += 4;  // 4, 5, 6: the schedule with zero k-panels skipped
  if (kVariants[p->variant].widths) {
    out4[0] = p->wmax;        // the widest column tile
    out4[2] += 8;             // 8, 12: classic over planned column widths
  }
  return 0;
}

// ----------------------------------------------------------------------------
// chained schedule (tc_chain.cuh)
// ----------------------------------------------------------------------------
struct TcChain {
  TcChainExtra X{};
  const TcPlan* p1 = nullptr;  // not owned
  const TcPlan* p2 = nullptr;
  int* d_ord = nullptr;
  int* d_blk0 = nullptr;
  unsigned long long* d_ready = nullptr;
  unsigned long long* d_epoch = nullptr;
  int grid = 0, smem = 0;
};

bool tc_chainable(const TcPlan* p1, const TcPlan* p2) {
  if (!p1 || !p2) return false;
  const Variant& a = kVariants[p1->variant];
  const Variant& b = kVariants[p2->variant];
  return a.pair && b.pair && !a.streamk && !b.streamk && a.kh == 1 && b.kh == 1 &&
         p1->probs_h.size() == p2->probs_h.size();
}

// The order of the units over G workers, by list scheduling on the modelled
// tile times: product 1 tiles block by block (problem, 256-row block, column
// tile), each to the worker free first; then product 2 tiles by the time at
// which the blocks of W they read are complete (then longest first), each to
// the worker free first, starting no earlier than that time.
static std::vector<int> chain_order(const TcPlan* p1, const TcPlan* p2, int G, double* span) {
  const std::vector<TcProb>& q1 = p1->probs_h;
  const std::vector<TcProb>& q2 = p2->probs_h;
  std::vector<double> avail(G, 0.0);
  std::vector<std::vector<int>> lists(G);
  auto take = [&](double ready, double cost, int unit) {
    int c = 0;
    for (int g = 1; g < G; ++g)
      if (avail[g] < avail[c]) c = g;
    const double start = std::max(avail[c], ready);
    avail[c] = start + cost;
    lists[c].push_back(unit);
    return avail[c];
  };
  std::vector<std::vector<double>> blk_done(q1.size());
  for (size_t p = 0; p < q1.size(); ++p) {
    const TcProb& pr = q1[p];
    blk_done[p].assign(pr.tiles_m, 0.0);
    for (int mt = 0; mt < pr.tiles_m; ++mt)
      for (int nt = 0; nt < pr.tiles_n; ++nt) {
        const int t = pr.tile0 + nt * pr.tiles_m + mt;
        blk_done[p][mt] = std::max(blk_done[p][mt], take(0.0, p1->cost_h[t], t));
      }
  }
  struct U2 {
    double ready, cost;
    int unit;
  };
  std::vector<U2> u2;
  const int t1 = p1->P.total_tiles;
  for (size_t p = 0; p < q2.size(); ++p) {
    const TcProb& pr = q2[p];
    const std::vector<int>& st = p2->starts_h[pr.sys];
    const int Np = pr.Np;
    for (int nt = 0; nt < pr.tiles_n; ++nt) {
      const int cb = st[nt], w = st[nt + 1] - st[nt];
      double ready = 0.0;
      const int seg[2][2] = {{cb, std::min(cb + w, Np)}, {std::max(cb, Np) - Np, cb + w - Np}};
      for (auto& sg : seg)
        if (sg[1] > sg[0])
          for (int b = sg[0] / 256; b <= (sg[1] - 1) / 256; ++b) ready = std::max(ready, blk_done[p][b]);
      for (int mt = 0; mt < pr.tiles_m; ++mt) {
        const int t = pr.tile0 + nt * pr.tiles_m + mt;
        u2.push_back({ready, p2->cost_h[t], t1 + t});
      }
    }
  }
  std::stable_sort(u2.begin(), u2.end(), [](const U2& a, const U2& b) {
    return a.ready < b.ready || (a.ready == b.ready && a.cost > b.cost);
  });
  for (const U2& u : u2) take(u.ready, u.cost, u.unit);
  size_t depth = 0;
  for (auto& l : lists) depth = std::max(depth, l.size());
  std::vector<int> ord(depth * G, -1);
  for (int c = 0; c < G; ++c)
    for (size_t j = 0; j < lists[c].size(); ++j) ord[j * G + c] = lists[c][j];
  if (span) *span = *std::max_element(avail.begin(), avail.end());
  return ord;
}

int tc_build_chain(const TcPlan* p1, const TcPlan* p2, TcChain** out, std::string* msg) {
  *out = nullptr;
  if (!tc_chainable(p1, p2)) {
    *msg = "the two products cannot be chained (2-SM pair, classic schedule and 64-column stages needed)";
    return -1;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // every pair must be resident at once (a product 2 tile may wait for a tile of
  // any other pair): at most the clusters of two that fit on the device
  int G = std::max(1, std::min(nsm / 2, std::max(p1->P.total_tiles, p2->P.total_tiles)));
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * G, 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = smem_pair<3, 1>();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int maxc = 0;
    if (cudaOccupancyMaxActiveClusters(&maxc, k_tc_chain<3>, &cfg) != cudaSuccess || maxc < 1) {
      *msg = "cannot query the resident clusters of the chained kernel";
      return -1;
    }
    G = std::min(G, maxc);
  }
  TcChain* c = new TcChain();
  c->p1 = p1;
  c->p2 = p2;
  c->grid = 2 * G;
  c->smem = smem_pair<3, 1>();
  const std::vector<int> ord = chain_order(p1, p2, G, nullptr);
  std::vector<int> blk0;
  int nblk = 0;
  for (const TcProb& pr : p1->probs_h) {
    blk0.push_back(nblk);
    nblk += pr.tiles_m;
  }
  if (cudaMalloc(&c->d_ord, sizeof(int) * ord.size()) != cudaSuccess ||
      cudaMalloc(&c->d_blk0, sizeof(int) * blk0.size()) != cudaSuccess ||
      cudaMalloc(&c->d_ready, sizeof(unsigned long long) * nblk) != cudaSuccess ||
      cudaMalloc(&c->d_epoch, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    tc_destroy_chain(c);
    *msg = "cudaMalloc failed for the chained schedule";
    return -1;
  }
  cudaMemcpy(c->d_ord, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_blk0, blk0.data(), sizeof(int) * blk0.size(), cudaMemcpyHostToDevice);
  cudaMemset(c->d_ready, 0, sizeof(unsigned long long) * nblk);
  cudaMemset(c->d_epoch, 0, 2 * sizeof(unsigned long long));
  c->X.ord = c->d_ord;
  c->X.n_ord = (int)ord.size();
  c->X.t1 = p1->P.total_tiles;
  c->X.ready = c->d_ready;
  c->X.blk0 = c->d_blk0;
  c->X.epoch = c->d_epoch;
  *out = c;
  return 0;
}

int tc_launch_chain(TcChain* c, cudaStream_t st) {
  if (!c) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->grid, 1, 1);
  cfg.blockDim = dim3(192, 1, 1);
  cfg.dynamicSmemBytes = c->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_tc_chain<3>, c->p1->P, c->p2->P, c->X) == cudaSuccess ? 0 : -1;
}

// median device times of 9 chained launches and of 9 pairs of separate launches
int tc_time_chain(TcChain* c, TcPlan* p1, TcPlan* p2, cudaStream_t st, double* ms_chain, double* ms_sep) {
  constexpr int R = 9;
  cudaEvent_t ev[R + 1];
  for (auto& e : ev) cudaEventCreate(&e);
  float a[R], b[R];
  for (int pass = 0; pass < 2; ++pass) {
    float* ms = pass ? b : a;
    for (int w = 0; w < 2; ++w) {
      if (pass) {
        launch_variant(p1, st);
        launch_variant(p2, st);
      } else {
        tc_launch_chain(c, st);
      }
    }
    cudaEventRecord(ev[0], st);
    for (int i = 0; i < R; ++i) {
      if (pass) {
        launch_variant(p1, st);
        launch_variant(p2, st);
      } else {
        tc_launch_chain(c, st);
      }
      cudaEventRecord(ev[i + 1], st);
    }
    cudaEventSynchronize(ev[R]);
    for (int i = 0; i < R; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  std::sort(a, a + R);
  std::sort(b, b + R);
  *ms_chain = a[R / 2];
  *ms_sep = b[R / 2];
  int err = 0, errc = 0;
  cudaMemcpy(&err, p1->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&errc, c->p1->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (cudaGetLastError() != cudaSuccess || err || errc) return -1;
  return 0;
}

void tc_reset_chain(TcChain* c, cudaStream_t st) {
  if (!c) return;
  int nblk = 0;
  for (const TcProb& pr : c->p1->probs_h) nblk += pr.tiles_m;
  cudaMemsetAsync(c->d_ready, 0, sizeof(unsigned long long) * nblk, st);
  cudaMemsetAsync(c->d_epoch, 0, 2 * sizeof(unsigned long long), st);
}

void tc_destroy_chain(TcChain* c) {
  if (!c) return;
  if (c->d_ord) cudaFree(c->d_ord);
  if (c->d_blk0) cudaFree(c->d_blk0);
  if (c->d_ready) cudaFree(c->d_ready);
  if (c->d_epoch) cudaFree(c->d_epoch);
  delete c;
}

}  // namespace vgtb
