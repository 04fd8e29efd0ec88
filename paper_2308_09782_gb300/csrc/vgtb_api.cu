// libvgtb host runtime: the C-ABI of include/vgtb.h.
//
// create():   validate the system, group its real-space blocks into targets
//             (distinct atom pairs) with their images, tabulate the Bloch phases,
//             build S_k (Eq. 7) and S_k^-1 (cuSOLVER Cholesky), and either the SCC
//             ground state (cuSOLVER generalized eigensolver + Anderson-mixed
//             charges, Sec. 3.1) or wait for a user density.
// propagate(): enqueue the step  obs -> scc -> phase -> product 1 -> product 2
//             -> leapfrog  for all trajectories and k-points together, captured
//             into a CUDA graph of `graph_steps` steps and replayed; a device step
//             counter lets every replay run the same graph.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/vgtb.h"
#include "vgtb_internal.h"
#include "vgtb_tc.h"

using namespace vgtb;

namespace {

thread_local std::string g_create_error;

struct HostSys {
  int N = 0, Np = 0, nat = 0, nk = 0, n_blk = 0, n_tgt = 0, nocc = 0;
  double omega = 0, nel = 0, dt = 0;
  std::vector<int> orb_off;
  std::vector<double> z, gamma;
  std::vector<int> tgt_I, tgt_J, tgt_img0, img_blk, atom_tgt0, tgt_el0;
  int n_el = 0;
  std::vector<long long> blk_off;
  std::vector<double> wk;
  // device
  double2* Sinv = nullptr;
  double2* D0 = nullptr;
  double2* R0 = nullptr;
  double* dq0 = nullptr;
  double* eps0 = nullptr;
  __nv_bfloat16* Sinv_p = nullptr;
  __nv_bfloat16* D0_p = nullptr;
  float* R0f = nullptr;
  double2* C0d = nullptr;   // Crank-Nicolson: [nk][nocc][Np] initial states as rows (C^dagger)
  std::vector<double> dq0_h, eps0_h;
  bool density_set = false;
  std::vector<int> trajs;  // trajectories of this system
  std::vector<char> k_set;  // which k-points received a user density
  float2* D0f = nullptr;    // split form, block-sparse first product: [nk][Np][Np] FP32 copy of D0
  int bsr_units = 0;        // block-sparse first product: CTAs per item (groups x column chunks)
  int bsr_tg_max = 0;       // most targets of one atom group
  int bsr_ent_max = 0;      // most column atoms in the union of one atom group
};

struct HostTraj {
  int sys = 0, item0 = 0;
  int n_times = 0;
  double* A = nullptr;
  double* J = nullptr;
  double* E = nullptr;
  double* q = nullptr;
  double* dq = nullptr;
  double* eps = nullptr;
  double* eps_lv = nullptr;
  float* epsf = nullptr;
  float* depsf = nullptr;
  float* af = nullptr;
  double* part = nullptr;
  double* cpart = nullptr;
  double* apart = nullptr;
  int* ticket = nullptr;
  int* status = nullptr;
};

}  // namespace

struct vgtb_ctx {
  vgtb_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<void*> allocs;
  std::vector<HostSys> sys;
  std::vector<HostTraj> trj;
  std::vector<DevItem> items_h;
  DevSys* d_sys = nullptr;
  DevTraj* d_trj = nullptr;
  DevItem* d_items = nullptr;
  int* d_wpre = nullptr;
  int total_warps = 0;
  int max_nat = 0, max_Np = 0, max_nk = 1;
  int* d_step = nullptr;
  int* d_counter = nullptr;
  int n_done = 0;
  bool split = false, delta = false, cn = false;
  // Crank-Nicolson work lists: density, M = S^-1 H, the fixed-point sweeps, the check
  GemmF64Item* d_gD = nullptr;
  GemmF64Item* d_gM = nullptr;
  std::vector<GemmF64Item*> sweep;  // device list of sweep j = 1..cn_iter
  CnCheckItem* d_cnchk = nullptr;
  int max_nocc = 0;
  // FP64 GEMM / leap work lists
  GemmF64Item* d_g1 = nullptr;
  GemmF64Item* d_g2 = nullptr;
  LeapItem* d_leap = nullptr;
  int n_items = 0;
  // tcgen05 plans
  TcPlan* tc1 = nullptr;
  TcPlan* tc2 = nullptr;
  TcChain* tcc = nullptr;  // both products in one launch (null: two launches)
  // block-sparse first product (every atom 4 orbitals; product1 BLOCKS, or AUTO on the FP64 path)
  bool bsr = false;
  BsrItem* d_bsr = nullptr;
  BsrSys* d_bsrsys = nullptr;
  int* d_bsr_u0 = nullptr;   // [n_items+1] first unit of each item
  int* d_bsr_ctr = nullptr;  // [2] unit counter and finished-CTA counter
  int bsr_units_max = 0, bsr_units_total = 0, bsr_tg_max = 0, bsr_ent_max = 0, bsr_grp_max = 0;
  // Crank-Nicolson: D = 2 C C^dagger formed at H's nonzero pattern only for the step's sums
  CnDensItem* d_cnd = nullptr;
  // graph
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  bool graph_profiled = false;
  // profiling
  bool profile = false;
  std::vector<cudaEvent_t> ev;
  long long prof_launch[VGTB_K_COUNT] = {0};
  double prof_ms[VGTB_K_COUNT] = {0};
  cusolverDnHandle_t solver = nullptr;
};

namespace {

int fail(vgtb_ctx* ctx, int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_create_error = buf;
  return code;
}

#define CK(x)                                                                                \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess) {                                                                 \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? VGTB_E_NOMEM : VGTB_E_CUDA,         \
                  "%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                        \
  } while (0)

#define CKS(x)                                                                          \
  do {                                                                                  \
    cusolverStatus_t s_ = (x);                                                          \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                  \
      return fail(ctx, VGTB_E_CUDA, "%s failed: cusolver status %d", #x, (int)s_);      \
  } while (0)

#define TRY(x)            \
  do {                    \
    int r_ = (x);         \
    if (r_ != VGTB_OK) return r_; \
  } while (0)

template <class T>
int dalloc(vgtb_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return VGTB_OK;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess)
    return fail(ctx, VGTB_E_NOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
  ctx->allocs.push_back(q);
  e = cudaMemsetAsync(q, 0, count * sizeof(T), ctx->stream);
  if (e != cudaSuccess) return fail(ctx, VGTB_E_CUDA, "cudaMemset failed: %s", cudaGetErrorString(e));
  *p = (T*)q;
  return VGTB_OK;
}

template <class T>
int upload(vgtb_ctx* ctx, T** p, const T* src, size_t count) {
  TRY(dalloc(ctx, p, count));
  if (count) CK(cudaMemcpyAsync(*p, src, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return VGTB_OK;
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// ---------------------------------------------------------------------------
// validation and target grouping of one system
// ---------------------------------------------------------------------------
int prepare_system(vgtb_ctx* ctx, int si, const vgtb_system& s, HostSys& h, DevSys& d, bool need_ground) {
  if (s.n_atoms < 1 || !s.pos || !s.orb_offset || !s.z_ref || s.n_blocks < 1 || !s.blk_ijl || !s.h0 || !s.s ||
      !s.ds || !s.gamma || s.n_k < 1 || !s.kpt || !s.wk)
    return fail(ctx, VGTB_E_INVALID, "system %d: missing array or empty dimension", si);
  if (!(s.dt > 0.0) || !std::isfinite(s.dt)) return fail(ctx, VGTB_E_INVALID, "system %d: dt must be > 0", si);
  h.nat = s.n_atoms;
  h.orb_off.assign(s.orb_offset, s.orb_offset + s.n_atoms + 1);
  if (h.orb_off[0] != 0) return fail(ctx, VGTB_E_INVALID, "system %d: orb_offset[0] must be 0", si);
  for (int i = 0; i < s.n_atoms; ++i)
    if (h.orb_off[i + 1] <= h.orb_off[i])
      return fail(ctx, VGTB_E_INVALID, "system %d: orb_offset must increase strictly (atom %d)", si, i);
  h.N = h.orb_off[s.n_atoms];
  h.Np = (h.N + 127) / 128 * 128;
  h.nel = s.n_electrons;
  if (!(s.n_electrons > 0.0) || s.n_electrons > 2.0 * h.N || !std::isfinite(s.n_electrons))
    return fail(ctx, VGTB_E_INVALID, "system %d: n_electrons must be in (0, 2N]", si);
  if (need_ground) {
    const double half = 0.5 * s.n_electrons;
    if (std::fabs(half - std::round(half)) > 1e-12)
      return fail(ctx, VGTB_E_INVALID, "system %d: the ground state and the Crank-Nicolson states need an even "
                  "electron count", si);
    h.nocc = (int)std::llround(half);
  }
  h.dt = s.dt;
  const double* L = s.lattice;
  const double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                     L[2] * (L[3] * L[7] - L[4] * L[6]);
  h.omega = std::fabs(det);
  if (!(h.omega > 0.0) || !finite_all(L, 9)) return fail(ctx, VGTB_E_INVALID, "system %d: singular lattice", si);
  if (!finite_all(s.pos, 3 * (size_t)s.n_atoms) || !finite_all(s.z_ref, s.n_atoms))
    return fail(ctx, VGTB_E_INVALID, "system %d: non-finite positions or Z", si);
  // blocks
  h.n_blk = s.n_blocks;
  h.blk_off.resize(s.n_blocks);
  long long tot = 0;
  std::map<std::tuple<int, int, int, int, int>, int> key;
  for (int b = 0; b < s.n_blocks; ++b) {
    const int* r = s.blk_ijl + 5 * b;
    if (r[0] < 0 || r[0] >= s.n_atoms || r[1] < 0 || r[1] >= s.n_atoms)
      return fail(ctx, VGTB_E_INVALID, "system %d: block %d atom index out of range", si, b);
    h.blk_off[b] = tot;
    tot += (long long)(h.orb_off[r[0] + 1] - h.orb_off[r[0]]) * (h.orb_off[r[1] + 1] - h.orb_off[r[1]]);
    if (!key.emplace(std::make_tuple(r[0], r[1], r[2], r[3], r[4]), b).second)
      return fail(ctx, VGTB_E_INVALID, "system %d: duplicate block (%d,%d,%d,%d,%d)", si, r[0], r[1], r[2], r[3], r[4]);
  }
  if (!finite_all(s.h0, tot) || !finite_all(s.s, tot) || !finite_all(s.ds, 3 * tot))
    return fail(ctx, VGTB_E_INVALID, "system %d: non-finite block values", si);
  // mirror blocks: (J, I, -n) with transposed S/H0 and negated transposed dS
  double smax = 0.0;
  for (long long i = 0; i < tot; ++i) smax = std::max(smax, std::fabs(s.s[i]) + std::fabs(s.h0[i]));
  for (int b = 0; b < s.n_blocks; ++b) {
    const int* r = s.blk_ijl + 5 * b;
    auto it = key.find(std::make_tuple(r[1], r[0], -r[2], -r[3], -r[4]));
    if (it == key.end())
      return fail(ctx, VGTB_E_INVALID, "system %d: block (%d,%d,%d,%d,%d) has no mirror block", si, r[0], r[1], r[2],
                  r[3], r[4]);
    const int m = it->second;
    const int ni = h.orb_off[r[0] + 1] - h.orb_off[r[0]], nj = h.orb_off[r[1] + 1] - h.orb_off[r[1]];
    for (int a = 0; a < ni; ++a)
      for (int c = 0; c < nj; ++c) {
        const long long e1 = h.blk_off[b] + a * nj + c, e2 = h.blk_off[m] + c * ni + a;
        const double tol = 1e-12 * std::max(1.0, smax);
        bool bad = std::fabs(s.s[e1] - s.s[e2]) > tol || std::fabs(s.h0[e1] - s.h0[e2]) > tol;
        for (int x = 0; x < 3; ++x) bad |= std::fabs(s.ds[x * tot + e1] + s.ds[x * tot + e2]) > tol;
        if (bad)
          return fail(ctx, VGTB_E_INVALID, "system %d: block %d and its mirror are not Hermitian partners", si, b);
      }
  }
  // gamma
  h.gamma.assign(s.gamma, s.gamma + (size_t)s.n_atoms * s.n_atoms);
  if (!finite_all(h.gamma.data(), h.gamma.size())) return fail(ctx, VGTB_E_INVALID, "system %d: non-finite gamma", si);
  double gmax = 0.0;
  for (double g : h.gamma) gmax = std::max(gmax, std::fabs(g));
  for (int i = 0; i < s.n_atoms; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(h.gamma[(size_t)i * s.n_atoms + j] - h.gamma[(size_t)j * s.n_atoms + i]) > 1e-12 * std::max(1.0, gmax))
        return fail(ctx, VGTB_E_INVALID, "system %d: gamma is not symmetric", si);
  // k points
  h.nk = s.n_k;
  if (!finite_all(s.kpt, 3 * (size_t)s.n_k) || !finite_all(s.wk, s.n_k))
    return fail(ctx, VGTB_E_INVALID, "system %d: non-finite k-points", si);
  h.wk.assign(s.wk, s.wk + s.n_k);
  double wsum = 0.0;
  for (double w : h.wk) wsum += w;
  if (std::fabs(wsum - 1.0) > 1e-10) return fail(ctx, VGTB_E_INVALID, "system %d: k weights sum to %.15g", si, wsum);
  h.z.assign(s.z_ref, s.z_ref + s.n_atoms);
  // targets: distinct (I, J) sorted by I then J; images in (n1, n2, n3) order
  std::vector<int> order(s.n_blocks);
  for (int b = 0; b < s.n_blocks; ++b) order[b] = b;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const int* x = s.blk_ijl + 5 * a;
    const int* y = s.blk_ijl + 5 * b;
    return std::lexicographical_compare(x, x + 5, y, y + 5);
  });
  h.tgt_I.clear();
  h.tgt_J.clear();
  h.tgt_img0.clear();
  h.img_blk.clear();
  for (int idx = 0; idx < s.n_blocks; ++idx) {
    const int b = order[idx];
    const int* r = s.blk_ijl + 5 * b;
    if (h.tgt_I.empty() || h.tgt_I.back() != r[0] || h.tgt_J.back() != r[1]) {
      h.tgt_I.push_back(r[0]);
      h.tgt_J.push_back(r[1]);
      h.tgt_img0.push_back((int)h.img_blk.size());
    }
    h.img_blk.push_back(b);
  }
  h.tgt_img0.push_back((int)h.img_blk.size());
  h.n_tgt = (int)h.tgt_I.size();
  h.tgt_el0.assign(h.n_tgt + 1, 0);
  for (int tg = 0; tg < h.n_tgt; ++tg)
    h.tgt_el0[tg + 1] = h.tgt_el0[tg] + (h.orb_off[h.tgt_I[tg] + 1] - h.orb_off[h.tgt_I[tg]]) *
                                             (h.orb_off[h.tgt_J[tg] + 1] - h.orb_off[h.tgt_J[tg]]);
  h.n_el = h.tgt_el0[h.n_tgt];
  h.atom_tgt0.assign(s.n_atoms + 1, 0);
  for (int t = 0; t < h.n_tgt; ++t) h.atom_tgt0[h.tgt_I[t] + 1]++;
  for (int i = 0; i < s.n_atoms; ++i) h.atom_tgt0[i + 1] += h.atom_tgt0[i];
  // phases e^{-i 2 pi k.n}
  std::vector<double2> ph((size_t)s.n_k * s.n_blocks);
  for (int k = 0; k < s.n_k; ++k)
    for (int b = 0; b < s.n_blocks; ++b) {
      const int* r = s.blk_ijl + 5 * b;
      const double th = 2.0 * M_PI * (s.kpt[3 * k] * r[2] + s.kpt[3 * k + 1] * r[3] + s.kpt[3 * k + 2] * r[4]);
      ph[(size_t)k * s.n_blocks + b] = make_double2(std::cos(th), -std::sin(th));
    }
  // upload
  memset(&d, 0, sizeof(d));
  d.N = h.N;
  d.Np = h.Np;
  d.scc_frozen = ctx->opt.scc == VGTB_SCC_FROZEN ? 1 : 0;
  d.nat = h.nat;
  d.nk = h.nk;
  d.n_tgt = h.n_tgt;
  d.n_blk = h.n_blk;
  d.omega = h.omega;
  d.inv_omega = 1.0 / h.omega;
  d.nel = h.nel;
  d.dt = h.dt;
  int* pi;
  double* pd;
  long long* pl;
  double2* pz;
  TRY(upload(ctx, &pi, h.orb_off.data(), h.orb_off.size()));
  d.orb_off = pi;
  TRY(upload(ctx, &pd, h.z.data(), h.z.size()));
  d.z = pd;
  TRY(upload(ctx, &pd, h.gamma.data(), h.gamma.size()));
  d.gamma = pd;
  TRY(upload(ctx, &pi, h.tgt_I.data(), h.tgt_I.size()));
  d.tgt_I = pi;
  TRY(upload(ctx, &pi, h.tgt_J.data(), h.tgt_J.size()));
  d.tgt_J = pi;
  TRY(upload(ctx, &pi, h.tgt_img0.data(), h.tgt_img0.size()));
  d.tgt_img0 = pi;
  TRY(upload(ctx, &pi, h.img_blk.data(), h.img_blk.size()));
  d.img_blk = pi;
  {
    std::vector<long long> io(h.img_blk.size());
    for (size_t g = 0; g < io.size(); ++g) io[g] = h.blk_off[h.img_blk[g]];
    TRY(upload(ctx, &pl, io.data(), io.size()));
    d.img_off = pl;
  }
  TRY(upload(ctx, &pl, h.blk_off.data(), h.blk_off.size()));
  d.blk_off = pl;
  TRY(upload(ctx, &pd, s.h0, (size_t)tot));
  d.h0 = pd;
  TRY(upload(ctx, &pd, s.s, (size_t)tot));
  d.s = pd;
  TRY(upload(ctx, &pd, s.ds, 3 * (size_t)tot));
  d.ds = pd;
  d.ds_stride = tot;
  TRY(upload(ctx, &pz, ph.data(), ph.size()));
  d.phase = pz;
  if (ctx->split) {
    // FP32 copies for the split form's phase build
    std::vector<float> f(3 * (size_t)tot);
    float* pf;
    for (long long i = 0; i < tot; ++i) f[i] = (float)s.h0[i];
    TRY(upload(ctx, &pf, f.data(), (size_t)tot));
    d.h0f = pf;
    for (long long i = 0; i < tot; ++i) f[i] = (float)s.s[i];
    TRY(upload(ctx, &pf, f.data(), (size_t)tot));
    d.sf = pf;
    for (long long i = 0; i < 3 * tot; ++i) f[i] = (float)s.ds[i];
    TRY(upload(ctx, &pf, f.data(), 3 * (size_t)tot));
    d.dsf = pf;
    std::vector<float2> pff(ph.size());
    for (size_t i = 0; i < ph.size(); ++i) pff[i] = make_float2((float)ph[i].x, (float)ph[i].y);
    float2* pf2;
    TRY(upload(ctx, &pf2, pff.data(), pff.size()));
    d.phasef = pf2;
  }
  TRY(upload(ctx, &pd, h.wk.data(), h.wk.size()));
  d.wk = pd;
  TRY(upload(ctx, &pi, h.atom_tgt0.data(), h.atom_tgt0.size()));
  d.atom_tgt0 = pi;
  TRY(upload(ctx, &pi, h.tgt_el0.data(), h.tgt_el0.size()));
  d.tgt_el0 = pi;
  {
    // vector phase build: 4 columns, column offset and every image's values 16-byte aligned
    std::vector<int> vec(h.n_tgt, 0);
    for (int tg = 0; tg < h.n_tgt; ++tg) {
      const int J = h.tgt_J[tg];
      bool ok = (h.orb_off[J + 1] - h.orb_off[J]) == 4 && (h.orb_off[J] % 4) == 0 && (tot % 4) == 0;
      for (int g = h.tgt_img0[tg]; ok && g < h.tgt_img0[tg + 1]; ++g) ok = (h.blk_off[h.img_blk[g]] % 4) == 0;
      vec[tg] = ok ? 1 : 0;
    }
    TRY(upload(ctx, &pi, vec.data(), vec.size()));
    d.tgt_vec = pi;
    if (ctx->split) {
      std::vector<int4> p0(h.n_tgt), p1(h.n_tgt);
      for (int tg = 0; tg < h.n_tgt; ++tg) {
        const int I = h.tgt_I[tg], J = h.tgt_J[tg];
        p0[tg] = make_int4(I, J, h.tgt_img0[tg], h.tgt_img0[tg + 1]);
        p1[tg] = make_int4(h.orb_off[I], h.orb_off[J], (h.orb_off[I + 1] - h.orb_off[I]) | (vec[tg] << 16),
                           h.orb_off[J + 1] - h.orb_off[J]);
      }
      int4* p4;
      TRY(upload(ctx, &p4, p0.data(), p0.size()));
      d.tgt_p0 = p4;
      TRY(upload(ctx, &p4, p1.data(), p1.size()));
      d.tgt_p1 = p4;
      const int n_img = (int)h.img_blk.size();
      std::vector<float2> pim((size_t)h.nk * n_img);
      for (int k = 0; k < h.nk; ++k)
        for (int g = 0; g < n_img; ++g) {
          const double2 v = ph[(size_t)k * s.n_blocks + h.img_blk[g]];
          pim[(size_t)k * n_img + g] = make_float2((float)v.x, (float)v.y);
        }
      float2* pf2;
      TRY(upload(ctx, &pf2, pim.data(), pim.size()));
      d.phase_img = pf2;
      d.n_img = n_img;
    }
    // element offsets of the nonzeros (row-major within each target) and per-atom ranges
    if ((long long)h.Np * h.Np > 2147483647LL) return fail(ctx, VGTB_E_INVALID, "system %d: Np too large", si);
    std::vector<int> eoff(h.n_el), eat(h.nat + 1);
    for (int tg = 0; tg < h.n_tgt; ++tg) {
      const int oi = h.orb_off[h.tgt_I[tg]], oj = h.orb_off[h.tgt_J[tg]];
      const int nj = h.orb_off[h.tgt_J[tg] + 1] - oj;
      for (int e = h.tgt_el0[tg]; e < h.tgt_el0[tg + 1]; ++e) {
        const int a = (e - h.tgt_el0[tg]) / nj, b = (e - h.tgt_el0[tg]) % nj;
        eoff[e] = (oi + a) * h.Np + oj + b;
      }
    }
    for (int i = 0; i <= h.nat; ++i) eat[i] = h.tgt_el0[h.atom_tgt0[i]];
    TRY(upload(ctx, &pi, eoff.data(), eoff.size()));
    d.el_off = pi;
    TRY(upload(ctx, &pi, eat.data(), eat.size()));
    d.el_atom0 = pi;
  }
  d.n_el = h.n_el;
  TRY(dalloc(ctx, &d.kS, (size_t)h.nk * h.n_el));
  TRY(dalloc(ctx, &d.kH0, (size_t)h.nk * h.n_el));
  TRY(dalloc(ctx, &d.kP, 3 * (size_t)h.nk * h.n_el));
  TRY(dalloc(ctx, &d.obs0, 5 * (size_t)h.n_tgt));
  if (ctx->split) TRY(dalloc(ctx, &d.obs0a, 5 * (size_t)h.nat));
  const size_t NN = (size_t)h.Np * h.Np;
  TRY(dalloc(ctx, &h.Sinv, NN * h.nk));
  TRY(dalloc(ctx, &h.D0, NN * h.nk));
  TRY(dalloc(ctx, &h.dq0, h.nat));
  TRY(dalloc(ctx, &h.eps0, h.nat));
  if (ctx->delta) TRY(dalloc(ctx, &h.R0, NN * h.nk));
  if (ctx->cn) TRY(dalloc(ctx, &h.C0d, (size_t)h.nk * h.nocc * h.Np));
  if (ctx->split) {
    TRY(dalloc(ctx, &h.Sinv_p, 4 * NN * h.nk));
    TRY(dalloc(ctx, &h.D0_p, 4 * NN * h.nk));
    TRY(dalloc(ctx, &h.R0f, 2 * NN * h.nk));
  }
  d.Sinv = h.Sinv;
  d.D0 = h.D0;
  d.R0 = h.R0;
  d.dq0 = h.dq0;
  d.eps0 = h.eps0;
  d.Sinv_p = h.Sinv_p;
  d.D0_p = h.D0_p;
  d.R0f = h.R0f;
  return VGTB_OK;
}

// ---------------------------------------------------------------------------
// S_k^-1 by Cholesky (cuSOLVER).  A row-major Hermitian buffer read as
// column-major is conj(S); potrf/potri of conj(S) give conj(S^-1), whose
// row-major reading is S^-1 again (upper triangle valid, then mirrored).
// ---------------------------------------------------------------------------
int build_sinv(vgtb_ctx* ctx, int si) {
  HostSys& h = ctx->sys[si];
  const size_t NN = (size_t)h.Np * h.Np;
  for (int k = 0; k < h.nk; ++k) launch_kblocks(ctx->d_sys, si, h.n_tgt, k, ctx->stream);
  int* info = nullptr;
  TRY(dalloc(ctx, &info, 1));
  for (int k = 0; k < h.nk; ++k) {
    double2* S = h.Sinv + k * NN;
    launch_bloch_setup(ctx->d_sys, si, h.n_tgt, k, 0, nullptr, S, ctx->stream);
    CK(cudaGetLastError());
    int lw = 0;
    CKS(cusolverDnZpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_LOWER, h.N, (cuDoubleComplex*)S, h.Np, &lw));
    int lw2 = 0;
    CKS(cusolverDnZpotri_bufferSize(ctx->solver, CUBLAS_FILL_MODE_LOWER, h.N, (cuDoubleComplex*)S, h.Np, &lw2));
    lw = std::max(lw, lw2);
    cuDoubleComplex* work = nullptr;
    CK(cudaMalloc(&work, sizeof(cuDoubleComplex) * std::max(lw, 1)));
    cusolverStatus_t st = cusolverDnZpotrf(ctx->solver, CUBLAS_FILL_MODE_LOWER, h.N, (cuDoubleComplex*)S, h.Np, work, lw, info);
    int hinfo = 0;
    cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (st != CUSOLVER_STATUS_SUCCESS || hinfo != 0) {
      cudaFree(work);
      if (hinfo > 0) return fail(ctx, VGTB_E_NOT_PD, "system %d: S_k at k=%d is not positive definite (minor %d)", si, k, hinfo);
      return fail(ctx, VGTB_E_CUDA, "cusolverDnZpotrf failed: status %d info %d", (int)st, hinfo);
    }
    st = cusolverDnZpotri(ctx->solver, CUBLAS_FILL_MODE_LOWER, h.N, (cuDoubleComplex*)S, h.Np, work, lw, info);
    cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(work);
    if (st != CUSOLVER_STATUS_SUCCESS || hinfo != 0)
      return fail(ctx, VGTB_E_CUDA, "cusolverDnZpotri failed: status %d info %d", (int)st, hinfo);
    // column-major lower = row-major upper is valid; mirror it
    launch_fill_hermitian_lower(S, h.N, h.Np, ctx->stream);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

// charges of a density set D (nk x Np^2) of system si: q_I on the host
// ---------------------------------------------------------------------------
// Block-sparse first product: groups of G consecutive atoms; for each group the
// union of the column atoms K of its targets (J, K), and for every member J the
// index of target (J, K) relative to the group's first target (-1 if none).
// The group's targets are contiguous because targets are sorted by row atom.
// ---------------------------------------------------------------------------
bool bsr_possible(const HostSys& h) {
  for (int i = 0; i < h.nat; ++i)
    if (h.orb_off[i + 1] - h.orb_off[i] != 4) return false;
  return true;
}

int build_bsr_tables(vgtb_ctx* ctx, HostSys& h, int fp64, BsrSys& b) {
  const int G = bsr_group(fp64);
  const int n_grp = (h.nat + G - 1) / G;
  std::vector<int> grp_t0(n_grp + 1), grp_e0(n_grp + 1, 0), ent_K;
  std::vector<short> ent_slot, tgt_ent(h.n_tgt, 0);
  int tg_max = 0;
  for (int g = 0; g < n_grp; ++g) {
    const int J0 = g * G, J1 = std::min(h.nat, J0 + G);
    const int t0 = h.atom_tgt0[J0], t1 = h.atom_tgt0[J1];
    grp_t0[g] = t0;
    tg_max = std::max(tg_max, t1 - t0);
    if (t1 - t0 > 32767) return fail(ctx, VGTB_E_UNSUPPORTED, "atom group with %d targets", t1 - t0);
    std::map<int, std::vector<short>> uni;  // column atom -> slots of the members
    for (int J = J0; J < J1; ++J)
      for (int t = h.atom_tgt0[J]; t < h.atom_tgt0[J + 1]; ++t) {
        auto& v = uni[h.tgt_J[t]];
        if (v.empty()) v.assign(G, (short)-1);
        v[J - J0] = (short)(t - t0);
      }
    for (auto& kv : uni) {
      for (int j = 0; j < G; ++j)
        if (kv.second[j] >= 0) tgt_ent[t0 + kv.second[j]] = (short)(1024 * j + (int)(ent_K.size() - grp_e0[g]));
      ent_K.push_back(kv.first);
      ent_slot.insert(ent_slot.end(), kv.second.begin(), kv.second.end());
    }
    grp_e0[g + 1] = (int)ent_K.size();
    if (grp_e0[g + 1] - grp_e0[g] > 1023) return fail(ctx, VGTB_E_UNSUPPORTED, "atom group with over 1023 partners");
    h.bsr_ent_max = std::max(h.bsr_ent_max, grp_e0[g + 1] - grp_e0[g]);
  }
  grp_t0[n_grp] = h.atom_tgt0[h.nat];
  memset(&b, 0, sizeof(b));
  b.Np = h.Np;
  b.nat = h.nat;
  b.n_grp = n_grp;
  int* pi;
  TRY(upload(ctx, &pi, grp_t0.data(), grp_t0.size()));
  b.grp_t0 = pi;
  TRY(upload(ctx, &pi, grp_e0.data(), grp_e0.size()));
  b.grp_e0 = pi;
  TRY(upload(ctx, &pi, ent_K.data(), ent_K.size()));
  b.ent_K = pi;
  short* ps;
  TRY(upload(ctx, &ps, ent_slot.data(), ent_slot.size()));
  b.ent_slot = ps;
  TRY(upload(ctx, &ps, tgt_ent.data(), tgt_ent.size()));
  b.tgt_ent = ps;
  h.bsr_units = bsr_units(fp64, n_grp, h.Np);
  h.bsr_tg_max = tg_max;
  return VGTB_OK;
}

int host_charges(vgtb_ctx* ctx, int si, const double2* D, std::vector<double>& q) {
  HostSys& h = ctx->sys[si];
  double* part = nullptr;
  TRY(dalloc(ctx, &part, h.n_tgt));
  launch_mulliken_setup(ctx->d_sys, si, h.n_tgt, D, part, ctx->stream);
  CK(cudaGetLastError());
  std::vector<double> p(h.n_tgt);
  CK(cudaMemcpyAsync(p.data(), part, sizeof(double) * h.n_tgt, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  q.assign(h.nat, 0.0);
  for (int i = 0; i < h.nat; ++i)
    for (int t = h.atom_tgt0[i]; t < h.atom_tgt0[i + 1]; ++t) q[i] += p[t];
  return VGTB_OK;
}

void gamma_mul(const HostSys& h, const std::vector<double>& dq, std::vector<double>& eps) {
  eps.assign(h.nat, 0.0);
  for (int i = 0; i < h.nat; ++i) {
    double e = 0.0;
    for (int j = 0; j < h.nat; ++j) e += h.gamma[(size_t)i * h.nat + j] * dq[j];
    eps[i] = e;
  }
}

// small dense solve (Gaussian elimination with partial pivoting), n <= 16
bool solve_small(std::vector<double> a, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[p * n + c])) p = r;
    if (std::fabs(a[p * n + c]) < 1e-300) return false;
    for (int j = 0; j < n; ++j) std::swap(a[c * n + j], a[p * n + j]);
    std::swap(b[c], b[p]);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[r * n + c] / a[c * n + c];
      for (int j = 0; j < n; ++j) a[r * n + j] -= f * a[c * n + j];
      b[r] -= f * b[c];
    }
  }
  for (int c = 0; c < n; ++c) b[c] /= a[c * n + c];
  return true;
}

// ---------------------------------------------------------------------------
// SCC ground state (Sec. 3.1): diagonalise H_k[dq] C = S_k C e at every k,
// occupy the lowest N_el/2 states twice, recompute dq; Pulay (DIIS) mixing
// of dq on the host until max |dq_out - dq_in| < tol.
// ---------------------------------------------------------------------------
int ground_state(vgtb_ctx* ctx, int si) {
  HostSys& h = ctx->sys[si];
  const size_t NN = (size_t)h.Np * h.Np;
  double2 *Hb = nullptr, *Sb = nullptr, *Vt = nullptr;
  double* w = nullptr;
  double* eps_d = nullptr;
  int* info = nullptr;
  TRY(dalloc(ctx, &Hb, NN));
  TRY(dalloc(ctx, &Sb, NN));
  TRY(dalloc(ctx, &Vt, (size_t)h.N * std::max(h.nocc, 1)));
  TRY(dalloc(ctx, &w, h.Np));
  TRY(dalloc(ctx, &eps_d, h.nat));
  TRY(dalloc(ctx, &info, 1));
  GemmF64Item gi{};
  GemmF64Item* d_gi = nullptr;
  TRY(dalloc(ctx, &d_gi, 1));
  int lw = 0;
  CKS(cusolverDnZhegvd_bufferSize(ctx->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                  h.N, (cuDoubleComplex*)Hb, h.Np, (cuDoubleComplex*)Sb, h.Np, w, &lw));
  cuDoubleComplex* work = nullptr;
  TRY(dalloc(ctx, &work, std::max(lw, 1)));
  const double tol = ctx->opt.scc_tol > 0 ? ctx->opt.scc_tol : 1e-11;
  const int max_it = ctx->opt.scc_max_iter > 0 ? ctx->opt.scc_max_iter : 200;
  const double mix = 0.2;
  const int hist = 8;
  std::vector<double> dq(h.nat, 0.0), eps, q, res;
  std::vector<std::vector<double>> xs, fs;
  bool any_gamma = false;
  for (double g : h.gamma) any_gamma |= (g != 0.0);
  std::vector<double> ev(h.N);
  for (int it = 1; it <= max_it; ++it) {
    gamma_mul(h, dq, eps);
    CK(cudaMemcpyAsync(eps_d, eps.data(), sizeof(double) * h.nat, cudaMemcpyHostToDevice, ctx->stream));
    for (int k = 0; k < h.nk; ++k) {
      CK(cudaMemsetAsync(Hb, 0, NN * sizeof(double2), ctx->stream));
      CK(cudaMemsetAsync(Sb, 0, NN * sizeof(double2), ctx->stream));
      launch_bloch_setup(ctx->d_sys, si, h.n_tgt, k, 1, eps_d, Hb, ctx->stream);
      launch_bloch_setup(ctx->d_sys, si, h.n_tgt, k, 0, nullptr, Sb, ctx->stream);
      CK(cudaGetLastError());
      CKS(cusolverDnZhegvd(ctx->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, h.N,
                           (cuDoubleComplex*)Hb, h.Np, (cuDoubleComplex*)Sb, h.Np, w, work, lw, info));
      int hinfo = 0;
      CK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(ev.data(), w, sizeof(double) * h.N, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if (hinfo > h.N) return fail(ctx, VGTB_E_NOT_PD, "system %d: S_k at k=%d is not positive definite", si, k);
      if (hinfo != 0) return fail(ctx, VGTB_E_CUDA, "cusolverDnZhegvd info %d", hinfo);
      if (h.nocc < h.N && ev[h.nocc] - ev[h.nocc - 1] < 1e-8)
        return fail(ctx, VGTB_E_NO_GAP, "system %d: no gap at N_el/2 at k=%d (%.3e Ha)", si, k, ev[h.nocc] - ev[h.nocc - 1]);
      // Crank-Nicolson keeps the occupied states: row n of the solver output is
      // conj(C_n), i.e. the rows of C^dagger
      if (ctx->cn)
        CK(cudaMemcpy2DAsync(h.C0d + (size_t)k * h.nocc * h.Np, sizeof(double2) * h.Np, Hb, sizeof(double2) * h.Np,
                             sizeof(double2) * h.N, h.nocc, cudaMemcpyDeviceToDevice, ctx->stream));
      // D_k = 2 V V^dagger over the occupied eigenvectors
      launch_vt_from_evecs(Hb, Vt, h.N, h.nocc, h.Np, ctx->stream);
      gi.A[0] = Vt;
      gi.R[0] = Vt;
      gi.a_par[0] = 0;
      gi.C = h.D0 + k * NN;
      gi.K[0] = h.nocc;
      gi.lda[0] = gi.ldr[0] = h.nocc;
      gi.nseg = 1;
      gi.M = gi.N = h.N;
      gi.ldc = h.Np;
      CK(cudaMemcpyAsync(d_gi, &gi, sizeof(gi), cudaMemcpyHostToDevice, ctx->stream));
      launch_gemm_f64(d_gi, 1, h.N, h.N, nullptr, ctx->stream);
      launch_scale(h.D0 + k * NN, (long long)NN, 2.0, ctx->stream);
      CK(cudaGetLastError());
    }
    TRY(host_charges(ctx, si, h.D0, q));
    res.assign(h.nat, 0.0);
    double rmax = 0.0;
    for (int i = 0; i < h.nat; ++i) {
      res[i] = (q[i] - h.z[i]) - dq[i];
      rmax = std::max(rmax, std::fabs(res[i]));
    }
    if (rmax < tol || !any_gamma) return VGTB_OK;
    xs.push_back(dq);
    fs.push_back(res);
    if ((int)xs.size() > hist) {
      xs.erase(xs.begin());
      fs.erase(fs.begin());
    }
    const int m = (int)fs.size();
    std::vector<double> nx(h.nat, 0.0);
    if (m == 1) {
      for (int i = 0; i < h.nat; ++i) nx[i] = dq[i] + mix * res[i];
    } else {
      // minimise |sum c_j f_j| with sum c_j = 1 (Lagrange system of size m+1)
      std::vector<double> a((m + 1) * (m + 1), 0.0), b(m + 1, 0.0);
      for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) {
          double s = 0.0;
          for (int i = 0; i < h.nat; ++i) s += fs[r][i] * fs[c][i];
          a[r * (m + 1) + c] = s;
        }
      for (int r = 0; r < m; ++r) {
        a[r * (m + 1) + m] = 1.0;
        a[m * (m + 1) + r] = 1.0;
      }
      b[m] = 1.0;
      if (!solve_small(a, b, m + 1)) {
        for (int i = 0; i < h.nat; ++i) nx[i] = dq[i] + mix * res[i];
      } else {
        for (int j = 0; j < m; ++j)
          for (int i = 0; i < h.nat; ++i) nx[i] += b[j] * (xs[j][i] + mix * fs[j][i]);
      }
    }
    dq.swap(nx);
  }
  return fail(ctx, VGTB_E_NO_CONVERGE, "system %d: SCC ground state not converged in %d iterations", si, max_it);
}

// After D0 is set: charges of D0, eps0, R0 (delta forms), split pieces, and
// every trajectory of the system back to step 0.
int finish_density(vgtb_ctx* ctx, int si) {
  HostSys& h = ctx->sys[si];
  const size_t NN = (size_t)h.Np * h.Np;
  for (int k = 0; k < h.nk; ++k) launch_hermitize(h.D0 + k * NN, h.N, h.Np, ctx->stream);
  if (ctx->delta) launch_obs0(ctx->d_sys, si, h.n_tgt, h.nat, ctx->split ? 1 : 0, ctx->stream);
  CK(cudaGetLastError());
  std::vector<double> q;
  TRY(host_charges(ctx, si, h.D0, q));
  h.dq0_h.assign(h.nat, 0.0);
  for (int i = 0; i < h.nat; ++i) h.dq0_h[i] = q[i] - h.z[i];
  gamma_mul(h, h.dq0_h, h.eps0_h);
  CK(cudaMemcpyAsync(h.dq0, h.dq0_h.data(), sizeof(double) * h.nat, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(h.eps0, h.eps0_h.data(), sizeof(double) * h.nat, cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->delta) {
    // R0 = -i(S^-1 H_ref D0 - h.c.) with H_ref = H(A = 0, eps0), all in FP64
    double2 *Hb = nullptr, *Wb = nullptr, *Xb = nullptr;
    TRY(dalloc(ctx, &Hb, NN));
    TRY(dalloc(ctx, &Wb, NN));
    TRY(dalloc(ctx, &Xb, NN));
    double* eps_d = h.eps0;
    GemmF64Item g[2] = {};
    GemmF64Item* dg = nullptr;
    LeapItem li{};
    LeapItem* dl = nullptr;
    TRY(dalloc(ctx, &dg, 2));
    TRY(dalloc(ctx, &dl, 1));
    for (int k = 0; k < h.nk; ++k) {
      CK(cudaMemsetAsync(Hb, 0, NN * sizeof(double2), ctx->stream));
      launch_bloch_setup(ctx->d_sys, si, h.n_tgt, k, 1, eps_d, Hb, ctx->stream);
      g[0] = GemmF64Item{};
      g[0].A[0] = h.D0 + k * NN;
      g[0].R[0] = Hb;
      g[0].K[0] = h.Np;
      g[0].lda[0] = g[0].ldr[0] = h.Np;
      g[0].nseg = 1;
      g[0].M = g[0].N = g[0].ldc = h.Np;
      g[0].C = Wb;
      g[1] = g[0];
      g[1].A[0] = h.Sinv + k * NN;
      g[1].R[0] = Wb;
      g[1].C = Xb;
      CK(cudaMemcpyAsync(dg, g, sizeof(g), cudaMemcpyHostToDevice, ctx->stream));
      launch_gemm_f64(dg, 1, h.Np, h.Np, nullptr, ctx->stream);
      launch_gemm_f64(dg + 1, 1, h.Np, h.Np, nullptr, ctx->stream);
      li = LeapItem{};
      li.X = Xb;
      li.Np = h.Np;
      li.mode = 1;
      li.out = h.R0 + k * NN;
      CK(cudaMemcpyAsync(dl, &li, sizeof(li), cudaMemcpyHostToDevice, ctx->stream));
      launch_leap(dl, 1, h.Np, 0, nullptr, 0.0, nullptr, nullptr, ctx->stream);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(ctx->stream));
    }
  }
  if (ctx->split) {
    for (int k = 0; k < h.nk; ++k) {
      if (h.D0f) launch_to_f32(h.D0 + k * NN, h.D0f + k * NN, (long long)NN, ctx->stream);
      if (h.D0_p) launch_split_planar(h.D0 + k * NN, h.D0_p + 4 * NN * k, h.N, h.Np, ctx->stream);
      launch_split_planar(h.Sinv + k * NN, h.Sinv_p + 4 * NN * k, h.N, h.Np, ctx->stream);
      launch_to_planar_f32(h.R0 + k * NN, h.R0f + 2 * NN * k, h.Np, ctx->stream);
    }
    CK(cudaGetLastError());
  }
  h.density_set = true;
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

// Reset every trajectory to step 0 (D = D0, or dD = 0 in the delta forms).
int reset_all(vgtb_ctx* ctx) {
  for (auto& it : ctx->items_h) {
    const HostSys& h = ctx->sys[it.sys];
    const size_t NN = (size_t)h.Np * h.Np;
    if (ctx->delta)
      CK(cudaMemsetAsync(it.D[0], 0, NN * sizeof(double2), ctx->stream));
    else
      CK(cudaMemcpyAsync(it.D[0], h.D0 + it.k * NN, NN * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
    if (ctx->cn)
      CK(cudaMemcpyAsync(it.Cd, h.C0d + (size_t)it.k * h.nocc * h.Np, (size_t)h.nocc * h.Np * sizeof(double2),
                         cudaMemcpyDeviceToDevice, ctx->stream));
    if (it.dD_p) CK(cudaMemsetAsync(it.dD_p, 0, 4 * NN * sizeof(__nv_bfloat16), ctx->stream));
    if (it.dDf) CK(cudaMemsetAsync(it.dDf, 0, NN * sizeof(float2), ctx->stream));
  }
  for (auto& t : ctx->trj) CK(cudaMemsetAsync(t.status, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_step, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), ctx->stream));
  ctx->n_done = 0;
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

int upload_traj_table(vgtb_ctx* ctx) {
  std::vector<DevTraj> dt(ctx->trj.size());
  for (size_t t = 0; t < ctx->trj.size(); ++t) {
    const HostTraj& h = ctx->trj[t];
    DevTraj& d = dt[t];
    memset(&d, 0, sizeof(d));
    d.sys = h.sys;
    d.item0 = h.item0;
    d.n_times = h.n_times;
    d.A = h.A;
    d.J = h.J;
    d.E = h.E;
    d.q = h.q;
    d.dq = h.dq;
    d.eps = h.eps;
    d.eps_lv = h.eps_lv;
    d.epsf = h.epsf;
    d.depsf = h.depsf;
    d.af = h.af;
    d.part = h.part;
    d.cpart = h.cpart;
    d.apart = h.apart;
    d.ticket = h.ticket;
    d.status = h.status;
  }
  CK(cudaMemcpyAsync(ctx->d_trj, dt.data(), sizeof(DevTraj) * dt.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

void drop_graph(vgtb_ctx* ctx) {
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  ctx->graph = nullptr;
}

// ---------------------------------------------------------------------------
// one step for every trajectory; ev != nullptr records 7 timing events (as
// external event nodes when the stream is being captured into a graph)
// ---------------------------------------------------------------------------
// Work lists of the Crank-Nicolson step.  With Y_0 = C, sweep j = 1..m-1
// writes Y_j = C + i (dt/2) Y_{j-1} M^dagger (in the dagger layout) into
// Y[j & 1]; sweep m writes 2 Y_m - C = C + i dt Y_{m-1} M^dagger over C in place.
int build_cn_lists(vgtb_ctx* ctx) {
  const int m = ctx->opt.cn_iter, n = ctx->n_items;
  const double theta = 0.5 * ctx->sys[0].dt;
  std::vector<GemmF64Item> gD(n), gM(n);
  std::vector<std::vector<GemmF64Item>> gs(m, std::vector<GemmF64Item>(n));
  std::vector<CnCheckItem> ck(n);
  for (int i = 0; i < n; ++i) {
    const DevItem& it = ctx->items_h[i];
    const HostSys& h = ctx->sys[it.sys];
    const size_t NN = (size_t)h.Np * h.Np;
    GemmF64Item d{};  // D = 2 C C^dagger: both operands are read as conj-transposed rows of C^dagger
    d.A[0] = it.Cd;
    d.R[0] = it.Cd;
    d.K[0] = h.nocc;
    d.lda[0] = d.ldr[0] = h.Np;
    d.nseg = 1;
    d.conj_t = 3;
    d.M = d.N = d.ldc = h.Np;
    d.C = it.D[0];
    d.epi = 1;
    d.coef = make_double2(2.0, 0.0);
    gD[i] = d;
    GemmF64Item mm{};  // M = S^-1 H = S^-1 (H^dagger)
    mm.A[0] = h.Sinv + it.k * NN;
    mm.R[0] = it.H;
    mm.K[0] = h.Np;
    mm.lda[0] = mm.ldr[0] = h.Np;
    mm.nseg = 1;
    mm.M = mm.N = mm.ldc = h.Np;
    mm.C = it.W;
    gM[i] = mm;
    for (int j = 1; j <= m; ++j) {
      GemmF64Item s{};  // out = C^dagger + coef (Y^dagger M^dagger)
      s.A[0] = (j == 1) ? it.Cd : it.Y[(j - 1) & 1];
      s.R[0] = it.W;
      s.K[0] = h.Np;
      s.lda[0] = s.ldr[0] = h.Np;
      s.nseg = 1;
      s.M = h.nocc;
      s.N = h.Np;
      s.ldc = h.Np;
      s.epi = 1;
      s.base = it.Cd;
      s.ldb = h.Np;
      s.coef = make_double2(0.0, j == m ? 2.0 * theta : theta);
      s.C = (j == m) ? it.Cd : it.Y[j & 1];
      gs[j - 1][i] = s;
    }
    CnCheckItem c{};
    c.a = it.Y[(m - 1) & 1];
    c.b = it.Y[(m - 2) & 1];
    c.rows = h.nocc;
    c.cols = h.N;
    c.ld = h.Np;
    c.traj = it.traj;
    ck[i] = c;
  }
  TRY(upload(ctx, &ctx->d_gD, gD.data(), gD.size()));
  TRY(upload(ctx, &ctx->d_gM, gM.data(), gM.size()));
  ctx->sweep.assign(m, nullptr);
  for (int j = 0; j < m; ++j) TRY(upload(ctx, &ctx->sweep[j], gs[j].data(), gs[j].size()));
  // the last two iterates are compared once there are two of them (m >= 3)
  if (m >= 3) TRY(upload(ctx, &ctx->d_cnchk, ck.data(), ck.size()));
  return VGTB_OK;
}

// Crank-Nicolson step (Eq. 5) for every trajectory and k:
//   D = 2 C C^dagger -> observables and SCC shift at t_n -> H(t_{n+1/2}) ->
//   M = S^-1 H -> fixed-point sweeps Y^dagger <- C^dagger + i (dt/2) Y^dagger M^dagger
//   (Y = (1 + i (dt/2) M)^-1 C) -> C^dagger(t_{n+1}) = 2 Y^dagger - C^dagger, fused
//   into the last sweep -> convergence check -> step counter.
// Event classes: obs (density product + sums), scc, phase, gemm1 (M), gemm2
// (sweeps), leap (check + counter).
// D_k = 2 C_k C_k^dagger for the charge, current and energy sums: at H's nonzero
// pattern only when the sampled kernel is set up, else the dense product
void launch_cn_density(vgtb_ctx* ctx, cudaStream_t st) {
  if (ctx->d_cnd)
    launch_cn_density_pattern(ctx->d_cnd, ctx->d_bsrsys, ctx->n_items, ctx->bsr_grp_max, ctx->bsr_ent_max, st);
  else
    launch_gemm_f64(ctx->d_gD, ctx->n_items, ctx->max_Np, ctx->max_Np, nullptr, st);
}

int enqueue_step_cn(vgtb_ctx* ctx, cudaEvent_t* ev, unsigned evflag) {
  cudaStream_t st = ctx->stream;
  const int nt = (int)ctx->trj.size();
  const int stride = ctx->opt.obs_stride > 0 ? ctx->opt.obs_stride : 1;
  launch_cn_density(ctx, st);
  launch_obs(ctx->d_sys, ctx->d_trj, ctx->d_items, ctx->d_wpre, nt, ctx->total_warps, ctx->d_step, 0, -1, st);
  if (ev) CK(cudaEventRecordWithFlags(ev[1], st, evflag));
  launch_scc(ctx->d_sys, ctx->d_trj, nt, ctx->d_step, stride, -1, 1, ctx->max_nat, 0, st);
  if (ev) CK(cudaEventRecordWithFlags(ev[2], st, evflag));
  launch_phase(ctx->d_sys, ctx->d_trj, ctx->d_items, ctx->d_wpre, nt, ctx->total_warps, ctx->d_step, PH_FP64_CN, -1,
               st);
  if (ev) CK(cudaEventRecordWithFlags(ev[3], st, evflag));
  if (ctx->bsr)
    launch_bsr(ctx->d_bsr, ctx->d_bsrsys, ctx->n_items, ctx->bsr_units_max, ctx->bsr_units_total, ctx->d_bsr_u0,
               ctx->d_bsr_ctr, 1, ctx->bsr_tg_max, nullptr, st);
  else
    launch_gemm_f64(ctx->d_gM, ctx->n_items, ctx->max_Np, ctx->max_Np, nullptr, st);
  if (ev) CK(cudaEventRecordWithFlags(ev[4], st, evflag));
  for (GemmF64Item* g : ctx->sweep) launch_gemm_f64(g, ctx->n_items, ctx->max_nocc, ctx->max_Np, nullptr, st);
  if (ev) CK(cudaEventRecordWithFlags(ev[5], st, evflag));
  if (ctx->d_cnchk)
    launch_cn_check(ctx->d_cnchk, ctx->n_items, ctx->max_nocc * ctx->max_Np, ctx->d_trj, ctx->opt.cn_tol, st);
  launch_increment(ctx->d_step, st);
  if (ev) CK(cudaEventRecordWithFlags(ev[6], st, evflag));
  CK(cudaGetLastError());
  return VGTB_OK;
}

// observables and SCC of the current level: split form k_obs_atoms_split + k_scc_eps,
// FP64 paths k_obs + k_scc_atoms + k_scc_eps
// finish = 0 (split step): the phase build's finisher CTAs add up J, E and the checks
void launch_obs_scc(vgtb_ctx* ctx, cudaEvent_t* ev, unsigned evflag, int stride, int finish = 1) {
  cudaStream_t st = ctx->stream;
  const int nt = (int)ctx->trj.size();
  if (ctx->split)
    launch_obs_atoms_split(ctx->d_sys, ctx->d_trj, ctx->d_items, nt, ctx->max_nat, ctx->d_step, stride, -1, 1, st);
  else
    launch_obs(ctx->d_sys, ctx->d_trj, ctx->d_items, ctx->d_wpre, nt, ctx->total_warps, ctx->d_step,
               ctx->delta ? 1 : 0, -1, st);
  if (ev) cudaEventRecordWithFlags(ev[1], st, evflag);
  launch_scc(ctx->d_sys, ctx->d_trj, nt, ctx->d_step, stride, -1, 1, ctx->max_nat, ctx->split ? 1 : 0, st,
             ctx->split ? finish : 1);
}

int enqueue_step(vgtb_ctx* ctx, cudaEvent_t* ev) {
  cudaStream_t st = ctx->stream;
  unsigned evflag = cudaEventRecordDefault;
  if (ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusActive) evflag = cudaEventRecordExternal;
  }
  const int nt = (int)ctx->trj.size();
  const int stride = ctx->opt.obs_stride > 0 ? ctx->opt.obs_stride : 1;
  if (ev) CK(cudaEventRecordWithFlags(ev[0], st, evflag));
  if (ctx->cn) return enqueue_step_cn(ctx, ev, evflag);
  launch_obs_scc(ctx, ev, evflag, stride, ctx->split ? 0 : 1);
  if (ev) CK(cudaEventRecordWithFlags(ev[2], st, evflag));
  if (ctx->split)
    launch_phase_split(ctx->d_sys, ctx->d_trj, ctx->d_items, ctx->d_wpre, nt, ctx->total_warps, ctx->max_nk,
                       ctx->d_step, 1, st);
  else
    launch_phase(ctx->d_sys, ctx->d_trj, ctx->d_items, ctx->d_wpre, nt, ctx->total_warps, ctx->d_step,
                 ctx->delta ? PH_FP64_DELTA : PH_FP64_PLAIN, -1, st);
  if (ev) CK(cudaEventRecordWithFlags(ev[3], st, evflag));
  if (ctx->bsr)
    launch_bsr(ctx->d_bsr, ctx->d_bsrsys, ctx->n_items, ctx->bsr_units_max, ctx->bsr_units_total, ctx->d_bsr_u0,
               ctx->d_bsr_ctr, ctx->split ? 0 : 1, ctx->bsr_tg_max, ctx->d_step, st);
  if (ctx->split && ctx->tcc) {
    // both products in one launch: its time counts as product 1's
    TRY(tc_launch_chain(ctx->tcc, st) == 0 ? VGTB_OK : fail(ctx, VGTB_E_CUDA, "chained tcgen05 launch failed"));
    if (ev) CK(cudaEventRecordWithFlags(ev[4], st, evflag));
  } else if (ctx->split) {
    if (!ctx->bsr)
      TRY(tc_launch(ctx->tc1, st) == 0 ? VGTB_OK : fail(ctx, VGTB_E_CUDA, "tcgen05 product 1 launch failed"));
    if (ev) CK(cudaEventRecordWithFlags(ev[4], st, evflag));
    TRY(tc_launch(ctx->tc2, st) == 0 ? VGTB_OK : fail(ctx, VGTB_E_CUDA, "tcgen05 product 2 launch failed"));
  } else {
    if (!ctx->bsr) launch_gemm_f64(ctx->d_g1, ctx->n_items, ctx->max_Np, ctx->max_Np, ctx->d_step, st);
    if (ev) CK(cudaEventRecordWithFlags(ev[4], st, evflag));
    launch_gemm_f64(ctx->d_g2, ctx->n_items, ctx->max_Np, ctx->max_Np, ctx->d_step, st);
  }
  if (ev) CK(cudaEventRecordWithFlags(ev[5], st, evflag));
  if (ctx->split)
    launch_leap_split(ctx->d_leap, ctx->n_items, ctx->max_Np, ctx->d_step, ctx->sys[0].dt, ctx->d_counter,
                      ctx->d_step, st);
  else
    launch_leap(ctx->d_leap, ctx->n_items, ctx->max_Np, 0, ctx->d_step, ctx->sys[0].dt, ctx->d_counter,
                ctx->d_step, st);
  if (ev) CK(cudaEventRecordWithFlags(ev[6], st, evflag));
  CK(cudaGetLastError());
  return VGTB_OK;
}

int accumulate_events(vgtb_ctx* ctx, int nsteps) {
  CK(cudaEventSynchronize(ctx->ev[7 * nsteps - 1]));
  for (int s = 0; s < nsteps; ++s) {
    cudaEvent_t* e = &ctx->ev[7 * s];
    for (int c = 0; c < VGTB_K_COUNT; ++c) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e[c], e[c + 1]));
      ctx->prof_ms[c] += ms;
      ctx->prof_launch[c] += 1;
    }
  }
  return VGTB_OK;
}

int ensure_events(vgtb_ctx* ctx, int nsteps) {
  while ((int)ctx->ev.size() < 7 * nsteps) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    ctx->ev.push_back(e);
  }
  return VGTB_OK;
}

int build_graph(vgtb_ctx* ctx, int G) {
  drop_graph(ctx);
  if (ctx->profile) TRY(ensure_events(ctx, G));
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  int rc = VGTB_OK;
  for (int s = 0; s < G && rc == VGTB_OK; ++s) rc = enqueue_step(ctx, ctx->profile ? &ctx->ev[7 * s] : nullptr);
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (rc != VGTB_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(ctx, VGTB_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, VGTB_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  ctx->graph_steps = G;
  ctx->graph_profiled = ctx->profile;
  return VGTB_OK;
}

int check_status(vgtb_ctx* ctx) {
  for (size_t t = 0; t < ctx->trj.size(); ++t) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, ctx->trj[t].status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (st & ST_TIMEOUT) return fail(ctx, VGTB_E_TIMEOUT, "trajectory %zu: a bounded device wait expired", t);
    // an unconverged Crank-Nicolson solve is the cause of any drift that follows it
    if (st & ST_CN_NOCONV)
      return fail(ctx, VGTB_E_UNSTABLE,
                  "trajectory %zu: Crank-Nicolson fixed point not converged (raise cn_iter or lower dt)", t);
    if (st & ST_NONFINITE) return fail(ctx, VGTB_E_UNSTABLE, "trajectory %zu: non-finite observables", t);
    if (st & ST_DRIFT) return fail(ctx, VGTB_E_UNSTABLE, "trajectory %zu: electron count drifted", t);
  }
  if (!ctx->split) return VGTB_OK;
  const int tc = tc_status(ctx->tc1, ctx->stream) | tc_status(ctx->tc2, ctx->stream);
  if (tc) {
    // an aborted chained launch left its block counts short: start them again
    if (ctx->tcc) tc_reset_chain(ctx->tcc, ctx->stream);
    return fail(ctx, VGTB_E_TIMEOUT, "tcgen05 product reported status %d (bounded wait expired)", tc);
  }
  return VGTB_OK;
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

void vgtb_default_options(vgtb_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = VGTB_FP64;
  opt->init = VGTB_INIT_GROUND;
  opt->obs_stride = 1;
  opt->graph_steps = 32;
  opt->timeout_ns = 2000000000LL;
  opt->scc_tol = 1e-11;
  opt->scc_max_iter = 200;
  opt->integrator = VGTB_LEAPFROG;
  opt->cn_iter = 12;
  opt->cn_tol = 1e-10;
  opt->tile_variant[0] = opt->tile_variant[1] = -1;
}

int vgtb_create(vgtb_ctx** out, const vgtb_system* sys, const vgtb_options* opt) {
  const int zero = 0;
  return vgtb_create_batch(out, 1, sys, 1, &zero, opt);
}

int vgtb_create_batch(vgtb_ctx** out, int n_sys, const vgtb_system* sys, int n_traj, const int* traj_sys,
                      const vgtb_options* opt) {
  if (!out) return fail(nullptr, VGTB_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_sys < 1 || !sys || n_traj < 1 || !traj_sys) return fail(nullptr, VGTB_E_INVALID, "empty batch");
  vgtb_ctx* ctx = new vgtb_ctx();
  vgtb_default_options(&ctx->opt);
  if (opt) ctx->opt = *opt;
  if (ctx->opt.obs_stride <= 0) ctx->opt.obs_stride = 1;
  if (ctx->opt.graph_steps <= 0) ctx->opt.graph_steps = 32;
  if (ctx->opt.timeout_ns <= 0) ctx->opt.timeout_ns = 2000000000LL;
  auto bail = [&](int rc) {
    g_create_error = ctx->err;
    vgtb_destroy(ctx);
    return rc;
  };
  if (ctx->opt.precision != VGTB_FP64 && ctx->opt.precision != VGTB_SPLIT_BF16X3)
    return bail(fail(ctx, VGTB_E_INVALID, "unknown precision %d", ctx->opt.precision));
  if (ctx->opt.init != VGTB_INIT_GROUND && ctx->opt.init != VGTB_INIT_USER)
    return bail(fail(ctx, VGTB_E_INVALID, "unknown init %d", ctx->opt.init));
  if (ctx->opt.integrator != VGTB_LEAPFROG && ctx->opt.integrator != VGTB_CRANK_NICOLSON)
    return bail(fail(ctx, VGTB_E_INVALID, "unknown integrator %d", ctx->opt.integrator));
  if (ctx->opt.scc != VGTB_SCC_ON && ctx->opt.scc != VGTB_SCC_FROZEN)
    return bail(fail(ctx, VGTB_E_INVALID, "unknown scc mode %d", ctx->opt.scc));
  if (ctx->opt.chain < VGTB_CHAIN_AUTO || ctx->opt.chain > VGTB_CHAIN_ON)
    return bail(fail(ctx, VGTB_E_INVALID, "unknown chain mode %d", ctx->opt.chain));
  if (ctx->opt.product1 < VGTB_P1_AUTO || ctx->opt.product1 > VGTB_P1_BLOCKS)
    return bail(fail(ctx, VGTB_E_INVALID, "unknown product1 form %d", ctx->opt.product1));
  ctx->split = ctx->opt.precision == VGTB_SPLIT_BF16X3;
  ctx->cn = ctx->opt.integrator == VGTB_CRANK_NICOLSON;
  if (ctx->cn && ctx->split)
    return bail(fail(ctx, VGTB_E_UNSUPPORTED, "the Crank-Nicolson integrator runs in FP64 precision only"));
  if (ctx->opt.cn_iter <= 0) ctx->opt.cn_iter = 12;
  if (ctx->opt.cn_iter < 2)
    return bail(fail(ctx, VGTB_E_INVALID, "cn_iter must be >= 2 (the last sweep writes C in place)"));
  if (!(ctx->opt.cn_tol > 0.0)) ctx->opt.cn_tol = 1e-10;
  ctx->delta = ctx->split || (ctx->opt.delta_form != 0 && !ctx->cn);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bail(fail(ctx, VGTB_E_CUDA, "no CUDA device"));
  for (int p = 0; p < 2; ++p)
    if (ctx->opt.tile_variant[p] < -1 || ctx->opt.tile_variant[p] >= tc_num_variants())
      return bail(fail(ctx, VGTB_E_INVALID, "tile_variant[%d] = %d out of range", p, ctx->opt.tile_variant[p]));
  if (ctx->split && !tc_gemm_supported())
    return bail(fail(ctx, VGTB_E_UNSUPPORTED, "split precision needs an sm_103a (GB300) device"));
  if (ctx->opt.cuda_stream) {
    ctx->stream = (cudaStream_t)ctx->opt.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(ctx, VGTB_E_CUDA, "stream creation failed"));
    ctx->own_stream = true;
  }
  if (cusolverDnCreate(&ctx->solver) != CUSOLVER_STATUS_SUCCESS)
    return bail(fail(ctx, VGTB_E_CUDA, "cusolverDnCreate failed"));
  cusolverDnSetStream(ctx->solver, ctx->stream);
  for (int t = 0; t < n_traj; ++t)
    if (traj_sys[t] < 0 || traj_sys[t] >= n_sys)
      return bail(fail(ctx, VGTB_E_INVALID, "traj_sys[%d] = %d out of range", t, traj_sys[t]));
  const double dt0 = sys[0].dt;
  for (int s = 0; s < n_sys; ++s)
    if (sys[s].dt != dt0) return bail(fail(ctx, VGTB_E_INVALID, "all systems of a batch share one dt"));
  ctx->sys.resize(n_sys);
  std::vector<DevSys> dsys(n_sys);
  int rc;
  for (int s = 0; s < n_sys; ++s) {
    rc = prepare_system(ctx, s, sys[s], ctx->sys[s], dsys[s], ctx->opt.init == VGTB_INIT_GROUND || ctx->cn);
    if (rc) return bail(rc);
    ctx->max_nocc = std::max(ctx->max_nocc, ctx->sys[s].nocc);
    ctx->max_nk = std::max(ctx->max_nk, ctx->sys[s].nk);
    ctx->max_nat = std::max(ctx->max_nat, ctx->sys[s].nat);
    ctx->max_Np = std::max(ctx->max_Np, ctx->sys[s].Np);
  }
  if (scc_configure(ctx->max_nat)) return bail(fail(ctx, VGTB_E_CUDA, "k_scc shared memory configuration failed"));
  // block-sparse first product when every atom of every system carries 4 orbitals
  // block-sparse first product: asked for, or by default on the FP64 path (on
  // the split form the dense tcgen05 product is faster at these sizes)
  bool blocks_ok = true;
  for (auto& h : ctx->sys) blocks_ok = blocks_ok && bsr_possible(h);
  if (ctx->opt.product1 == VGTB_P1_BLOCKS && !blocks_ok)
    return bail(fail(ctx, VGTB_E_UNSUPPORTED, "block-sparse first product needs 4 orbitals on every atom"));
  // (Crank-Nicolson: the product M = S^-1 H of every step, FP64)
  ctx->bsr = blocks_ok &&
             (ctx->opt.product1 == VGTB_P1_BLOCKS || (ctx->opt.product1 == VGTB_P1_AUTO && !ctx->split));
  std::vector<BsrSys> bsys(n_sys);
  if (ctx->bsr) {
    for (int s = 0; s < n_sys; ++s) {
      if ((rc = build_bsr_tables(ctx, ctx->sys[s], ctx->split ? 0 : 1, bsys[s]))) return bail(rc);
      ctx->bsr_units_max = std::max(ctx->bsr_units_max, ctx->sys[s].bsr_units);
      ctx->bsr_tg_max = std::max(ctx->bsr_tg_max, ctx->sys[s].bsr_tg_max);
      ctx->bsr_ent_max = std::max(ctx->bsr_ent_max, ctx->sys[s].bsr_ent_max);
      ctx->bsr_grp_max = std::max(ctx->bsr_grp_max, bsys[s].n_grp);
    }
    if (bsr_configure(ctx->split ? 0 : 1, ctx->bsr_tg_max))
      return bail(fail(ctx, VGTB_E_UNSUPPORTED, "block-sparse product: %d targets per atom group exceed shared memory",
                       ctx->bsr_tg_max));
    if ((rc = upload(ctx, &ctx->d_bsrsys, bsys.data(), bsys.size()))) return bail(rc);
    if (ctx->split)
      for (int s = 0; s < n_sys; ++s) {
        HostSys& h = ctx->sys[s];
        if ((rc = dalloc(ctx, &h.D0f, (size_t)h.nk * h.Np * h.Np))) return bail(rc);
        dsys[s].D0f = h.D0f;
      }
  }
  if ((rc = upload(ctx, &ctx->d_sys, dsys.data(), dsys.size()))) return bail(rc);
  // trajectories and items; the split form keeps each operand family of a
  // system contiguous over its items so that one 4-D tensor map covers it
  ctx->trj.resize(n_traj);
  std::vector<int> wpre(n_traj + 1, 0);
  std::vector<int> sys_items(n_sys, 0), sys_next(n_sys, 0);
  for (int t = 0; t < n_traj; ++t) sys_items[traj_sys[t]] += ctx->sys[traj_sys[t]].nk;
  struct Fam {
    __nv_bfloat16 *dD = nullptr, *Hemb = nullptr, *dHemb = nullptr, *Wemb = nullptr;
    float* Xf = nullptr;
  };
  std::vector<Fam> fam(n_sys);
  if (ctx->split) {
    for (int s = 0; s < n_sys; ++s) {
      const size_t NN = (size_t)ctx->sys[s].Np * ctx->sys[s].Np, ni = sys_items[s];
      if (ni == 0) continue;
      if (!ctx->bsr) {
        if ((rc = dalloc(ctx, &fam[s].dD, 4 * NN * ni))) return bail(rc);
        if ((rc = dalloc(ctx, &fam[s].Hemb, 8 * NN * ni))) return bail(rc);
        if ((rc = dalloc(ctx, &fam[s].dHemb, 8 * NN * ni))) return bail(rc);
      }
      if ((rc = dalloc(ctx, &fam[s].Wemb, 8 * NN * ni))) return bail(rc);
      if ((rc = dalloc(ctx, &fam[s].Xf, 2 * NN * ni))) return bail(rc);
    }
  }
  for (int t = 0; t < n_traj; ++t) {
    HostTraj& T = ctx->trj[t];
    HostSys& h = ctx->sys[traj_sys[t]];
    T.sys = traj_sys[t];
    T.item0 = (int)ctx->items_h.size();
    h.trajs.push_back(t);
    wpre[t + 1] = wpre[t] + h.n_tgt;
    const size_t NN = (size_t)h.Np * h.Np;
    for (int k = 0; k < h.nk; ++k) {
      DevItem it;
      memset(&it, 0, sizeof(it));
      it.sys = T.sys;
      it.traj = t;
      it.k = k;
      double2* lv = nullptr;
      // Crank-Nicolson rebuilds D from C at every level: one buffer serves both parities
      if ((rc = dalloc(ctx, &lv, ctx->cn ? NN : 2 * NN))) return bail(rc);
      it.D[0] = lv;
      it.D[1] = ctx->cn ? lv : lv + NN;
      if (ctx->split) {
        const size_t li = sys_next[T.sys]++;
        if (ctx->bsr) {
          float2 *kh = nullptr, *kdh = nullptr;
          if ((rc = dalloc(ctx, &it.dDf, NN))) return bail(rc);
          if ((rc = dalloc(ctx, &kh, (size_t)h.n_el))) return bail(rc);
          if ((rc = dalloc(ctx, &kdh, (size_t)h.n_el))) return bail(rc);
          it.kH = kh;
          it.kdH = kdh;
        } else {
          it.dD_p = fam[T.sys].dD + 4 * NN * li;
          it.Hemb_p = fam[T.sys].Hemb + 8 * NN * li;
          it.dHemb_p = fam[T.sys].dHemb + 8 * NN * li;
        }
        it.Wemb_p = fam[T.sys].Wemb + 8 * NN * li;
        it.Xf = fam[T.sys].Xf + 2 * NN * li;
      } else if (ctx->cn) {
        const size_t nc = (size_t)h.nocc * h.Np;
        if (ctx->bsr) {
          double2* kh = nullptr;
          if ((rc = dalloc(ctx, &kh, (size_t)h.n_el))) return bail(rc);
          it.kH = kh;
        } else if ((rc = dalloc(ctx, &it.H, NN))) {
          return bail(rc);
        }
        if ((rc = dalloc(ctx, &it.W, NN))) return bail(rc);
        if ((rc = dalloc(ctx, &it.Cd, nc))) return bail(rc);
        if ((rc = dalloc(ctx, &it.Y[0], nc))) return bail(rc);
        if ((rc = dalloc(ctx, &it.Y[1], nc))) return bail(rc);
      } else {
        if (ctx->bsr) {
          double2 *kh = nullptr, *kdh = nullptr;
          if ((rc = dalloc(ctx, &kh, (size_t)h.n_el))) return bail(rc);
          if (ctx->delta && (rc = dalloc(ctx, &kdh, (size_t)h.n_el))) return bail(rc);
          it.kH = kh;
          it.kdH = kdh;
        } else {
          if ((rc = dalloc(ctx, &it.H, NN))) return bail(rc);
          if (ctx->delta && (rc = dalloc(ctx, &it.dH, NN))) return bail(rc);
        }
        if ((rc = dalloc(ctx, &it.W, NN))) return bail(rc);
        if ((rc = dalloc(ctx, &it.X, NN))) return bail(rc);
      }
      ctx->items_h.push_back(it);
    }
    if ((rc = dalloc(ctx, &T.dq, h.nat))) return bail(rc);
    if ((rc = dalloc(ctx, &T.eps, h.nat))) return bail(rc);
    if (ctx->cn && (rc = dalloc(ctx, &T.eps_lv, 2 * (size_t)h.nat))) return bail(rc);
    if (ctx->split) {
      if ((rc = dalloc(ctx, &T.epsf, h.nat))) return bail(rc);
      if ((rc = dalloc(ctx, &T.depsf, h.nat))) return bail(rc);
      if ((rc = dalloc(ctx, &T.af, 3))) return bail(rc);
    }
    if ((rc = dalloc(ctx, &T.part, 5 * (size_t)h.n_tgt))) return bail(rc);
    if ((rc = dalloc(ctx, &T.cpart, 6 * (size_t)((h.nat + kSccRowsPerCta - 1) / kSccRowsPerCta)))) return bail(rc);
    if ((rc = dalloc(ctx, &T.apart, 4 * (size_t)h.nat))) return bail(rc);
    if ((rc = dalloc(ctx, &T.ticket, 1))) return bail(rc);
    if ((rc = dalloc(ctx, &T.status, 1))) return bail(rc);
  }
  ctx->n_items = (int)ctx->items_h.size();
  ctx->total_warps = wpre[n_traj];
  if ((rc = upload(ctx, &ctx->d_wpre, wpre.data(), wpre.size()))) return bail(rc);
  if ((rc = upload(ctx, &ctx->d_items, ctx->items_h.data(), ctx->items_h.size()))) return bail(rc);
  if ((rc = dalloc(ctx, &ctx->d_trj, n_traj))) return bail(rc);
  if ((rc = dalloc(ctx, &ctx->d_step, 1))) return bail(rc);
  if ((rc = dalloc(ctx, &ctx->d_counter, 1))) return bail(rc);
  if ((rc = upload_traj_table(ctx))) return bail(rc);
  // work lists of the FP64 products and of the leapfrog
  std::vector<GemmF64Item> g1(ctx->n_items), g2(ctx->n_items);
  std::vector<LeapItem> lv(ctx->n_items);
  for (int i = 0; i < ctx->n_items; ++i) {
    const DevItem& it = ctx->items_h[i];
    const HostSys& h = ctx->sys[it.sys];
    const size_t NN = (size_t)h.Np * h.Np;
    GemmF64Item a{}, b{};
    a.A[0] = it.D[0];
    a.a_par[0] = (long long)NN;
    a.R[0] = it.H;
    a.K[0] = h.Np;
    a.lda[0] = a.ldr[0] = h.Np;
    a.nseg = 1;
    if (ctx->delta) {
      a.A[1] = h.D0 + it.k * NN;
      a.R[1] = it.dH;
      a.K[1] = h.Np;
      a.lda[1] = a.ldr[1] = h.Np;
      a.nseg = 2;
    }
    a.M = a.N = a.ldc = h.Np;
    a.C = it.W;
    b.A[0] = h.Sinv + it.k * NN;
    b.R[0] = it.W;
    b.K[0] = h.Np;
    b.lda[0] = b.ldr[0] = h.Np;
    b.nseg = 1;
    b.M = b.N = b.ldc = h.Np;
    b.C = it.X;
    g1[i] = a;
    g2[i] = b;
    LeapItem l{};
    l.X = ctx->split ? (const void*)it.Xf : (const void*)it.X;
    l.R0 = (ctx->delta && !ctx->split) ? h.R0 + it.k * NN : nullptr;
    l.R0f = ctx->split ? h.R0f + 2 * NN * it.k : nullptr;
    l.D[0] = it.D[0];
    l.D[1] = it.D[1];
    l.pieces = it.dD_p;
    l.f32 = it.dDf;
    l.Np = h.Np;
    l.mode = 0;
    lv[i] = l;
  }
  if (ctx->cn) {
    if ((rc = build_cn_lists(ctx))) return bail(rc);
  } else if (!ctx->split) {
    if ((rc = upload(ctx, &ctx->d_g1, g1.data(), g1.size()))) return bail(rc);
    if ((rc = upload(ctx, &ctx->d_g2, g2.data(), g2.size()))) return bail(rc);
  }
  if ((rc = upload(ctx, &ctx->d_leap, lv.data(), lv.size()))) return bail(rc);
  if (ctx->bsr) {
    std::vector<BsrItem> bl(ctx->n_items);
    for (int i = 0; i < ctx->n_items; ++i) {
      const DevItem& it = ctx->items_h[i];
      const HostSys& h = ctx->sys[it.sys];
      const size_t NN = (size_t)h.Np * h.Np;
      BsrItem b{};
      b.sys = it.sys;
      b.nseg = ctx->delta ? 2 : 1;
      b.R[0] = it.kH;
      b.R[1] = it.kdH;
      if (ctx->cn) {
        b.nseg = 1;                            // M = S^-1 H^dagger of the midpoint H
        b.A[0] = h.Sinv + it.k * NN;
        b.W = it.W;
      } else if (ctx->split) {
        b.A[0] = it.dDf;                       // FP32 copy of the current dD level
        b.A[1] = h.D0f + it.k * NN;
        b.W = it.Wemb_p;
      } else {
        b.A[0] = it.D[0];                      // level of the step's parity
        b.a_par = (long long)NN;
        b.A[1] = ctx->delta ? (const void*)(h.D0 + it.k * NN) : nullptr;
        b.W = it.W;
      }
      bl[i] = b;
    }
    if ((rc = upload(ctx, &ctx->d_bsr, bl.data(), bl.size()))) return bail(rc);
    std::vector<int> u0(ctx->n_items + 1, 0);
    for (int i = 0; i < ctx->n_items; ++i) u0[i + 1] = u0[i] + ctx->sys[ctx->items_h[i].sys].bsr_units;
    ctx->bsr_units_total = u0[ctx->n_items];
    if ((rc = upload(ctx, &ctx->d_bsr_u0, u0.data(), u0.size()))) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->d_bsr_ctr, 2))) return bail(rc);
    if (ctx->cn && ctx->bsr_tg_max <= cn_density_max_targets() && cn_density_configure(ctx->bsr_ent_max) == 0) {
      std::vector<CnDensItem> cd(ctx->n_items);
      for (int i = 0; i < ctx->n_items; ++i) {
        const DevItem& it = ctx->items_h[i];
        cd[i] = CnDensItem{it.sys, it.Cd, it.D[0], ctx->sys[it.sys].nocc};
      }
      if ((rc = upload(ctx, &ctx->d_cnd, cd.data(), cd.size()))) return bail(rc);
    }
  }
  // setup: S^-1, ground state
  for (int s = 0; s < n_sys; ++s) {
    if ((rc = build_sinv(ctx, s))) return bail(rc);
  }
  if (ctx->split) {
    std::vector<TcSysView> views(n_sys);
    for (int s = 0; s < n_sys; ++s) {
      views[s].Np = ctx->sys[s].Np;
      views[s].nk = ctx->sys[s].nk;
      views[s].n_items = sys_items[s];
      views[s].Sinv_p = ctx->sys[s].Sinv_p;
      views[s].D0_p = ctx->sys[s].D0_p;
      views[s].dD_p = fam[s].dD;
      views[s].Hemb_p = fam[s].Hemb;
      views[s].dHemb_p = fam[s].dHemb;
      views[s].Wemb_p = fam[s].Wemb;
      if (ctx->opt.product1 != VGTB_P1_DENSE) {  // nonzero pattern: zero k-panels of product 1 are skipped
        views[s].orb_off = &ctx->sys[s].orb_off;
        views[s].tgt_I = &ctx->sys[s].tgt_I;
        views[s].tgt_J = &ctx->sys[s].tgt_J;
      }
    }
    std::string msg;
    // alt1 / alt2: the fastest chainable plans when the autotuner's picks are
    // other variants (a stream-K schedule, say), so that the one-launch
    // schedule competes against the fastest pair of separate launches
    TcPlan *alt1 = nullptr, *alt2 = nullptr;
    const bool want_alt = ctx->opt.chain != VGTB_CHAIN_OFF;
    if (tc_build_plans(views, ctx->items_h, ctx->opt.timeout_ns, ctx->opt.autotune, ctx->opt.tile_variant, ctx->stream,
                       ctx->bsr ? nullptr : &ctx->tc1, &ctx->tc2, &msg, want_alt ? &alt1 : nullptr,
                       want_alt ? &alt2 : nullptr)) {
      // a failure in product 2 can follow a product 1 that already kept an alternate
      if (alt1) tc_destroy_plan(alt1);
      if (alt2) tc_destroy_plan(alt2);
      return bail(fail(ctx, VGTB_E_CUDA, "tcgen05 plan: %s", msg.c_str()));
    }
    TcPlan* c1 = (alt1 && !tc_chainable(ctx->tc1, ctx->tc1)) ? alt1 : ctx->tc1;
    TcPlan* c2 = (alt2 && !tc_chainable(ctx->tc2, ctx->tc2)) ? alt2 : ctx->tc2;
    if (ctx->opt.chain != VGTB_CHAIN_OFF && tc_chainable(c1, c2)) {
      if (tc_build_chain(c1, c2, &ctx->tcc, &msg)) {
        if (alt1) tc_destroy_plan(alt1);
        if (alt2) tc_destroy_plan(alt2);
        return bail(fail(ctx, VGTB_E_CUDA, "tcgen05 chained plan: %s", msg.c_str()));
      }
      if (ctx->opt.chain == VGTB_CHAIN_AUTO) {
        double ms_chain = 0, ms_sep = 0;
        // a launch that failed or ran into the wait limit keeps two launches
        const int tr = tc_time_chain(ctx->tcc, ctx->tc1, ctx->tc2, ctx->stream, &ms_chain, &ms_sep);
        if (tr || ms_chain >= ms_sep) {
          tc_destroy_chain(ctx->tcc);
          ctx->tcc = nullptr;
        }
        if (tr) {
          cudaStreamSynchronize(ctx->stream);
          cudaGetLastError();
          tc_clear_error(ctx->tc1);
          tc_clear_error(ctx->tc2);
          tc_clear_error(c1);
          tc_clear_error(c2);
        }
      }
    }
    // the chain runs on its own plans: they become the context's products
    if (ctx->tcc && c1 != ctx->tc1) {
      tc_destroy_plan(ctx->tc1);
      ctx->tc1 = c1;
    } else if (alt1 && alt1 != ctx->tc1) {
      tc_destroy_plan(alt1);
    }
    if (ctx->tcc && c2 != ctx->tc2) {
      tc_destroy_plan(ctx->tc2);
      ctx->tc2 = c2;
    } else if (alt2 && alt2 != ctx->tc2) {
      tc_destroy_plan(alt2);
    }
  }
  if (ctx->opt.init == VGTB_INIT_GROUND) {
    for (int s = 0; s < n_sys; ++s) {
      if ((rc = ground_state(ctx, s))) return bail(rc);
      if ((rc = finish_density(ctx, s))) return bail(rc);
    }
    if ((rc = reset_all(ctx))) return bail(rc);
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bail(fail(ctx, VGTB_E_CUDA, "setup failed: %s", cudaGetErrorString(e)));
  *out = ctx;
  return VGTB_OK;
}

int vgtb_set_density(vgtb_ctx* ctx, int s, int k, const double* d0) {
  if (!ctx) return VGTB_E_INVALID;
  if (ctx->cn)
    return fail(ctx, VGTB_E_INVALID, "the Crank-Nicolson integrator starts from states: use vgtb_set_coefficients");
  if (s < 0 || s >= (int)ctx->sys.size()) return fail(ctx, VGTB_E_INVALID, "system index %d out of range", s);
  HostSys& h = ctx->sys[s];
  if (k < 0 || k >= h.nk) return fail(ctx, VGTB_E_INVALID, "k index %d out of range", k);
  if (!d0 || !finite_all(d0, 2 * (size_t)h.N * h.N)) return fail(ctx, VGTB_E_INVALID, "density is NULL or non-finite");
  const size_t NN = (size_t)h.Np * h.Np;
  CK(cudaMemcpy2DAsync(h.D0 + k * NN, sizeof(double2) * h.Np, d0, sizeof(double2) * h.N, sizeof(double2) * h.N, h.N,
                       cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // the system is ready once every k has been set
  h.k_set.resize(h.nk, 0);
  h.k_set[k] = 1;
  bool all = true;
  for (char c : h.k_set) all &= c != 0;
  if (all || h.density_set) {
    TRY(finish_density(ctx, s));
    TRY(reset_all(ctx));
  }
  return VGTB_OK;
}

int vgtb_set_coefficients(vgtb_ctx* ctx, int s, int k, int n_occ, const double* c) {
  if (!ctx) return VGTB_E_INVALID;
  if (!ctx->cn) return fail(ctx, VGTB_E_INVALID, "vgtb_set_coefficients needs the Crank-Nicolson integrator");
  if (s < 0 || s >= (int)ctx->sys.size()) return fail(ctx, VGTB_E_INVALID, "system index %d out of range", s);
  HostSys& h = ctx->sys[s];
  if (k < 0 || k >= h.nk) return fail(ctx, VGTB_E_INVALID, "k index %d out of range", k);
  if (n_occ != h.nocc) return fail(ctx, VGTB_E_INVALID, "n_occ = %d, the system has %d occupied states", n_occ, h.nocc);
  if (!c || !finite_all(c, 2 * (size_t)h.N * h.nocc))
    return fail(ctx, VGTB_E_INVALID, "coefficients are NULL or non-finite");
  const size_t NN = (size_t)h.Np * h.Np;
  double2* tmp = nullptr;
  CK(cudaMallocAsync(&tmp, sizeof(double2) * (size_t)h.N * h.nocc, ctx->stream));
  CK(cudaMemcpyAsync(tmp, c, sizeof(double2) * (size_t)h.N * h.nocc, cudaMemcpyHostToDevice, ctx->stream));
  double2* Cd = h.C0d + (size_t)k * h.nocc * h.Np;
  launch_conj_transpose(tmp, h.nocc, Cd, h.Np, h.nocc, h.N, ctx->stream);
  // D_k(0) = 2 C C^dagger (charges of the start, vgtb_get_initial_density)
  GemmF64Item g{};
  g.A[0] = g.R[0] = Cd;
  g.K[0] = h.nocc;
  g.lda[0] = g.ldr[0] = h.Np;
  g.nseg = 1;
  g.conj_t = 3;
  g.M = g.N = h.N;
  g.ldc = h.Np;
  g.C = h.D0 + k * NN;
  g.epi = 1;
  g.coef = make_double2(2.0, 0.0);
  GemmF64Item* dg = nullptr;
  CK(cudaMallocAsync(&dg, sizeof(g), ctx->stream));
  CK(cudaMemcpyAsync(dg, &g, sizeof(g), cudaMemcpyHostToDevice, ctx->stream));
  launch_gemm_f64(dg, 1, h.N, h.N, nullptr, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaFreeAsync(tmp, ctx->stream));
  CK(cudaFreeAsync(dg, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  h.k_set.resize(h.nk, 0);
  h.k_set[k] = 1;
  bool all = true;
  for (char x : h.k_set) all &= x != 0;
  if (all || h.density_set) {
    TRY(finish_density(ctx, s));
    TRY(reset_all(ctx));
  }
  return VGTB_OK;
}

int vgtb_get_coefficients(vgtb_ctx* ctx, int t, int k, double* c_out) {
  if (!ctx) return VGTB_E_INVALID;
  if (!ctx->cn) return fail(ctx, VGTB_E_INVALID, "vgtb_get_coefficients needs the Crank-Nicolson integrator");
  if (t < 0 || t >= (int)ctx->trj.size()) return fail(ctx, VGTB_E_INVALID, "trajectory %d out of range", t);
  const HostTraj& T = ctx->trj[t];
  const HostSys& h = ctx->sys[T.sys];
  if (k < 0 || k >= h.nk || !c_out) return fail(ctx, VGTB_E_INVALID, "bad k or NULL output");
  const DevItem& it = ctx->items_h[T.item0 + k];
  double2* tmp = nullptr;
  CK(cudaMallocAsync(&tmp, sizeof(double2) * (size_t)h.N * h.nocc, ctx->stream));
  launch_conj_transpose(it.Cd, h.Np, tmp, h.nocc, h.N, h.nocc, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c_out, tmp, sizeof(double2) * (size_t)h.N * h.nocc, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaFreeAsync(tmp, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

int vgtb_set_field(vgtb_ctx* ctx, int t, int n_times, const double* A) {
  if (!ctx) return VGTB_E_INVALID;
  if (t < 0 || t >= (int)ctx->trj.size()) return fail(ctx, VGTB_E_INVALID, "trajectory %d out of range", t);
  if (n_times < 1 || !A || !finite_all(A, 3 * (size_t)n_times))
    return fail(ctx, VGTB_E_INVALID, "field table is empty or non-finite");
  HostTraj& T = ctx->trj[t];
  const HostSys& h = ctx->sys[T.sys];
  if (T.n_times != n_times) {
    const int stride = ctx->opt.obs_stride;
    TRY(dalloc(ctx, &T.A, 3 * (size_t)n_times));
    TRY(dalloc(ctx, &T.J, 3 * (size_t)n_times));
    TRY(dalloc(ctx, &T.E, (size_t)n_times));
    TRY(dalloc(ctx, &T.q, (size_t)((n_times - 1) / stride + 1) * h.nat));
    T.n_times = n_times;
  }
  CK(cudaMemcpyAsync(T.A, A, sizeof(double) * 3 * n_times, cudaMemcpyHostToDevice, ctx->stream));
  TRY(upload_traj_table(ctx));
  return reset_all(ctx);
}

int vgtb_propagate(vgtb_ctx* ctx, int nsteps) {
  if (!ctx) return VGTB_E_INVALID;
  if (nsteps < 0) return fail(ctx, VGTB_E_INVALID, "nsteps < 0");
  for (auto& h : ctx->sys)
    if (!h.density_set) return fail(ctx, VGTB_E_STATE, "no initial density set");
  for (size_t t = 0; t < ctx->trj.size(); ++t)
    if (ctx->trj[t].n_times < ctx->n_done + nsteps + 1)
      return fail(ctx, VGTB_E_STATE, "trajectory %zu: field table has %d levels, step %d needs %d", t,
                  ctx->trj[t].n_times, ctx->n_done + nsteps, ctx->n_done + nsteps + 1);
  const int G = ctx->opt.graph_steps;
  int left = nsteps;
  if (G > 1 && left >= G) {
    if (!ctx->graph || ctx->graph_steps != G || ctx->graph_profiled != ctx->profile) TRY(build_graph(ctx, G));
    while (left >= G) {
      CK(cudaGraphLaunch(ctx->graph, ctx->stream));
      if (ctx->profile) TRY(accumulate_events(ctx, G));
      left -= G;
    }
  }
  while (left > 0) {
    const int chunk = std::min(left, 64);
    if (ctx->profile) TRY(ensure_events(ctx, chunk));
    for (int s = 0; s < chunk; ++s) TRY(enqueue_step(ctx, ctx->profile ? &ctx->ev[7 * s] : nullptr));
    if (ctx->profile) TRY(accumulate_events(ctx, chunk));
    left -= chunk;
  }
  // observables of the final level
  const int nt = (int)ctx->trj.size();
  if (ctx->cn) launch_cn_density(ctx, ctx->stream);
  if (ctx->cn) {
    launch_obs(ctx->d_sys, ctx->d_trj, ctx->d_items, ctx->d_wpre, nt, ctx->total_warps, ctx->d_step, 0, -1,
               ctx->stream);
    launch_scc(ctx->d_sys, ctx->d_trj, nt, ctx->d_step, ctx->opt.obs_stride, -1, 1, ctx->max_nat, 0, ctx->stream);
  } else {
    launch_obs_scc(ctx, nullptr, 0, ctx->opt.obs_stride);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->n_done += nsteps;
  return check_status(ctx);
}

int vgtb_steps_done(const vgtb_ctx* ctx) { return ctx ? ctx->n_done : -1; }

int vgtb_observables(vgtb_ctx* ctx, int t, double* J, double* E, double* q) {
  if (!ctx) return VGTB_E_INVALID;
  if (t < 0 || t >= (int)ctx->trj.size()) return fail(ctx, VGTB_E_INVALID, "trajectory %d out of range", t);
  const HostTraj& T = ctx->trj[t];
  if (!T.J) return fail(ctx, VGTB_E_STATE, "no field set for trajectory %d", t);
  const int n = ctx->n_done + 1;
  if (J) CK(cudaMemcpyAsync(J, T.J, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream));
  if (E) CK(cudaMemcpyAsync(E, T.E, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  if (q) {
    const int nq = ctx->n_done / ctx->opt.obs_stride + 1;
    CK(cudaMemcpyAsync(q, T.q, sizeof(double) * nq * ctx->sys[T.sys].nat, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

int vgtb_get_density(vgtb_ctx* ctx, int t, int k, double* d_out) {
  if (!ctx) return VGTB_E_INVALID;
  if (t < 0 || t >= (int)ctx->trj.size()) return fail(ctx, VGTB_E_INVALID, "trajectory %d out of range", t);
  const HostTraj& T = ctx->trj[t];
  const HostSys& h = ctx->sys[T.sys];
  if (k < 0 || k >= h.nk || !d_out) return fail(ctx, VGTB_E_INVALID, "bad k or NULL output");
  const DevItem& it = ctx->items_h[T.item0 + k];
  const size_t NN = (size_t)h.Np * h.Np;
  const int cur = ctx->n_done & 1;
  // Crank-Nicolson steps form D only at H's nonzero pattern: the whole D = 2 C C^dagger now
  if (ctx->cn && ctx->d_cnd) launch_gemm_f64(ctx->d_gD, ctx->n_items, ctx->max_Np, ctx->max_Np, nullptr, ctx->stream);
  std::vector<double2> a(NN), b;
  CK(cudaMemcpyAsync(a.data(), it.D[cur], NN * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->delta) {
    b.resize(NN);
    CK(cudaMemcpyAsync(b.data(), h.D0 + it.k * NN, NN * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < h.N; ++i)
    for (int j = 0; j < h.N; ++j) {
      double2 v = a[(size_t)i * h.Np + j];
      if (ctx->delta) {
        v.x += b[(size_t)i * h.Np + j].x;
        v.y += b[(size_t)i * h.Np + j].y;
      }
      d_out[2 * ((size_t)i * h.N + j)] = v.x;
      d_out[2 * ((size_t)i * h.N + j) + 1] = v.y;
    }
  return VGTB_OK;
}

int vgtb_spectrum(vgtb_ctx* ctx, int t, int n0, int n1, double e0, double tau0, int n_omega, const double* omega,
                  double* sigma, double* eps) {
  if (!ctx) return VGTB_E_INVALID;
  if (t < 0 || t >= (int)ctx->trj.size()) return fail(ctx, VGTB_E_INVALID, "trajectory %d out of range", t);
  const HostTraj& T = ctx->trj[t];
  if (!T.J) return fail(ctx, VGTB_E_STATE, "no field set for trajectory %d", t);
  if (n0 < 0 || n1 <= n0) return fail(ctx, VGTB_E_INVALID, "need 0 <= n0 < n1");
  if (n1 > ctx->n_done) return fail(ctx, VGTB_E_STATE, "level %d not propagated yet (%d steps done)", n1, ctx->n_done);
  if (n_omega < 1 || !omega || !sigma || !eps) return fail(ctx, VGTB_E_INVALID, "empty frequency list or NULL output");
  if (!(e0 != 0.0) || !std::isfinite(e0) || !(tau0 > 0.0)) return fail(ctx, VGTB_E_INVALID, "need e0 != 0, tau0 > 0");
  for (int i = 0; i < n_omega; ++i)
    if (!(omega[i] > 0.0) || !std::isfinite(omega[i])) return fail(ctx, VGTB_E_INVALID, "frequencies must be > 0");
  double *dw = nullptr, *ds = nullptr, *de = nullptr;
  CK(cudaMallocAsync(&dw, sizeof(double) * n_omega, ctx->stream));
  CK(cudaMallocAsync(&ds, sizeof(double) * 6 * n_omega, ctx->stream));
  CK(cudaMallocAsync(&de, sizeof(double) * 6 * n_omega, ctx->stream));
  CK(cudaMemcpyAsync(dw, omega, sizeof(double) * n_omega, cudaMemcpyHostToDevice, ctx->stream));
  launch_conductivity(T.J, n0, n1, ctx->sys[T.sys].dt, e0, tau0, dw, n_omega, ds, de, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(sigma, ds, sizeof(double) * 6 * n_omega, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(eps, de, sizeof(double) * 6 * n_omega, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaFreeAsync(dw, ctx->stream));
  CK(cudaFreeAsync(ds, ctx->stream));
  CK(cudaFreeAsync(de, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

int vgtb_group_charges(vgtb_ctx* ctx, int t, int n_groups, const int* group, double* out) {
  if (!ctx) return VGTB_E_INVALID;
  if (t < 0 || t >= (int)ctx->trj.size()) return fail(ctx, VGTB_E_INVALID, "trajectory %d out of range", t);
  const HostTraj& T = ctx->trj[t];
  if (!T.q) return fail(ctx, VGTB_E_STATE, "no field set for trajectory %d", t);
  const int nat = ctx->sys[T.sys].nat;
  if (n_groups < 1 || !group || !out) return fail(ctx, VGTB_E_INVALID, "need n_groups >= 1 and non-NULL arrays");
  for (int i = 0; i < nat; ++i)
    if (group[i] >= n_groups) return fail(ctx, VGTB_E_INVALID, "group[%d] = %d >= n_groups", i, group[i]);
  const int nlev = ctx->n_done / ctx->opt.obs_stride + 1;
  int* dg = nullptr;
  double* dout = nullptr;
  CK(cudaMallocAsync(&dg, sizeof(int) * nat, ctx->stream));
  CK(cudaMallocAsync(&dout, sizeof(double) * (size_t)nlev * n_groups, ctx->stream));
  CK(cudaMemcpyAsync(dg, group, sizeof(int) * nat, cudaMemcpyHostToDevice, ctx->stream));
  launch_group_charge(T.q, nat, dg, n_groups, nlev, dout, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, dout, sizeof(double) * (size_t)nlev * n_groups, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaFreeAsync(dg, ctx->stream));
  CK(cudaFreeAsync(dout, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

int vgtb_get_initial_density(vgtb_ctx* ctx, int s, int k, double* d_out) {
  if (!ctx) return VGTB_E_INVALID;
  if (s < 0 || s >= (int)ctx->sys.size()) return fail(ctx, VGTB_E_INVALID, "system index %d out of range", s);
  const HostSys& h = ctx->sys[s];
  if (k < 0 || k >= h.nk || !d_out) return fail(ctx, VGTB_E_INVALID, "bad k or NULL output");
  if (!h.density_set) return fail(ctx, VGTB_E_STATE, "no initial density set");
  const size_t NN = (size_t)h.Np * h.Np;
  CK(cudaMemcpy2DAsync(d_out, sizeof(double2) * h.N, h.D0 + k * NN, sizeof(double2) * h.Np, sizeof(double2) * h.N,
                       h.N, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

// State layout: 4 header words (tag, n, items, form), then per item the two
// leapfrog levels (2 Np^2 complex), or for Crank-Nicolson per item C^dagger
// (nocc x Np complex) followed by the two latest SCC shifts of every
// trajectory (2 nat doubles).
long long vgtb_state_size(const vgtb_ctx* ctx) {
  if (!ctx) return -1;
  long long b = 4 * sizeof(long long);
  for (auto& it : ctx->items_h) {
    const HostSys& h = ctx->sys[it.sys];
    b += ctx->cn ? (long long)h.nocc * h.Np * (long long)sizeof(double2)
                 : 2LL * h.Np * h.Np * (long long)sizeof(double2);
  }
  if (ctx->cn)
    for (auto& t : ctx->trj) b += 2LL * ctx->sys[t.sys].nat * (long long)sizeof(double);
  return b;
}

static long long state_form(const vgtb_ctx* ctx) { return ctx->cn ? 2 : (ctx->delta ? 1 : 0); }

int vgtb_get_state(vgtb_ctx* ctx, void* buf, long long bytes) {
  if (!ctx || !buf) return VGTB_E_INVALID;
  if (bytes < vgtb_state_size(ctx)) return fail(ctx, VGTB_E_INVALID, "state buffer too small");
  long long* hd = (long long*)buf;
  hd[0] = 0x7674627374617465LL;  // tag
  hd[1] = ctx->n_done;
  hd[2] = ctx->n_items;
  hd[3] = state_form(ctx);
  char* p = (char*)buf + 4 * sizeof(long long);
  for (auto& it : ctx->items_h) {
    const HostSys& h = ctx->sys[it.sys];
    const size_t bytes_it = ctx->cn ? (size_t)h.nocc * h.Np * sizeof(double2) : 2 * (size_t)h.Np * h.Np * sizeof(double2);
    CK(cudaMemcpyAsync(p, ctx->cn ? (const void*)it.Cd : (const void*)it.D[0], bytes_it, cudaMemcpyDeviceToHost,
                       ctx->stream));
    p += bytes_it;
  }
  if (ctx->cn)
    for (auto& t : ctx->trj) {
      const size_t b = 2 * (size_t)ctx->sys[t.sys].nat * sizeof(double);
      CK(cudaMemcpyAsync(p, t.eps_lv, b, cudaMemcpyDeviceToHost, ctx->stream));
      p += b;
    }
  CK(cudaStreamSynchronize(ctx->stream));
  return VGTB_OK;
}

int vgtb_set_state(vgtb_ctx* ctx, const void* buf, long long bytes) {
  if (!ctx || !buf) return VGTB_E_INVALID;
  if (bytes < vgtb_state_size(ctx)) return fail(ctx, VGTB_E_INVALID, "state buffer too small");
  const long long* hd = (const long long*)buf;
  if (hd[0] != 0x7674627374617465LL || hd[2] != ctx->n_items || hd[3] != state_form(ctx))
    return fail(ctx, VGTB_E_INVALID, "state does not belong to a context of this shape");
  const int n = (int)hd[1];
  for (auto& t : ctx->trj)
    if (t.n_times < n + 1) return fail(ctx, VGTB_E_STATE, "field table shorter than the saved step");
  const char* p = (const char*)buf + 4 * sizeof(long long);
  for (auto& it : ctx->items_h) {
    const HostSys& h = ctx->sys[it.sys];
    const size_t NN = (size_t)h.Np * h.Np;
    if (ctx->cn) {
      CK(cudaMemcpyAsync(it.Cd, p, (size_t)h.nocc * h.Np * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
      p += (size_t)h.nocc * h.Np * sizeof(double2);
      continue;
    }
    CK(cudaMemcpyAsync(it.D[0], p, 2 * NN * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    if (it.dD_p) launch_split_planar(it.D[n & 1], it.dD_p, h.N, h.Np, ctx->stream);
    if (it.dDf) launch_to_f32(it.D[n & 1], it.dDf, (long long)NN, ctx->stream);
    p += 2 * NN * sizeof(double2);
  }
  if (ctx->cn)
    for (auto& t : ctx->trj) {
      const size_t b = 2 * (size_t)ctx->sys[t.sys].nat * sizeof(double);
      CK(cudaMemcpyAsync(t.eps_lv, p, b, cudaMemcpyHostToDevice, ctx->stream));
      p += b;
    }
  CK(cudaMemcpyAsync(ctx->d_step, &n, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->n_done = n;
  return VGTB_OK;
}

int vgtb_profile(vgtb_ctx* ctx, int enable) {
  if (!ctx) return VGTB_E_INVALID;
  ctx->profile = enable != 0;
  for (int c = 0; c < VGTB_K_COUNT; ++c) {
    ctx->prof_ms[c] = 0.0;
    ctx->prof_launch[c] = 0;
  }
  return VGTB_OK;
}

int vgtb_kernel_stats(vgtb_ctx* ctx, long long* launches, double* ms, int n) {
  if (!ctx) return VGTB_E_INVALID;
  for (int c = 0; c < std::min(n, (int)VGTB_K_COUNT); ++c) {
    if (launches) launches[c] = ctx->prof_launch[c];
    if (ms) ms[c] = ctx->prof_ms[c];
  }
  return VGTB_K_COUNT;
}

int vgtb_tile_config(const vgtb_ctx* ctx, int product, int* cfg) {
  if (!ctx || !cfg || (product != 1 && product != 2)) return VGTB_E_INVALID;
  if (!ctx->split) return VGTB_E_STATE;
  if (product == 1 && ctx->bsr) {
    cfg[0] = bsr_group(0);   // atoms per group (output columns / 4)
    cfg[1] = kBsrThreads;    // output rows per CTA
    cfg[2] = 3;              // block-sparse CUDA-core product
    cfg[3] = 0;
    return VGTB_OK;
  }
  if (tc_plan_info(product == 1 ? ctx->tc1 : ctx->tc2, cfg)) return VGTB_E_STATE;
  if (ctx->tcc) cfg[2] += 16;  // both products in one launch
  return VGTB_OK;
}

const char* vgtb_last_error(const vgtb_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void vgtb_destroy(vgtb_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  drop_graph(ctx);
  for (auto e : ctx->ev) cudaEventDestroy(e);
  tc_destroy_chain(ctx->tcc);
  tc_destroy_plan(ctx->tc1);
  tc_destroy_plan(ctx->tc2);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

}  // extern "C"
