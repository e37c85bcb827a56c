// Host side of libqg: input validation, FP64 set-up of the DC network data
// (reduced-Laplacian inverse, PTDF rows at generator buses, line-outage block),
// warp-aligned CSR packs and block spans for the stage kernels, and the C ABI
// declared in include/qg.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "qg_internal.h"
#include "qg_sparse.h"

using namespace qg;

namespace {

thread_local std::string g_create_error;

constexpr int DENSE_MAX_N = 8192;  // the dense inverse used at set-up holds n^2 doubles
constexpr int SPARSE_AUTO_N = 4096; // QG_DC_AUTO picks the sparse factor above this many buses
constexpr int TAIL_DEGREE = 32;     // minimum-degree elimination stops above this degree
constexpr long long CTG_WAVE = 152 * 3;  // contingency blocks resident at once (152 SMs x 3 blocks)
constexpr long long SMALL_PLAN = 65536;  // branch-periods of a plan that takes the latency layouts
constexpr long long CTG_LARGE = 1LL << 22;  // (monitored branch, outage) pairs per period of a large grid

// Contingency-block shape of a plan (stage 2): how many period chunks each 64 x 64 tile is split
// into (ntc) and how many monitored-branch tiles one block walks (mg); 0 picks the heuristic.
struct Knobs {
  int ntc = 0, mg = 0;
};

struct HostInst {
  int n, M, G, Z, T, K, ref, X = 0;
  std::vector<int> from, to, gen_bus, gen_zone, ctg;
  std::vector<int> xf;         // transformer branch ids [X]
  std::vector<int> br_xf;      // branch -> transformer index, -1 for lines [M]
  std::vector<double> tau_lo, tau_hi, phi_lo, phi_hi;
  std::vector<double> r, x, bch, smax, sctg, ca, cb, cr, pmin, pmax, qmin, qmax, ramp, vmin, vmax;
  std::vector<double> dt, load_p, load_q, rreq;
  // device models: consumers, bid blocks (Example 3), on-status with startup / shutdown (Example 2)
  std::vector<int> cons;                         // [G] 1 = consumer
  int L = 0;                                     // bid blocks per device
  std::vector<double> blk_c, blk_w;              // [G x L]
  bool commit = false;
  std::vector<double> c_on, c_su, c_sd, u_init;  // [G]
  // derived (FP64)
  std::vector<double> y, gsr, bsr;
  int Gc = 0;                 // dense DC product columns: generator buses, then transformers
  std::vector<int> gbus;      // distinct generator buses, ascending
  std::vector<int> gen_gb;    // generator -> index into gbus
  std::vector<double> ptdfg;  // M x Gb
  std::vector<double> cload;  // T x M
  std::vector<double> rsum;   // M
  std::vector<double> ltot;   // T
  std::vector<double> lodf;   // M x K
  int Ks = 0;                 // outages each evaluation covers (K without screening)
  std::vector<int> sel;       // their indices into ctg (screening: the current selection)
  // warp packs (code, row) of the two bus CSRs
  std::vector<int> bal_code, bal_row, adj_code, adj_row;
  // sparse DC mode: factor with a dense tail, node positions, gather lists (see qg_sparse.h)
  bool sparse = false;
  int nS = 0, nT = 0, levels = 0;
  std::vector<int> bus_pos, pos_bus, pos_gb, fw_ptr, fw_col, bw_ptr, bw_col, inc_ptr, inc_code, adj_rows;
  std::vector<double> fw_val, bw_val, dinv, sinv, z1;
};

}  // namespace

struct qg_ctx {
  int n_inst = 0;
  qg_options opt{};
  std::vector<HostInst> hi;
  Plan plan{};
  long long n_x = 0;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  Dev<double, double> d64{};
  Dev<float, df32> d32{};
  double *d_obj = nullptr, *d_terms = nullptr;
  void *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
  void *d_xs = nullptr;    // staging for qg_eval_grad_host (Real)
  double *d_xd = nullptr;  // staging doubles
  long long *d_step = nullptr, *d_step0 = nullptr;
  unsigned int *d_ticket = nullptr;
  // cached CUDA graph of one (evaluation + fused Adam) iteration for qg_solve
  cudaGraphExec_t gexec = nullptr;
  cudaGraphExec_t gexec_u = nullptr;  // SOLVE_UNROLL iterations in one graph (same parameters)
  // cached graph of qg_eval_grad_host for one set of pinned host buffers
  cudaGraphExec_t hexec = nullptr;
  const void *h_x = nullptr, *h_obj = nullptr, *h_g = nullptr;
  const void *g_x = nullptr;
  double g_lr = 0, g_b1 = 0, g_b2 = 0;
  double *g_trace = nullptr;
  const double *g_sched = nullptr;
  int g_trace_len = 0;
  // optional per-kernel timing: ev[0..5] bracket the five stage kernels, ev[6] ends a stand-alone Adam step
  bool screen = false;                 // contingency screening (0 < ctg_frac < 1)
  std::vector<long long> lf0;          // per instance: offset of its full line-outage block (screening)
  void *lodf_full = nullptr;           // screening: the full block (element type of d32/d64.lodf)
  double *lodf64_full = nullptr;       // screening, FP64 path: the full exact block
  int *d_sel = nullptr;                // screening: [sum Ks] selected outage indices per instance
  bool profiling = false;
  Knobs knobs{};                       // the contingency-block shape in use (0: heuristic)
  // batch rounding (Alg. 1): fixed flags, distances, projections, the original box (allocated on the
  // first round), and the host copy of the fixed flags
  unsigned char *d_fixed = nullptr;
  double *d_dist = nullptr;
  void *d_proj = nullptr, *d_lo0 = nullptr, *d_hi0 = nullptr;
  int *d_idx = nullptr;
  std::vector<unsigned char> fixed;
  cudaEvent_t ev[N_PHASES + 1] = {};
  std::string err;
};

namespace {

int fail(qg_ctx *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  g_create_error = msg;
  return code;
}

#define CUDA_TRY(h, call)                                                                                      \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess) return fail((h), QG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dalloc(qg_ctx *h, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(*p);
  bounds_register(*p, count * sizeof(T));
  e = cudaMemset(*p, 0, count * sizeof(T));
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
  return QG_OK;
}

template <typename T>
int upload(qg_ctx *h, T **p, const std::vector<T> &v) {
  int rc = dalloc(h, p, v.size());
  if (rc) return rc;
  if (!v.empty()) {
    cudaError_t e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  }
  return QG_OK;
}

bool finite_all(const std::vector<double> &v) {
  for (double a : v)
    if (!std::isfinite(a)) return false;
  return true;
}

// Copy and validate one instance.
int read_instance(qg_ctx *h, const qg_network &N, const qg_horizon &H, const qg_contingencies &C, HostInst &I,
                  int b) {
  auto bad = [&](const std::string &m) { return fail(h, QG_ERR_INVALID_ARG, "instance " + std::to_string(b) + ": " + m); };
  if (N.n_bus < 2 || N.n_branch < 1 || N.n_gen < 1 || N.n_zone < 1 || H.T < 1 || C.K < 0) return bad("sizes out of range");
  if (N.ref_bus < 0 || N.ref_bus >= N.n_bus) return bad("ref_bus out of range");
  {  // per-instance element counts index 32-bit: checked before any array is read
    const long long T = H.T, xf = std::max(N.n_xf, 0), blk = std::max(N.n_blk, 0);
    const long long n_x = T * (2LL * N.n_bus + 4LL * N.n_gen + 2 * xf);  // with an on-status block
    if (n_x > INT32_MAX || T * N.n_branch > INT32_MAX || T * N.n_zone > INT32_MAX ||
        (long long)N.n_gen * blk > INT32_MAX)
      return bad("sizes too large: T (2n + 4G + 2X), T M, T Z and G n_blk must stay below 2^31");
  }
  if (!N.br_from || !N.br_to || !N.br_r || !N.br_x || !N.br_b || !N.s_max || !N.s_max_ctg || !N.gen_bus ||
      !N.gen_zone || !N.cost_a || !N.cost_b || !N.cost_r || !N.pmin || !N.pmax || !N.qmin || !N.qmax || !N.ramp ||
      !N.vmin || !N.vmax || !H.dt || !H.load_p || !H.load_q || !H.reserve_req || (C.K > 0 && !C.branch))
    return bad("null array");
  I.n = N.n_bus; I.M = N.n_branch; I.G = N.n_gen; I.Z = N.n_zone; I.T = H.T; I.K = C.K; I.ref = N.ref_bus;
  const int n = I.n, M = I.M, G = I.G, Z = I.Z, T = I.T, K = I.K;
  I.from.assign(N.br_from, N.br_from + M);
  I.to.assign(N.br_to, N.br_to + M);
  I.gen_bus.assign(N.gen_bus, N.gen_bus + G);
  I.gen_zone.assign(N.gen_zone, N.gen_zone + G);
  I.ctg.assign(C.branch, C.branch + K);
  auto cp = [](const double *p, int cnt) { return std::vector<double>(p, p + cnt); };
  I.r = cp(N.br_r, M); I.x = cp(N.br_x, M); I.bch = cp(N.br_b, M); I.smax = cp(N.s_max, M); I.sctg = cp(N.s_max_ctg, M);
  I.ca = cp(N.cost_a, G); I.cb = cp(N.cost_b, G); I.cr = cp(N.cost_r, G); I.pmin = cp(N.pmin, G);
  I.pmax = cp(N.pmax, G); I.qmin = cp(N.qmin, G); I.qmax = cp(N.qmax, G); I.ramp = cp(N.ramp, G);
  I.vmin = cp(N.vmin, n); I.vmax = cp(N.vmax, n);
  I.dt = cp(H.dt, T); I.load_p = cp(H.load_p, T * n); I.load_q = cp(H.load_q, T * n); I.rreq = cp(H.reserve_req, T * Z);
  for (int j = 0; j < M; ++j) {
    if (I.from[j] < 0 || I.from[j] >= n || I.to[j] < 0 || I.to[j] >= n || I.from[j] == I.to[j])
      return bad("branch " + std::to_string(j) + " has a bad end bus");
    if (!(I.x[j] > 0.0) || !(I.r[j] >= 0.0)) return bad("branch " + std::to_string(j) + " needs x > 0, r >= 0");
    if (!(I.smax[j] >= 0.0) || !(I.sctg[j] >= 0.0)) return bad("negative rating");
  }
  for (int g = 0; g < G; ++g) {
    if (I.gen_bus[g] < 0 || I.gen_bus[g] >= n) return bad("generator bus out of range");
    if (I.gen_zone[g] < 0 || I.gen_zone[g] >= Z) return bad("generator zone out of range");
    if (I.pmin[g] > I.pmax[g] || I.qmin[g] > I.qmax[g] || I.pmax[g] < 0) return bad("generator limits");
  }
  for (int i = 0; i < n; ++i)
    if (I.vmin[i] > I.vmax[i]) return bad("voltage limits");
  for (int t = 0; t < T; ++t)
    if (!(I.dt[t] > 0.0)) return bad("dt must be > 0");
  std::vector<char> seen(M, 0);
  for (int k = 0; k < K; ++k) {
    if (I.ctg[k] < 0 || I.ctg[k] >= M) return bad("contingency branch out of range");
    if (seen[I.ctg[k]]) return bad("duplicate contingency");
    seen[I.ctg[k]] = 1;
  }
  if (N.n_xf < 0 || N.n_xf > M) return bad("n_xf out of range");
  I.X = N.n_xf;
  I.br_xf.assign(M, -1);
  if (I.X > 0) {
    if (!N.xf_branch || !N.tau_min || !N.tau_max || !N.phi_min || !N.phi_max) return bad("null transformer array");
    I.xf.assign(N.xf_branch, N.xf_branch + I.X);
    I.tau_lo = cp(N.tau_min, I.X); I.tau_hi = cp(N.tau_max, I.X);
    I.phi_lo = cp(N.phi_min, I.X); I.phi_hi = cp(N.phi_max, I.X);
    for (int q = 0; q < I.X; ++q) {
      const int j = I.xf[q];
      if (j < 0 || j >= M) return bad("transformer branch out of range");
      if (I.br_xf[j] >= 0) return bad("duplicate transformer branch");
      I.br_xf[j] = q;
      if (!(I.tau_lo[q] > 0.0) || !(I.tau_lo[q] <= I.tau_hi[q]) || !(I.phi_lo[q] <= I.phi_hi[q]))
        return bad("transformer limits");
    }
  }
  I.cons.assign(G, 0);
  if (N.dev_cons)
    for (int g = 0; g < G; ++g) I.cons[g] = N.dev_cons[g] != 0;
  if (N.n_blk < 0 || N.n_blk > 64) return bad("n_blk out of range [0, 64]");
  I.L = N.n_blk;
  if (I.L > 0) {
    if (!N.blk_price || !N.blk_width) return bad("null bid-block array");
    I.blk_c = cp(N.blk_price, G * I.L);
    I.blk_w = cp(N.blk_width, G * I.L);
    for (double w : I.blk_w)
      if (!(w >= 0.0)) return bad("bid-block widths must be >= 0");
  }
  if (N.commit != 0 && N.commit != 1) return bad("commit must be 0 or 1");
  I.commit = N.commit == 1;
  if (I.commit) {
    if (!N.c_on || !N.c_su || !N.c_sd || !N.u_init) return bad("null commitment array");
    I.c_on = cp(N.c_on, G); I.c_su = cp(N.c_su, G); I.c_sd = cp(N.c_sd, G); I.u_init = cp(N.u_init, G);
    for (int g = 0; g < G; ++g)
      if (!(I.c_on[g] >= 0.0) || !(I.c_su[g] >= 0.0) || !(I.c_sd[g] >= 0.0) || !(I.u_init[g] >= 0.0) ||
          !(I.u_init[g] <= 1.0))
        return bad("commitment costs must be >= 0 and u_init in [0, 1]");
  }
  for (auto *v : {&I.r, &I.x, &I.bch, &I.smax, &I.sctg, &I.ca, &I.cb, &I.cr, &I.pmin, &I.pmax, &I.qmin, &I.qmax,
                  &I.ramp, &I.vmin, &I.vmax, &I.dt, &I.load_p, &I.load_q, &I.rreq, &I.tau_lo, &I.tau_hi, &I.phi_lo,
                  &I.phi_hi, &I.blk_c, &I.blk_w, &I.c_on, &I.c_su, &I.c_sd})
    if (!finite_all(*v)) return bad("non-finite input");
  return QG_OK;
}

// Warp packs of a bus CSR: rows (buses) in order, each row's entries contiguous and never
// straddling a pack of PACK lanes; unused lanes are pads (code kind 3, row -1).
bool pack_rows(const std::vector<std::vector<int>> &rows, std::vector<int> &code, std::vector<int> &row) {
  code.clear();
  row.clear();
  int fill = 0;
  for (size_t i = 0; i < rows.size(); ++i) {
    const int len = (int)rows[i].size();
    if (len > PACK) return false;
    if (fill + len > PACK) {
      for (; fill < PACK; ++fill) { code.push_back(3); row.push_back(-1); }
      fill = 0;
    }
    for (int c : rows[i]) { code.push_back(c); row.push_back((int)i); }
    fill += len;
    if (fill == PACK) fill = 0;
  }
  if (fill > 0)
    for (; fill < PACK; ++fill) { code.push_back(3); row.push_back(-1); }
  return true;
}

int build_packs(qg_ctx *h, HostInst &I, int b);

// Error for outages whose SMW denominator vanishes (the outage islands the grid).
int islanding_error(qg_ctx *h, int b, const std::vector<int> &bad_k) {
  std::string s = "instance " + std::to_string(b) + ": outage of branch(es)";
  for (size_t q = 0; q < bad_k.size() && q < 8; ++q) s += " " + std::to_string(bad_k[q]);
  s += " islands the grid (|1 - PTDF_kk| < 1e-9)";
  return fail(h, QG_ERR_ISLANDING, s);
}

// Sparse DC set-up (Sec. II-E) for large grids, all in FP64: the factor Yhat = L diag(D_S, S) L^T
// with minimum-degree elimination up to degree TAIL_DEGREE and the inverse of the dense tail
// Schur complement S; node positions (eliminated nodes in order, then the tail); the forward
// gather rows of [M1; M2] and the backward gather rows (the reach columns, see qg_sparse.h);
// z1 = Yhat^-1 1 and PTDF 1 = y_m (z1_f - z1_o) for the uniform slack; and the line-outage block
// L[m,k] = y_m a_m^T u_k / (1 - y_k a_k^T u_k) from the solves u_k = Yhat^-1 a_k.  No PTDF.
int build_dc_sparse(qg_ctx *h, HostInst &I, int b, const std::vector<int> &red,
                    std::vector<std::map<int, double>> &off, std::vector<double> &diag) {
  const int n = I.n, M = I.M, K = I.K, nr = n - 1;
  TailLDL F;
  if (!F.factor(nr, off, diag, TAIL_DEGREE))
    return fail(h, QG_ERR_ISLANDING, "instance " + std::to_string(b) + ": the DC Laplacian is singular (disconnected grid)");
  off.clear();
  I.nS = F.n_sparse();
  I.nT = (int)F.tail.size();
  I.levels = F.levels;
  const std::vector<int> pos = F.positions();  // reduced id -> position
  I.bus_pos.assign(n, -1);
  I.pos_bus.assign(nr, -1);
  I.pos_gb.assign(nr, -1);
  std::vector<int> gmap(n, -1);
  for (size_t q = 0; q < I.gbus.size(); ++q) gmap[I.gbus[q]] = (int)q;
  for (int i = 0; i < n; ++i)
    if (red[i] >= 0) {
      const int p = pos[red[i]];
      I.bus_pos[i] = p;
      I.pos_bus[p] = i;
      I.pos_gb[p] = gmap[i];
    }
  std::vector<std::vector<std::pair<int, double>>> R;
  F.reach_columns(R);
  // backward rows: the reach columns themselves; forward rows: their transpose
  I.bw_ptr.assign(1, 0);
  I.bw_col.clear();
  I.bw_val.clear();
  std::vector<int> cnt(nr, 0);
  for (int q = 0; q < I.nS; ++q) {
    for (auto &e : R[q]) {
      I.bw_col.push_back(e.first);
      I.bw_val.push_back(e.second);
      ++cnt[e.first];
    }
    I.bw_ptr.push_back((int)I.bw_col.size());
  }
  I.fw_ptr.assign(nr + 1, 0);
  for (int p = 0; p < nr; ++p) I.fw_ptr[p + 1] = I.fw_ptr[p] + cnt[p];
  I.fw_col.assign(I.fw_ptr[nr], 0);
  I.fw_val.assign(I.fw_ptr[nr], 0.0);
  std::vector<int> fill(I.fw_ptr.begin(), I.fw_ptr.end() - 1);
  for (int q = 0; q < I.nS; ++q)
    for (auto &e : R[q]) {
      I.fw_col[fill[e.first]] = q;
      I.fw_val[fill[e.first]++] = e.second;
    }
  I.dinv.resize(I.nS);
  for (int q = 0; q < I.nS; ++q) I.dinv[q] = 1.0 / F.cols[q].d;
  I.sinv = F.Sinv;
  I.Gc = (int)I.gbus.size();
  // adjoint back-gather rows: eliminated positions at generator buses or transformer ends
  std::vector<char> need(nr, 0);
  for (int q = 0; q < I.nS; ++q)
    if (I.pos_gb[q] >= 0) need[q] = 1;
  for (int q = 0; q < I.X; ++q)
    for (int bus : {I.from[I.xf[q]], I.to[I.xf[q]]})
      if (I.bus_pos[bus] >= 0) need[I.bus_pos[bus]] = 1;
  I.adj_rows.clear();
  for (int q = 0; q < I.nS; ++q)
    if (need[q]) I.adj_rows.push_back(q);
  // incident branches per position (+ at the from-end)
  std::vector<std::vector<int>> inc(nr);
  for (int j = 0; j < M; ++j) {
    if (I.bus_pos[I.from[j]] >= 0) inc[I.bus_pos[I.from[j]]].push_back(j << 1);
    if (I.bus_pos[I.to[j]] >= 0) inc[I.bus_pos[I.to[j]]].push_back(j << 1 | 1);
  }
  I.inc_ptr.assign(1, 0);
  I.inc_code.clear();
  for (int p = 0; p < nr; ++p) {
    I.inc_code.insert(I.inc_code.end(), inc[p].begin(), inc[p].end());
    I.inc_ptr.push_back((int)I.inc_code.size());
  }
  // z1 = Yhat^-1 1, PTDF 1
  std::vector<double> ones(nr, 1.0);
  F.solve(ones.data());
  I.z1.assign(nr, 0.0);
  for (int r = 0; r < nr; ++r) I.z1[pos[r]] = ones[r];
  auto zb = [&](int bus) { return red[bus] >= 0 ? ones[red[bus]] : 0.0; };
  I.rsum.assign(M, 0.0);
  for (int m = 0; m < M; ++m) I.rsum[m] = I.y[m] * (zb(I.from[m]) - zb(I.to[m]));
  // line-outage block from K solves
  I.lodf.assign((size_t)M * K, 0.0);
  std::vector<char> bad(K, 0);
  parallel_for(K, [&](int k) {
    const int jk = I.ctg[k];
    std::vector<double> u(nr, 0.0);
    if (red[I.from[jk]] >= 0) u[red[I.from[jk]]] += 1.0;
    if (red[I.to[jk]] >= 0) u[red[I.to[jk]]] -= 1.0;
    F.solve(u.data());
    auto ub = [&](int bus) { return red[bus] >= 0 ? u[red[bus]] : 0.0; };
    const double den = 1.0 - I.y[jk] * (ub(I.from[jk]) - ub(I.to[jk]));
    if (std::fabs(den) < 1e-9) {
      bad[k] = 1;
      return;
    }
    for (int m = 0; m < M; ++m) I.lodf[(size_t)m * K + k] = I.y[m] * (ub(I.from[m]) - ub(I.to[m])) / den;
  });
  std::vector<int> bad_k;
  for (int k = 0; k < K; ++k)
    if (bad[k]) bad_k.push_back(I.ctg[k]);
  if (!bad_k.empty()) return islanding_error(h, b, bad_k);
  return QG_OK;
}

// DC network set-up (Sec. II-E), all in FP64:
//   y_j = -b_sr = x / (r^2 + x^2);  Yhat = E_hat^T Y_x E_hat (reference bus removed);
//   Z = Yhat^-1 (zero row and column at the reference bus), from sparse LDL^T solves;
//   PTDF[m, i] = y_m (Z[f_m, i] - Z[o_m, i]) (flow on m per unit injection at i, withdrawn at the reference);
//   line-outage block L[m, k] = PTDF u_k / (1 - PTDF_kk), u_k = Z (e_f - e_o): the rank-1 SMW
//   correction of Eq. rank_correct written on branch flows.
// Kept for the kernels: PTDF columns of the generator buses, PTDF load_t and PTDF 1.
int build_dc(qg_ctx *h, HostInst &I, int b) {
  const int n = I.n, M = I.M, K = I.K, T = I.T;
  // generator buses
  std::vector<int> gmap(n, -1);
  I.gbus.clear();
  for (int g = 0; g < I.G; ++g) gmap[I.gen_bus[g]] = 0;
  for (int i = 0; i < n; ++i)
    if (gmap[i] == 0) {
      gmap[i] = (int)I.gbus.size();
      I.gbus.push_back(i);
    }
  I.gen_gb.resize(I.G);
  for (int g = 0; g < I.G; ++g) I.gen_gb[g] = gmap[I.gen_bus[g]];
  I.ltot.assign(T, 0.0);
  for (int t = 0; t < T; ++t)
    for (int i = 0; i < n; ++i) I.ltot[t] += I.load_p[(size_t)t * n + i];
  I.y.resize(M); I.gsr.resize(M); I.bsr.resize(M);
  for (int j = 0; j < M; ++j) {
    const double den = I.r[j] * I.r[j] + I.x[j] * I.x[j];
    I.y[j] = I.x[j] / den;
    I.gsr[j] = I.r[j] / den;
    I.bsr[j] = -I.x[j] / den;
  }
  std::vector<int> red(n, -1);
  int c = 0;
  for (int i = 0; i < n; ++i)
    if (i != I.ref) red[i] = c++;
  const int nr = n - 1;
  std::vector<std::map<int, double>> off(nr);
  std::vector<double> diag(nr, 0.0);
  for (int j = 0; j < M; ++j) {
    const int a = red[I.from[j]], bb = red[I.to[j]];
    if (a >= 0) diag[a] += I.y[j];
    if (bb >= 0) diag[bb] += I.y[j];
    if (a >= 0 && bb >= 0) {
      off[a][bb] -= I.y[j];
      off[bb][a] -= I.y[j];
    }
  }
  if (I.sparse) {
    int rc = build_dc_sparse(h, I, b, red, off, diag);
    if (rc) return rc;
    return build_packs(h, I, b);
  }
  SparseLDL F;
  if (!F.factor(nr, off, diag))
    return fail(h, QG_ERR_ISLANDING, "instance " + std::to_string(b) + ": the DC Laplacian is singular (disconnected grid)");
  if (n > DENSE_MAX_N)
    return fail(h, QG_ERR_UNSUPPORTED, "instance " + std::to_string(b) + ": n = " + std::to_string(n) +
                                           " exceeds the dense set-up limit " + std::to_string(DENSE_MAX_N));
  std::vector<double> Zm((size_t)n * n, 0.0);
  std::vector<double> col(nr);
  for (int cc = 0; cc < nr; ++cc) {
    std::fill(col.begin(), col.end(), 0.0);
    col[cc] = 1.0;
    F.solve(col.data());
    const int bc = cc < I.ref ? cc : cc + 1;
    for (int rr = 0; rr < nr; ++rr) Zm[(size_t)(rr < I.ref ? rr : rr + 1) * n + bc] = col[rr];
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double v = 0.5 * (Zm[(size_t)i * n + j] + Zm[(size_t)j * n + i]);
      Zm[(size_t)i * n + j] = v;
      Zm[(size_t)j * n + i] = v;
    }
  const int Gb = (int)I.gbus.size();
  const int Gc = Gb + I.X;
  I.Gc = Gc;
  // PTDF rows: generator-bus columns, then per transformer x the column -PSDF[:, x] =
  // -Y_x E_hat Yhat^-1 a_x (flow change per unit phase-shift flow b_x, Eq. Yb_solve with
  // c_t = p_inj - E^T b_t), load products and row sums
  I.ptdfg.assign((size_t)M * Gc, 0.0);
  I.cload.assign((size_t)T * M, 0.0);
  I.rsum.assign(M, 0.0);
  std::vector<double> row(n);
  for (int m = 0; m < M; ++m) {
    const double *zf = &Zm[(size_t)I.from[m] * n], *zo = &Zm[(size_t)I.to[m] * n];
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
      row[i] = I.y[m] * (zf[i] - zo[i]);
      s += row[i];
    }
    I.rsum[m] = s;
    for (int q = 0; q < Gb; ++q) I.ptdfg[(size_t)m * Gc + q] = row[I.gbus[q]];
    for (int q = 0; q < I.X; ++q) {
      const int fx = I.from[I.xf[q]], ox = I.to[I.xf[q]];
      I.ptdfg[(size_t)m * Gc + Gb + q] = -(row[fx] - row[ox]);
    }
    for (int t = 0; t < T; ++t) {
      const double *lp = &I.load_p[(size_t)t * n];
      double a = 0.0;
      for (int i = 0; i < n; ++i) a += row[i] * lp[i];
      I.cload[(size_t)t * M + m] = a;
    }
  }
  // line-outage block
  I.lodf.assign((size_t)M * K, 0.0);
  std::vector<int> bad_k;
  for (int k = 0; k < K; ++k) {
    const int jk = I.ctg[k];
    const int fk = I.from[jk], ok = I.to[jk];
    auto u = [&](int bus) { return Zm[(size_t)bus * n + fk] - Zm[(size_t)bus * n + ok]; };
    const double den = 1.0 - I.y[jk] * (u(fk) - u(ok));
    if (std::fabs(den) < 1e-9) {
      bad_k.push_back(jk);
      continue;
    }
    for (int m = 0; m < M; ++m) I.lodf[(size_t)m * K + k] = I.y[m] * (u(I.from[m]) - u(I.to[m])) / den;
  }
  if (!bad_k.empty()) return islanding_error(h, b, bad_k);
  return build_packs(h, I, b);
}

// Bus CSR packs: balance (branch ends, then generators) and branch-end adjoints.
int build_packs(qg_ctx *h, HostInst &I, int b) {
  const int n = I.n, M = I.M;
  std::vector<std::vector<int>> bal(n), adj(n);
  for (int j = 0; j < M; ++j) {
    bal[I.from[j]].push_back(j << 2 | 0);
    bal[I.to[j]].push_back(j << 2 | 1);
    adj[I.from[j]].push_back(j << 2 | 0);
    adj[I.to[j]].push_back(j << 2 | 1);
  }
  for (int g = 0; g < I.G; ++g) bal[I.gen_bus[g]].push_back(g << 2 | 2);
  if (!pack_rows(bal, I.bal_code, I.bal_row) || !pack_rows(adj, I.adj_code, I.adj_row))
    return fail(h, QG_ERR_UNSUPPORTED, "instance " + std::to_string(b) + ": a bus has more than 32 incident entries");
  return QG_OK;
}

template <typename Real>
std::vector<Real> cast(const std::vector<double> &v) {
  return std::vector<Real>(v.begin(), v.end());
}

inline df32 split(double v) {
  df32 r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

template <typename Dc>
std::vector<Dc> to_dc(const std::vector<double> &v);
template <>
std::vector<double> to_dc<double>(const std::vector<double> &v) { return v; }
template <>
std::vector<df32> to_dc<df32>(const std::vector<double> &v) {
  std::vector<df32> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = split(v[i]);
  return o;
}

// A stage holds at most three spans per instance (stage 1: DC flows, branches, zones) plus one
// for the sparse solver's adjoint right-hand side, so MAXB instances never overflow the table.
static_assert(MAXSPAN >= 3 * MAXB + 1, "span table too small for MAXB instances");

void add_span(Spans &S, int per_t, int nt, int inst, int role) {
  if (per_t <= 0 || nt <= 0) return;
  Span &s = S.s[S.n++];
  s.first = S.n_blocks;
  s.per_t = per_t;
  s.nt = nt;
  s.inst = inst;
  s.role = role;
  S.n_blocks += per_t * nt;
}

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Instance table, spans of the five stage kernels and objective-slot owners.
int build_plan(qg_ctx *h, std::vector<int> &slot_map, const Knobs &kn) {
  Plan &P = h->plan;
  const int B = h->n_inst;
  std::memset(&P, 0, sizeof(P));
  P.tab.n_inst = B;
  long long x0 = 0, tb0 = 0, tm0 = 0, tg0 = 0, tz0 = 0, tk0 = 0, pg0 = 0, l0 = 0, pm0 = 0, pk0 = 0, gi0 = 0, tx0 = 0,
            pf0 = 0, lm0 = 0, rm0 = 0;
  int xf0 = 0;
  // Contingency block shape, shared by the batch: about one wave of CTG_WAVE blocks when the
  // 64 x 64 tiles are few (the periods split across blocks), several waves when they are many
  // (tiles grouped per block, so fewer column partials are written and summed).
  long long tiles = 0;
  for (int b = 0; b < B; ++b)
    if (h->hi[b].Ks > 0) tiles += (long long)ceil_div(h->hi[b].M, CT_BM) * ceil_div(h->hi[b].Ks, CT_BK);
  // heuristic: about one wave of blocks when tiles are few; at most 24 periods per block (the shared
  // memory of longer chunks leaves fewer than 3 blocks on an SM)
  int maxT_all = 1;
  for (int b = 0; b < B; ++b) maxT_all = std::max(maxT_all, h->hi[b].T);
  const int ntc_all = kn.ntc > 0 ? kn.ntc
                                 : (int)std::max({1LL, tiles > 0 ? CTG_WAVE / tiles : 1LL,
                                                  (long long)ceil_div(maxT_all, 24)});
  // at most ~64 column partials per outage for stage 3 to sum serially
  int max_nmt = 0;
  for (int b = 0; b < B; ++b) max_nmt = std::max(max_nmt, ceil_div(h->hi[b].M, CT_BM));
  const int mg_all = kn.mg > 0 ? kn.mg
                               : (int)std::max({1LL, tiles / (4LL * CTG_WAVE), (long long)ceil_div(max_nmt, 64)});
  // Small plans (at most SMALL_PLAN branch-periods in all) are latency bound: on the mixed path they
  // take layouts that cut dependent memory rounds at the price of some repeated work (the bus
  // balances in stage 1 recompute the branch flows; stage 3 splits each branch's sums over four
  // threads; stage 4's warps form the adjoint products and update the devices at once, one objective
  // slot per block).  Larger plans are throughput bound and keep the leaner layouts.
  long long bp = 0;
  for (int b = 0; b < B; ++b) bp += (long long)h->hi[b].M * h->hi[b].T;
  const bool small_mixed = h->opt.precision == QG_MIXED && bp <= SMALL_PLAN;
  // bound test of the contingency screen: on unless switched off.  The on-demand path pays where most
  // (warp, chunk) pairs pass the test, as on large meshed grids, whose line-outage rows are mostly
  // small entries: by default it is taken when instances of at least CTG_LARGE (monitored branch,
  // outage) pairs per period hold at least half of the plan's elements; otherwise the eager path
  // (each tile staged and loaded up front)
  long long el_all = 0, el_large = 0;
  for (int b = 0; b < B; ++b) {
    const long long mk = (long long)h->hi[b].M * h->hi[b].Ks, el = mk * h->hi[b].T;
    el_all += el;
    if (mk >= CTG_LARGE) el_large += el;
  }
  // (on small grids the test clears too few chunks to pay for itself: no test by default)
  const int cb = h->opt.ctg_bound;
  const int ctg_lazy = cb == QG_CTG_BOUND_LAZY || (cb == QG_CTG_BOUND_AUTO && el_all > 0 && 2 * el_large >= el_all);
  const int ctg_bound = ctg_lazy || cb == QG_CTG_BOUND_EAGER;
  P.tab.s3q = small_mixed ? S3_SPLIT_MAX : 1;
  int bus0 = 0, br0 = 0, gen0 = 0, zone0 = 0, ctg0 = 0, gb0 = 0, tp0 = 0, bal0 = 0, adj0 = 0;
  for (int b = 0; b < B; ++b) {
    const HostInst &H = h->hi[b];
    Inst &D = P.tab.I[b];
    D.n = H.n; D.M = H.M; D.G = H.G; D.Z = H.Z; D.T = H.T; D.K = H.Ks; D.Gb = (int)H.gbus.size();
    D.Kp = ceil_div(H.Ks, 4) * 4;
    D.X = H.X; D.xf0 = xf0; D.Gc = H.Gc; D.tx0 = tx0;
    D.xtau0 = x0 + (long long)H.T * (2LL * H.n + 3LL * H.G);
    D.xu0 = D.xtau0 + 2LL * H.T * H.X;
    D.uc = H.commit ? 1 : 0;
    D.bus0 = bus0; D.br0 = br0; D.gen0 = gen0; D.zone0 = zone0; D.ctg0 = ctg0; D.gb0 = gb0; D.tp0 = tp0;
    D.n_mt = ceil_div(H.M, CT_BM);
    D.n_kt = ceil_div(H.Ks, CT_BK);
    D.ctg_mg = std::min(mg_all, D.n_mt);
    D.n_mg = ceil_div(D.n_mt, D.ctg_mg);
    D.ctg_tb = ceil_div(H.T, std::min(ntc_all, H.T));
    D.ctg_ntc = ceil_div(H.T, D.ctg_tb);
    // latency layouts of small plans on the mixed path (see `small` below): four threads per
    // branch-period in stage 3, two CSR packs per warp in stage 4
    D.s4p = small_mixed ? S4_PACKS : 1;
    D.n_sb = ceil_div(H.M, NTHR / P.tab.s3q);
    D.bal0 = bal0; D.n_bal_pack = (int)H.bal_code.size() / PACK;
    D.adj0 = adj0; D.n_adj_pack = (int)H.adj_code.size() / PACK;
    D.x0 = x0; D.tb0 = tb0; D.tm0 = tm0; D.tg0 = tg0; D.tz0 = tz0; D.tk0 = tk0; D.pg0 = pg0; D.l0 = l0;
    D.pm0 = pm0; D.pk0 = pk0; D.gi0 = gi0; D.pf0 = pf0; D.lm0 = lm0; D.rm0 = rm0;
    D.ctg_bound = ctg_bound; D.ctg_lazy = ctg_lazy;
    D.inv_n = 1.0 / H.n;
    D.hours = 0.0;
    for (int t = 0; t < H.T; ++t) D.hours += H.dt[t];
    D.nfloor_ctg = (double)H.M * H.Ks - H.Ks;
    x0 += (long long)H.T * (2LL * H.n + 3LL * H.G + 2LL * H.X + (H.commit ? H.G : 0));
    tx0 += (long long)H.T * H.X; xf0 += H.X;
    tb0 += (long long)H.T * H.n; tm0 += (long long)H.T * H.M; tg0 += (long long)H.T * H.G;
    tz0 += (long long)H.T * H.Z; tk0 += (long long)H.T * H.Ks; pg0 += (long long)H.M * D.Gc; l0 += (long long)H.M * D.Kp;
    pf0 += (long long)D.n_kt * H.T * D.n_mt;
    lm0 += (long long)D.n_kt * 4 * D.n_mt * CT_BM;
    rm0 += (long long)H.T * D.n_mt * CT_BM;  // ctg_ntc ceil(ctg_tb / 8) <= T chunks, whatever the shape
    P.ctg_lazy = ctg_lazy;
    P.ctg_bound = ctg_bound;
    pm0 += (long long)D.n_kt * H.T * H.M; pk0 += (long long)D.n_mg * H.T * H.Ks; gi0 += (long long)H.T * (D.Gc + 1);
    bus0 += H.n; br0 += H.M; gen0 += H.G; zone0 += H.Z; ctg0 += H.Ks; gb0 += D.Gb; tp0 += H.T;
    bal0 += (int)H.bal_code.size(); adj0 += (int)H.adj_code.size();
    P.maxT = std::max(P.maxT, H.T);
    P.maxTB = std::max(P.maxTB, D.ctg_tb);
  }
  P.n_x = x0;
  auto &I = P.tab.I;
  // roles with the longest blocks first in each launch
  const HostInst &H0 = h->hi[0];
  P.sp = H0.sparse ? 1 : 0;
  if (P.sp) {
    const int nr = H0.n - 1;
    P.sp_inj_blocks = ceil_div((long long)nr * H0.T, NTHR);
    P.sp_fw_blocks = ceil_div(H0.nS, NTHR / 32) + H0.nT;  // eliminated rows 8 per block, tail rows 1 per block
    // column splits: about two waves of tail blocks, at least SP_BK columns per split
    const int n_rt = ceil_div(H0.nT, SP_RB);
    const int ks0 = n_rt > 0 ? std::max(1, std::min(ceil_div(2 * CTG_WAVE, n_rt), ceil_div(H0.nT, SP_BK))) : 1;
    P.sp_tail_kc = std::max(SP_BK, ceil_div(ceil_div(H0.nT, ks0), SP_BK) * SP_BK);
    P.sp_tail_ks = std::max(1, ceil_div(H0.nT, P.sp_tail_kc));
    P.sp_tail_blocks = n_rt * P.sp_tail_ks;
    P.sp_bw_blocks = ceil_div(H0.nS, NTHR / 32);
    P.sp_bwa_blocks = ceil_div((long long)H0.adj_rows.size(), NTHR / 32);
  }
  const int dcf = P.sp ? R_SDCF : R_DCF;
  for (int b = 0; b < B; ++b) add_span(P.s1, ceil_div(I[b].M, DCF_BM), ceil_div(I[b].T, DCF_TC), b, dcf);
  for (int b = 0; b < B; ++b) add_span(P.s1, ceil_div(I[b].M, NTHR), I[b].T, b, R_BRANCH);
  // bus balances: stage 1 on the mixed path (each branch end's flow recomputed in place: the balance
  // does not wait for the branch role); stage 2 on the FP64 path (from stage 1's flows)
  const bool bal1 = small_mixed;
  if (bal1)
    for (int b = 0; b < B; ++b) add_span(P.s1, ceil_div(I[b].n_bal_pack, PACKS_PER_BLOCK), I[b].T, b, R_BUS);
  for (int b = 0; b < B; ++b) add_span(P.s1, I[b].Z, I[b].T, b, R_ZONE);
  for (int b = 0; b < B; ++b) add_span(P.s2, I[b].ctg_ntc * I[b].n_mg * I[b].n_kt, I[b].K > 0 ? 1 : 0, b, R_CTG);
  if (!bal1) {
    // a stage-2 bus-balance block is a few microseconds of work: on large plans each covers several
    // periods, so that they stay within about four waves of the launch's blocks (they take the
    // contingency blocks' shared memory, so an SM holds as few of them)
    long long nbus = 0;
    for (int b = 0; b < B; ++b) nbus += (long long)ceil_div(I[b].n_bal_pack, PACKS_PER_BLOCK) * I[b].T;
    const int tc = (int)std::max(1LL, std::min(8LL, nbus / (4 * CTG_WAVE)));
    for (int b = 0; b < B; ++b) {
      I[b].bus_tc = tc;
      add_span(P.s2, ceil_div(I[b].n_bal_pack, PACKS_PER_BLOCK), ceil_div(I[b].T, tc), b, R_BUS);
    }
  }
  // objective slots: the blocks of s1 and s2 in launch order, renumbered instance-major so that each
  // instance's slots are one contiguous range; then the fold slots of stage 3 (one per fold block:
  // the sum of up to NTHR stage-1/2 slots of one instance) and one slot per stage-5 device block
  std::vector<int> owner;
  for (const Spans *S : {&P.s1, &P.s2})
    for (int k = 0; k < S->n; ++k)
      for (int q = 0; q < S->s[k].per_t * S->s[k].nt; ++q) owner.push_back(S->s[k].inst);
  std::vector<int> count(B, 0);
  for (int o : owner) ++count[o];
  int lo = 0, fold_slot = 0;
  for (int b = 0; b < B; ++b) {
    I[b].obj_lo = lo;
    I[b].obj_n = count[b];
    lo += count[b];
    I[b].fold_nb = ceil_div(count[b], NTHR);
    I[b].fold_slot0 = fold_slot;
    fold_slot += I[b].fold_nb;
  }
  P.n_fold_slots = fold_slot;
  slot_map.assign(owner.size(), 0);
  std::vector<int> next(B);
  for (int b = 0; b < B; ++b) next[b] = I[b].obj_lo;
  for (size_t q = 0; q < owner.size(); ++q) slot_map[q] = next[owner[q]]++;
  // stage 3: the fold blocks first (they start while the branch blocks are dispatched), then branches
  for (int b = 0; b < B; ++b) add_span(P.s3, I[b].fold_nb, 1, b, R_OBJ);
  for (int b = 0; b < B; ++b) add_span(P.s3, I[b].n_sb, I[b].T, b, R_BRANCH);
  // adjoint DC products and devices.  Dense mode: one warp per (period, generator bus or transformer
  // column) in stage 4 computes the adjoint product; on the mixed path the warp also updates the
  // devices at the bus (stage 4 is the last stage); the FP64 path leaves the devices to stage 5 blocks
  // of 32 (period, device) pairs, so that each warp's FP64 instructions serve 32 devices.  Sparse
  // mode: the adjoint solve follows stage 4, and stage 5 updates the devices (FP64 path: one warp of
  // pairs per block; mixed path: a full block of pairs), then the transformers.
  const bool fuse = !P.sp && small_mixed;
  P.tab.fuse = fuse ? 1 : 0;
  int gen_slot = 0;
  if (!P.sp)
    for (int b = 0; b < B; ++b) {
      const int per_t = ceil_div(I[b].Gc, NTHR / 32);
      if (fuse) {
        I[b].gen_first = P.s4.n_blocks;
        I[b].gen_pb = 0;
        I[b].gen_nb = per_t * I[b].T;
        I[b].gen_slot0 = gen_slot;
        gen_slot += I[b].gen_nb;
      }
      add_span(P.s4, per_t, I[b].T, b, R_GBUS);
    }
  else
    add_span(P.s4, ceil_div(H0.n - 1, 32), ceil_div(H0.T, DCF_TC), 0, R_SDCA);
  if (!fuse) {
    // FP64: one warp of pairs per block (GB300's FP64 pipe costs as much for a warp with one active
    // lane as for a full one), 8 pairs of four lanes each without on-status, else 32 of one
    for (int b = 0; b < B; ++b) {
      const int gen_pb = h->opt.precision == QG_FP64 ? (I[b].uc ? 32 : 8) : NTHR;
      I[b].gen_first = P.s5.n_blocks;
      I[b].gen_pb = gen_pb;
      I[b].gen_nb = ceil_div((long long)I[b].T * I[b].G, gen_pb);
      I[b].gen_slot0 = gen_slot;
      gen_slot += I[b].gen_nb;
      add_span(P.s5, I[b].gen_nb, 1, b, R_GEN);
    }
    for (int b = 0; b < B; ++b) add_span(P.s5, ceil_div(I[b].X, NTHR), I[b].T, b, R_XF);
  }
  for (int b = 0; b < B; ++b) add_span(P.s4, ceil_div(I[b].n_adj_pack, PACKS_PER_BLOCK * I[b].s4p), I[b].T, b, R_BUS);
  P.n_gen_slots = gen_slot;
  return QG_OK;
}

// Compacted line-outage block of one instance: column j < Ks is the full block's column sel[j];
// columns up to the padded stride are `pad` (NaN for the screening copies).
template <typename E>
__global__ void k_lodf_gather(const E *__restrict__ full, E *__restrict__ comp, const int *__restrict__ sel, int M,
                              int Kpf, int Ks, int Kpc, E pad) {
  const long long n = (long long)M * Kpc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / Kpc), j = (int)(i % Kpc);
    comp[i] = j < Ks ? full[(long long)m * Kpf + sel[j]] : pad;
  }
}

template <typename E>
cudaError_t launch_gather(const void *full, const void *comp, const int *sel, long long f0, long long c0, int M, int Kpf,
                          int Ks, int Kpc, E pad, cudaStream_t s) {
  const long long n = (long long)M * Kpc;
  const int nb = (int)std::max(1LL, std::min((n + 255) / 256, 152LL * 16));
  k_lodf_gather<E><<<nb, 256, 0, s>>>(static_cast<const E *>(full) + f0, const_cast<E *>(static_cast<const E *>(comp)) + c0,
                                      sel, M, Kpf, Ks, Kpc, pad);
  return cudaGetLastError();
}

// Gather instance b's selected columns of the full line-outage block(s) into the compacted copies.
template <typename Real, typename Dc>
int gather_lodf(qg_ctx *h, const Dev<Real, Dc> &d, int b) {
  const Inst &I = h->plan.tab.I[b];
  const HostInst &H = h->hi[b];
  const int Kpf = ceil_div(H.K, 4) * 4;
  const long long f0 = h->lf0[b];
  const int *sel = h->d_sel + I.ctg0;
  cudaError_t e;
  if (d.lodf_dtype == QG_LODF_BF16) {
    e = launch_gather<__nv_bfloat16>(h->lodf_full, d.lodf, sel, f0, I.l0, H.M, Kpf, I.K, I.Kp,
                                     __float2bfloat16_rn(NAN), h->stream);
  } else if (d.lodf_dtype == QG_LODF_BF16X2) {
    __nv_bfloat162 pad;
    pad.x = pad.y = __float2bfloat16_rn(NAN);
    e = launch_gather<__nv_bfloat162>(h->lodf_full, d.lodf, sel, f0, I.l0, H.M, Kpf, I.K, I.Kp, pad, h->stream);
  } else {
    e = launch_gather<float>(h->lodf_full, d.lodf, sel, f0, I.l0, H.M, Kpf, I.K, I.Kp, NAN, h->stream);
  }
  if (e == cudaSuccess && d.lodf64)
    e = launch_gather<double>(h->lodf64_full, d.lodf64, sel, f0, I.l0, H.M, Kpf, I.K, I.Kp, 0.0, h->stream);
  if (e == cudaSuccess) e = launch_lmax(d.lodf, d.lodf_dtype, const_cast<float *>(d.lmax), I, h->stream);
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("line-outage gather: ") + cudaGetErrorString(e));
  return QG_OK;
}

// Make instance b's current selection (hi[b].sel) the outages later evaluations cover: the
// outage index of every branch, the outaged branch of every selected column and the compacted
// line-outage block(s).  Synchronizes the stream.
int upload_selection(qg_ctx *h, int b) {
  const HostInst &H = h->hi[b];
  const Inst &I = h->plan.tab.I[b];
  const int n = (int)H.sel.size();
  std::vector<int> kidx(H.M, -1), cbr(n);
  for (int j = 0; j < n; ++j) {
    kidx[H.ctg[H.sel[j]]] = j;
    cbr[j] = H.ctg[H.sel[j]];
  }
  const bool mx = h->opt.precision == QG_MIXED;
  const int *d_kidx = mx ? h->d32.br_kidx : h->d64.br_kidx;
  const int *d_cbr = mx ? h->d32.ctg_br : h->d64.ctg_br;
  CUDA_TRY(h, cudaMemcpyAsync(const_cast<int *>(d_kidx) + I.br0, kidx.data(), sizeof(int) * H.M, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(const_cast<int *>(d_cbr) + I.ctg0, cbr.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_sel + I.ctg0, H.sel.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  const int rc = mx ? gather_lodf(h, h->d32, b) : gather_lodf(h, h->d64, b);
  if (rc) return rc;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // the host vectors above are freed on return
  return QG_OK;
}

// Build every device array of one precision flavour.
template <typename Real, typename Dc>
int build_device(qg_ctx *h, Dev<Real, Dc> &d, const std::vector<int> &slot_map) {
  const int B = h->n_inst;
  const Plan &P = h->plan;
  std::vector<int2> br_end;
  std::vector<int> br_kidx, gen_bus, gen_zone, gen_gb, gb_ptr{0}, gb_gen, gb_dev0, gb_ndev, zgen_ptr{0}, zgen, ctg_br,
      bal_code, bal_row,
      adj_code, adj_row, br_xf, xf_br;
  std::vector<double> br_g, br_b, br_hch, br_smax, br_s2, ga, gbv, gcr, gpmax, gramp, load_p, load_q, rreq, dt, lo, hi,
      ltot, ptdfg, ptdfaT, cload, rsum, lodf, gsgn, gpmin, gqmin, gqmax, gcon, gcsu, gcsd, guinit, blk_c, blk_lo, blk_w;
  std::vector<int> blk_ptr{0};
  for (int b = 0; b < B; ++b) {
    const HostInst &H = h->hi[b];
    const Inst &D = P.tab.I[b];
    for (int j = 0; j < H.M; ++j) {
      br_end.push_back(make_int2(H.from[j], H.to[j]));
      br_kidx.push_back(-1);
      br_g.push_back(H.gsr[j]);
      br_b.push_back(H.bsr[j]);
      br_hch.push_back(0.5 * H.bch[j]);
      br_smax.push_back(H.smax[j]);
      br_s2.push_back(H.sctg[j] * H.sctg[j]);
    }
    for (int j = 0; j < H.Ks; ++j) {
      br_kidx[D.br0 + H.ctg[H.sel[j]]] = j;
      ctg_br.push_back(H.ctg[H.sel[j]]);
    }
    br_xf.insert(br_xf.end(), H.br_xf.begin(), H.br_xf.end());
    xf_br.insert(xf_br.end(), H.xf.begin(), H.xf.end());
    for (int g = 0; g < H.G; ++g) {
      gen_bus.push_back(H.gen_bus[g]);
      gen_zone.push_back(H.gen_zone[g]);
      gen_gb.push_back(H.gen_gb[g]);
      ga.push_back(H.ca[g]); gbv.push_back(H.cb[g]); gcr.push_back(H.cr[g]); gpmax.push_back(H.pmax[g]);
      gramp.push_back(H.ramp[g]);
      gsgn.push_back(H.cons[g] ? -1.0 : 1.0);
      gpmin.push_back(H.pmin[g]); gqmin.push_back(H.qmin[g]); gqmax.push_back(H.qmax[g]);
      gcon.push_back(H.commit ? H.c_on[g] : 0.0); gcsu.push_back(H.commit ? H.c_su[g] : 0.0);
      gcsd.push_back(H.commit ? H.c_sd[g] : 0.0); guinit.push_back(H.commit ? H.u_init[g] : 1.0);
      // bid blocks: kept only for devices with a positive total width; the cumulative starts are
      // summed in FP64 in block order
      double tot = 0.0;
      for (int l = 0; l < H.L; ++l) tot += H.blk_w[(size_t)g * H.L + l];
      if (tot > 0.0) {
        double cum = 0.0;
        for (int l = 0; l < H.L; ++l) {
          blk_c.push_back(H.blk_c[(size_t)g * H.L + l]);
          blk_lo.push_back(cum);
          blk_w.push_back(H.blk_w[(size_t)g * H.L + l]);
          cum += H.blk_w[(size_t)g * H.L + l];
        }
      }
      blk_ptr.push_back((int)blk_c.size());
    }
    std::vector<std::vector<int>> gbg(H.gbus.size()), zg(H.Z);
    for (int g = 0; g < H.G; ++g) {
      gbg[H.gen_gb[g]].push_back(D.gen0 + g);
      zg[H.gen_zone[g]].push_back(D.gen0 + g);
    }
    for (auto &v : gbg) {
      gb_dev0.push_back(v.empty() ? -1 : v[0]);
      gb_ndev.push_back((int)v.size());
      gb_gen.insert(gb_gen.end(), v.begin(), v.end());
      gb_ptr.push_back((int)gb_gen.size());
    }
    for (auto &v : zg) {
      zgen.insert(zgen.end(), v.begin(), v.end());
      zgen_ptr.push_back((int)zgen.size());
    }
    bal_code.insert(bal_code.end(), H.bal_code.begin(), H.bal_code.end());
    bal_row.insert(bal_row.end(), H.bal_row.begin(), H.bal_row.end());
    adj_code.insert(adj_code.end(), H.adj_code.begin(), H.adj_code.end());
    adj_row.insert(adj_row.end(), H.adj_row.begin(), H.adj_row.end());
    load_p.insert(load_p.end(), H.load_p.begin(), H.load_p.end());
    load_q.insert(load_q.end(), H.load_q.begin(), H.load_q.end());
    rreq.insert(rreq.end(), H.rreq.begin(), H.rreq.end());
    dt.insert(dt.end(), H.dt.begin(), H.dt.end());
    ltot.insert(ltot.end(), H.ltot.begin(), H.ltot.end());
    if (!H.sparse) {
      ptdfg.insert(ptdfg.end(), H.ptdfg.begin(), H.ptdfg.end());
      // columns of the adjoint DC products (Eqs. 2nd_lin_sys, correction), one row per column: the
      // injection adjoint at a generator bus minus its mean over all buses is
      // sum_m dz/df_m (PTDF[m, gb] - (PTDF 1)[m] / n), so the slack's mean is folded into the column;
      // transformer columns are used as they are
      const int Gc = H.Gc, Gb = (int)H.gbus.size();
      for (int q = 0; q < Gc; ++q)
        for (int m = 0; m < H.M; ++m) ptdfaT.push_back(H.ptdfg[(size_t)m * Gc + q] - (q < Gb ? H.rsum[m] / H.n : 0.0));
      cload.insert(cload.end(), H.cload.begin(), H.cload.end());
    }
    rsum.insert(rsum.end(), H.rsum.begin(), H.rsum.end());
    // line-outage block with its row stride padded to Kp; NaN marks the pads and each outage's own
    // branch (the contingency kernel's screen rejects NaN elements)
    {  // with screening this is the full block (every outage), gathered per selection on the device
      const int Kp = h->screen ? ceil_div(H.K, 4) * 4 : P.tab.I[b].Kp;
      const size_t base = lodf.size();
      if (h->screen) h->lf0.push_back((long long)base);
      lodf.resize(base + (size_t)H.M * Kp, NAN);
      for (int m = 0; m < H.M; ++m)
        for (int k = 0; k < H.K; ++k)
          if (H.ctg[k] != m) lodf[base + (size_t)m * Kp + k] = H.lodf[(size_t)m * H.K + k];
    }
    const double inf = INFINITY;
    for (int t = 0; t < H.T; ++t)
      for (int i = 0; i < H.n; ++i) { lo.push_back(H.vmin[i]); hi.push_back(H.vmax[i]); }
    for (int t = 0; t < H.T; ++t)
      for (int i = 0; i < H.n; ++i) {
        lo.push_back(i == H.ref ? 0.0 : -inf);
        hi.push_back(i == H.ref ? 0.0 : inf);
      }
    // with commitment the u-scaled limits are penalties and the box only keeps p >= 0 and q's range
    // around 0; consumers hold no reserve
    for (int t = 0; t < H.T; ++t)
      for (int g = 0; g < H.G; ++g) { lo.push_back(H.commit ? 0.0 : H.pmin[g]); hi.push_back(H.pmax[g]); }
    for (int t = 0; t < H.T; ++t)
      for (int g = 0; g < H.G; ++g) {
        lo.push_back(H.commit ? std::min(H.qmin[g], 0.0) : H.qmin[g]);
        hi.push_back(H.commit ? std::max(H.qmax[g], 0.0) : H.qmax[g]);
      }
    for (int t = 0; t < H.T; ++t)
      for (int g = 0; g < H.G; ++g) { lo.push_back(0.0); hi.push_back(H.cons[g] ? 0.0 : H.pmax[g]); }
    for (int t = 0; t < H.T; ++t)
      for (int q = 0; q < H.X; ++q) { lo.push_back(H.tau_lo[q]); hi.push_back(H.tau_hi[q]); }
    for (int t = 0; t < H.T; ++t)
      for (int q = 0; q < H.X; ++q) { lo.push_back(H.phi_lo[q]); hi.push_back(H.phi_hi[q]); }
    if (H.commit)
      for (int t = 0; t < H.T; ++t)
        for (int g = 0; g < H.G; ++g) { lo.push_back(0.0); hi.push_back(1.0); }
  }
  int rc = 0;
  {
    int2 *p2;
    if ((rc = upload(h, &p2, br_end))) return rc;
    d.br_end = p2;
  }
  int *p;
  Real *r;
  Dc *z;
#define UPI(field, vec) if ((rc = upload(h, &p, vec))) return rc; d.field = p;
#define UPR(field, vec) { auto tmp_ = cast<Real>(vec); if ((rc = upload(h, &r, tmp_))) return rc; d.field = r; }
#define UPD(field, vec) { auto tmp_ = to_dc<Dc>(vec); if ((rc = upload(h, &z, tmp_))) return rc; d.field = z; }
  UPI(br_kidx, br_kidx) UPI(gen_bus, gen_bus) UPI(gen_zone, gen_zone) UPI(gen_gb, gen_gb) UPI(gb_ptr, gb_ptr)
  UPI(gb_gen, gb_gen) UPI(gb_dev0, gb_dev0) UPI(gb_ndev, gb_ndev) UPI(zgen_ptr, zgen_ptr) UPI(zgen, zgen) UPI(ctg_br, ctg_br) UPI(bal_code, bal_code)
  UPI(bal_row, bal_row) UPI(adj_code, adj_code) UPI(adj_row, adj_row) UPI(br_xf, br_xf) UPI(xf_br, xf_br)
  UPR(br_g, br_g) UPR(br_b, br_b) UPR(br_hch, br_hch) UPR(br_smax, br_smax) UPR(br_s2ctg, br_s2)
  UPR(gen_a, ga) UPR(gen_b, gbv) UPR(gen_cr, gcr) UPR(gen_pmax, gpmax)
  UPR(gen_sgn, gsgn) UPR(gen_pmin, gpmin) UPR(gen_qmin, gqmin) UPR(gen_qmax, gqmax) UPR(gen_con, gcon)
  UPR(gen_csu, gcsu) UPR(gen_csd, gcsd) UPR(gen_uinit, guinit) UPI(blk_ptr, blk_ptr) UPR(blk_c, blk_c)
  UPR(blk_lo, blk_lo) UPR(blk_w, blk_w)
  UPR(load_p, load_p) UPR(load_q, load_q) UPR(dt, dt) UPR(lo, lo) UPR(hi, hi)
  UPD(ltot, ltot) UPD(ptdfg, ptdfg) UPD(ptdfaT, ptdfaT) UPD(cload, cload) UPD(rsum, rsum)
  {
    double *q64;
#define UP64(field, vec) if ((rc = upload(h, &q64, vec))) return rc; d.field = q64;
    UP64(lim_pmax, gpmax) UP64(lim_pmin, gpmin) UP64(lim_qmin, gqmin) UP64(lim_qmax, gqmax) UP64(lim_ramp, gramp)
    UP64(lim_rreq, rreq) UP64(lim_dt, dt)
#undef UP64
  }
#undef UPI
#undef UPR
#undef UPD
  // line-outage block: the arithmetic copy of the mixed path (FP32 / BF16 / BF16 hi+lo), or the
  // FP32 screening copy plus the exact FP64 copy of the FP64 path
  const bool f64 = sizeof(Real) == 8;
  const int dtype = f64 ? QG_LODF_F32 : h->opt.lodf_dtype;
  d.lodf_dtype = dtype;
  if (dtype == QG_LODF_BF16) {
    std::vector<__nv_bfloat16> v(lodf.size());
    for (size_t i = 0; i < v.size(); ++i) v[i] = __float2bfloat16_rn((float)lodf[i]);
    __nv_bfloat16 *q;
    if ((rc = upload(h, &q, v))) return rc;
    d.lodf = q;
  } else if (dtype == QG_LODF_BF16X2) {
    std::vector<__nv_bfloat162> v(lodf.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float f = (float)lodf[i];
      const __nv_bfloat16 hb = __float2bfloat16_rn(f);
      v[i].x = hb;
      v[i].y = __float2bfloat16_rn(f - __bfloat162float(hb));
    }
    __nv_bfloat162 *q;
    if ((rc = upload(h, &q, v))) return rc;
    d.lodf = q;
  } else {
    std::vector<float> v(lodf.begin(), lodf.end());
    float *q;
    if ((rc = upload(h, &q, v))) return rc;
    d.lodf = q;
  }
  if (f64) {
    for (double &v : lodf)
      if (std::isnan(v)) v = 0.0;  // never read: only elements that pass the FP32 screen are recomputed
    double *q;
    if ((rc = upload(h, &q, lodf))) return rc;
    d.lodf64 = q;
  }
  {  // row maxima of the line-outage block for the stage-2 bound test
    long long nl = 0;
    for (int b = 0; b < B; ++b) nl += (long long)P.tab.I[b].n_kt * 4 * P.tab.I[b].n_mt * CT_BM;
    float *lm;
    if ((rc = dalloc(h, &lm, (size_t)std::max(nl, 1LL)))) return rc;
    d.lmax = lm;
  }
  if (!h->screen)
    for (int b = 0; b < B; ++b)
      CUDA_TRY(h, launch_lmax(d.lodf, d.lodf_dtype, const_cast<float *>(d.lmax), P.tab.I[b], h->stream));
  if (h->screen) {  // the uploaded blocks are the full ones; the kernels read compacted copies
    h->lodf_full = const_cast<void *>(d.lodf);
    h->lodf64_full = const_cast<double *>(d.lodf64);
    long long lc = 0;
    std::vector<int> sel;
    for (int b = 0; b < B; ++b) {
      lc += (long long)h->hi[b].M * P.tab.I[b].Kp;
      sel.insert(sel.end(), h->hi[b].sel.begin(), h->hi[b].sel.end());
    }
    const size_t esz = dtype == QG_LODF_BF16 ? 2 : 4;
    unsigned char *cq;
    if ((rc = dalloc(h, &cq, (size_t)lc * esz))) return rc;
    d.lodf = cq;
    if (f64) {
      double *c64;
      if ((rc = dalloc(h, &c64, (size_t)lc))) return rc;
      d.lodf64 = c64;
    }
    if ((rc = upload(h, &h->d_sel, sel))) return rc;
    Real *pz, *zs;
    long long spk = 0, stk = 0;
    for (int b = 0; b < B; ++b) {
      spk += (long long)P.tab.I[b].n_mg * P.tab.I[b].T * P.tab.I[b].K;
      stk += (long long)P.tab.I[b].T * P.tab.I[b].K;
    }
    if ((rc = dalloc(h, &pz, (size_t)spk)) || (rc = dalloc(h, &zs, (size_t)stk))) return rc;
    d.pz = pz;
    d.zs = zs;
    d.score = 1;
    for (int b = 0; b < B; ++b)
      if ((rc = gather_lodf(h, d, b))) return rc;
    CUDA_TRY(h, cudaDeviceSynchronize());
  }
  // sparse DC mode (instance 0)
  d.sp = P.sp;
  if (P.sp) {
    const HostInst &H = h->hi[0];
    d.nr = H.n - 1;
    d.nS = H.nS;
    d.nT = H.nT;
    d.n_pchunk = ceil_div(d.nr, 32);
    d.n_adj_rows = (int)H.adj_rows.size();
    std::vector<double> ydc(H.y);
#define UPI(field, vec) if ((rc = upload(h, &p, vec))) return rc; d.field = p;
#define UPD(field, vec) { auto tmp_ = to_dc<Dc>(vec); if ((rc = upload(h, &z, tmp_))) return rc; d.field = z; }
    UPI(bus_pos, H.bus_pos) UPI(pos_gb, H.pos_gb) UPI(pos_bus, H.pos_bus) UPI(fw_ptr, H.fw_ptr) UPI(fw_col, H.fw_col)
    UPI(bw_ptr, H.bw_ptr) UPI(bw_col, H.bw_col) UPI(adj_rows, H.adj_rows) UPI(inc_ptr, H.inc_ptr)
    UPI(inc_code, H.inc_code)
    UPD(fw_val, H.fw_val) UPD(bw_val, H.bw_val) UPD(dinv, H.dinv) UPD(sinv, H.sinv) UPD(z1, H.z1) UPD(ydc, ydc)
    UPD(load_dc, H.load_p)
#undef UPI
#undef UPD
    const long long nrT = (long long)d.nr * H.T;
    Dc *c;
    if ((rc = dalloc(h, &c, (size_t)nrT))) return rc;
    d.sp_rhs = c;
    if ((rc = dalloc(h, &c, (size_t)nrT))) return rc;
    d.sp_u = c;
    if ((rc = dalloc(h, &c, (size_t)nrT))) return rc;
    d.sp_th = c;
    if ((rc = dalloc(h, &c, (size_t)std::max(1LL, (long long)d.nT * H.T)))) return rc;
    d.sp_zt = c;
    if ((rc = dalloc(h, &c, (size_t)H.T))) return rc;
    d.sp_mu = c;
    if ((rc = dalloc(h, &c, (size_t)d.n_pchunk * H.T))) return rc;
    d.sp_part = c;
    if ((rc = dalloc(h, &c, (size_t)std::max(1LL, (long long)P.sp_tail_ks * d.nT * H.T)))) return rc;
    d.sp_tpart = c;
    unsigned int *tk;
    if ((rc = dalloc(h, &tk, (size_t)std::max(1, ceil_div(d.nT, SP_RB))))) return rc;
    d.sp_tick = tk;
  }
  const qg_options &o = h->opt;
  d.c_p = (Real)o.c_p; d.c_q = (Real)o.c_q; d.c_s = (Real)o.c_s; d.c_rz = (Real)o.c_rz;
  d.rho = (Real)o.rho; d.eps = (Real)o.eps; d.beta = (Real)o.beta;
  d.c_s64 = o.c_s; d.eps64 = o.eps; d.beta64 = o.beta;
  // work buffers
  long long sTM = 0, sTn = 0, sTZ = 0, sTK = 0, sTG = 0, sPM = 0, sPK = 0, sGI = 0, sTX = 0;
  for (int b = 0; b < B; ++b) {
    const Inst &I = P.tab.I[b];
    sTM += (long long)I.T * I.M; sTn += (long long)I.T * I.n; sTZ += (long long)I.T * I.Z;
    sTK += (long long)I.T * I.K; sTG += (long long)I.T * I.G;
    sPM += (long long)I.n_kt * I.T * I.M; sPK += (long long)I.n_mg * I.T * I.K;
    sGI += (long long)I.T * (I.Gc + 1); sTX += (long long)I.T * I.X;
  }
  Real *w;
  Dc *c;
  float *fl;
#define WR(field, cnt) if ((rc = dalloc(h, &w, (size_t)(cnt)))) return rc; d.field = w;
#define WD(field, cnt) if ((rc = dalloc(h, &c, (size_t)(cnt)))) return rc; d.field = c;
#define WF(field, cnt) if ((rc = dalloc(h, &fl, (size_t)(cnt)))) return rc; d.field = fl;
  d.n_pairs = sTG;
  WR(pf, sTM) WR(qf, sTM) WR(pt, sTM) WR(qt, sTM) WR(qm2, sTM) WR(fre, sTM) WR(fk, sTK) WR(pold, sTG) WR(uold, sTG)
  WR(dP, sTn) WR(dQ, sTn) WR(dZ, sTZ) WR(pm, sPM) WR(pq, sPM) WR(pk, sPK) WR(gF, sTM) WR(avf, sTM) WR(avo, sTM)
  WR(ad, sTM) WR(atx, sTX)
  WD(gip, sGI)
  WF(f32, sTM) WF(fk32, sTK)
#undef WR
#undef WD
#undef WF
  unsigned char *qs;
  if ((rc = dalloc(h, &qs, (size_t)sTM))) return rc;
  d.qside = qs;
  long long sPF = 0;
  for (int b = 0; b < B; ++b) sPF += (long long)P.tab.I[b].n_kt * P.tab.I[b].T * P.tab.I[b].n_mt;
  unsigned char *pf;
  if ((rc = dalloc(h, &pf, (size_t)std::max(1LL, sPF)))) return rc;
  d.pmf = pf;
  {
    long long sRM = 0;
    for (int b = 0; b < B; ++b) sRM += (long long)P.tab.I[b].T * P.tab.I[b].n_mt * CT_BM;
    float *rm;
    if ((rc = dalloc(h, &rm, (size_t)std::max(1LL, sRM)))) return rc;
    d.ctg_rmin = rm;
  }
  Dc *op;
  d.n_obj12 = (int)slot_map.size();
  d.n_gen_slots = P.n_gen_slots;
  d.n_obj_slots = d.n_obj12 + P.n_gen_slots + P.n_fold_slots;
  if ((rc = dalloc(h, &op, (size_t)d.n_obj_slots * N_TERMS))) return rc;
  d.objp = op;
  int *si;
  if ((rc = upload(h, &si, slot_map))) return rc;
  d.slot_map = si;
  d.obj = h->d_obj;
  d.terms = h->d_terms;
  d.g = static_cast<Real *>(h->d_g);
  d.ticket = h->d_ticket;
  d.step = h->d_step;
  d.trace_step0 = h->d_step0;
  d.am = static_cast<Real *>(h->d_m);
  d.av = static_cast<Real *>(h->d_v);
  return QG_OK;
}

int check_device(qg_ctx *h) {
  int dev = -1, count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) return fail(h, QG_ERR_NO_DEVICE, "no CUDA device");
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(h, QG_ERR_NO_DEVICE, "cudaGetDevice failed");
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return fail(h, QG_ERR_NO_DEVICE, "cudaGetDeviceProperties failed");
  if (p.major != 10 || p.minor != 3)
    return fail(h, QG_ERR_NO_DEVICE, std::string("libqg is built for sm_103a; device is ") + p.name);
  return QG_OK;
}

constexpr int SOLVE_UNROLL = 8;  // Adam iterations per graph launch in long solves

void drop_graphs(qg_ctx *h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->gexec_u) cudaGraphExecDestroy(h->gexec_u);
  if (h->hexec) cudaGraphExecDestroy(h->hexec);
  h->gexec = h->gexec_u = h->hexec = nullptr;
}

void free_all(qg_ctx *h) {
  drop_graphs(h);
  for (auto &e : h->ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  for (void *p : h->allocs) {
    bounds_unregister(p);
    cudaFree(p);
  }
  h->allocs.clear();
}

bool mixed(const qg_ctx *h) { return h->opt.precision == QG_MIXED; }

// One evaluation; with adam, the projected Adam update is fused into stages 4 and 5 using the
// handle's moments and the given hyper-parameters.
// step_off: this iteration's place in a graph of several (it reads step + step_off); defer: leave
// the objective sum and the step count to a run_finish after the graph's last iteration (fused
// iterations without a trace); otherwise the evaluation ends with its own closing kernel.
int run_eval(qg_ctx *h, const void *x, bool adam, double lr, double b1, double b2, double *trace, int trace_len,
             const double *sched = nullptr, int sched_len = 0, int step_off = 0, bool defer = false) {
  cudaEvent_t *ev = h->profiling ? h->ev : nullptr;
  cudaError_t e;
  if (mixed(h)) {
    Dev<float, df32> d = h->d32;
    d.lr = lr; d.b1 = b1; d.b2 = b2; d.aeps = h->opt.adam_eps; d.paper_eps = h->opt.adam_paper_eps;
    d.trace = trace; d.trace_len = trace_len; d.sched = sched; d.sched_len = sched_len;
    d.step_off = step_off;
    e = launch_eval<float, df32>(d, h->plan, x, adam, !defer, h->stream, ev);
  } else {
    Dev<double, double> d = h->d64;
    d.lr = lr; d.b1 = b1; d.b2 = b2; d.aeps = h->opt.adam_eps; d.paper_eps = h->opt.adam_paper_eps;
    d.trace = trace; d.trace_len = trace_len; d.sched = sched; d.sched_len = sched_len;
    d.step_off = step_off;
    e = launch_eval<double, double>(d, h->plan, x, adam, !defer, h->stream, ev);
  }
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("evaluation launch: ") + cudaGetErrorString(e));
  return QG_OK;
}

// Frees one device allocation made by dalloc / upload.
void dfree(qg_ctx *h, const void *p) {
  if (!p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), const_cast<void *>(p));
  if (it != h->allocs.end()) {
    bounds_unregister(*it);
    cudaFree(*it);
    h->allocs.erase(it);
  }
}

// Re-plans the handle with the contingency-block shape kn: new spans and instance offsets, and new
// plan-dependent work buffers (outage-column partials, score partials, objective slots and the slot
// map); every other device array stays.  The captured solve graph is dropped (re-captured on use).
template <typename Real, typename Dc>
int replan_dev(qg_ctx *h, Dev<Real, Dc> &d, const Knobs &kn) {
  std::vector<int> slot_map;
  int rc = build_plan(h, slot_map, kn);
  if (rc) return rc;
  const Plan &P = h->plan;
  if (P.s1.n > MAXSPAN || P.s2.n > MAXSPAN) return fail(h, QG_ERR_UNSUPPORTED, "too many block spans");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // no launch in flight uses the old buffers
  long long spk = 0;
  for (int b = 0; b < h->n_inst; ++b) spk += (long long)P.tab.I[b].n_mg * P.tab.I[b].T * P.tab.I[b].K;
  dfree(h, d.pk);
  dfree(h, d.objp);
  dfree(h, d.slot_map);
  Real *pk;
  if ((rc = dalloc(h, &pk, (size_t)std::max(1LL, spk)))) return rc;
  d.pk = pk;
  if (d.score) {
    dfree(h, d.pz);
    Real *pz;
    if ((rc = dalloc(h, &pz, (size_t)std::max(1LL, spk)))) return rc;
    d.pz = pz;
  }
  d.n_obj12 = (int)slot_map.size();
  d.n_gen_slots = P.n_gen_slots;
  d.n_obj_slots = d.n_obj12 + P.n_gen_slots + P.n_fold_slots;
  Dc *op;
  if ((rc = dalloc(h, &op, (size_t)d.n_obj_slots * N_TERMS))) return rc;
  d.objp = op;
  int *si;
  if ((rc = upload(h, &si, slot_map))) return rc;
  d.slot_map = si;
  const cudaError_t e = prepare_eval<Real, Dc>(P.maxTB, h->screen, P.ctg_lazy != 0);
  if (e != cudaSuccess) {
    cudaGetLastError();  // a refused attribute is not a sticky error
    return fail(h, QG_ERR_UNSUPPORTED, std::string("prepare_eval: ") + cudaGetErrorString(e));
  }
  drop_graphs(h);
  h->knobs = kn;
  return QG_OK;
}

int replan(qg_ctx *h, const Knobs &kn) { return mixed(h) ? replan_dev(h, h->d32, kn) : replan_dev(h, h->d64, kn); }

// Mean device time in ms of `reps` evaluations at x (after two untimed ones), or a negative value
// on failure.  With `flush` (a device buffer larger than L2, flush_bytes long) every timed
// evaluation starts from an L2 holding none of the evaluation's data, and only the evaluations are
// timed.
double time_evals(qg_ctx *h, const void *x, int reps, void *flush, size_t flush_bytes) {
  std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
  bool ok = std::all_of(ev.begin(), ev.end(), [](cudaEvent_t e) { return e != nullptr; });
  ok = ok && run_eval(h, x, false, 0, 0, 0, nullptr, 0) == QG_OK && run_eval(h, x, false, 0, 0, 0, nullptr, 0) == QG_OK;
  for (int r = 0; ok && r < reps; ++r) {
    if (flush) ok = cudaMemsetAsync(flush, r & 0xff, flush_bytes, h->stream) == cudaSuccess;
    ok = ok && cudaEventRecord(ev[2 * r], h->stream) == cudaSuccess;
    ok = ok && run_eval(h, x, false, 0, 0, 0, nullptr, 0) == QG_OK;
    ok = ok && cudaEventRecord(ev[2 * r + 1], h->stream) == cudaSuccess;
  }
  ok = ok && cudaStreamSynchronize(h->stream) == cudaSuccess;
  double ms = 0.0;
  for (int r = 0; ok && r < reps; ++r) {
    float t = 0.0f;
    ok = cudaEventElapsedTime(&t, ev[2 * r], ev[2 * r + 1]) == cudaSuccess;
    ms += t;
  }
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  return ok ? ms / reps : -1.0;
}

// Closing kernel of n deferred iterations: the objective of the last one (read at its schedule
// row), then step += n.
int run_finish(qg_ctx *h, int n, const double *sched, int sched_len) {
  cudaError_t e;
  if (mixed(h)) {
    Dev<float, df32> d = h->d32;
    d.sched = sched; d.sched_len = sched_len; d.step_off = n - 1;
    e = launch_finish<float, df32>(d, h->plan, n, h->stream);
  } else {
    Dev<double, double> d = h->d64;
    d.sched = sched; d.sched_len = sched_len; d.step_off = n - 1;
    e = launch_finish<double, double>(d, h->plan, n, h->stream);
  }
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("closing kernel launch: ") + cudaGetErrorString(e));
  return QG_OK;
}

int run_adam(qg_ctx *h, void *x, void *m, void *v, double lr, double b1, double b2) {
  cudaError_t e;
  if (mixed(h))
    e = launch_adam<float>((float *)x, (float *)m, (float *)v, (const float *)h->d_g, h->d32.lo, h->d32.hi, h->n_x,
                           h->d_step, h->d_ticket, lr, b1, b2, h->opt.adam_eps, h->opt.adam_paper_eps, h->stream);
  else
    e = launch_adam<double>((double *)x, (double *)m, (double *)v, (const double *)h->d_g, h->d64.lo, h->d64.hi,
                            h->n_x, h->d_step, h->d_ticket, lr, b1, b2, h->opt.adam_eps, h->opt.adam_paper_eps,
                            h->stream);
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("adam launch: ") + cudaGetErrorString(e));
  if (h->profiling) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(h->stream, &st);
    if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(h->ev[N_PHASES], h->stream, cudaEventRecordExternal);
    else cudaEventRecord(h->ev[N_PHASES], h->stream);
  }
  return QG_OK;
}

__global__ void k_d2f(const double *a, float *b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f2d(const float *a, double *b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// Host-buffer evaluation through the caller's page-locked buffers' device mappings: x read into the
// handle's variable array (rounded to FP32 on the mixed path) ...
template <typename Real>
__global__ void k_host_in(const double *hx, Real *xs, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    xs[i] = (Real)hx[i];
}

// ... and the gradient and the objectives written back (each may be NULL).
template <typename Real>
__global__ void k_host_out(const Real *g, double *hg, long long n, const double *obj, double *hobj, int n_inst) {
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (hobj && i0 < n_inst) hobj[i0] = obj[i0];
  if (!hg) return;
  for (long long i = i0; i < n; i += (long long)gridDim.x * blockDim.x) hg[i] = (double)g[i];
}

}  // namespace

// =============================================================================================
// Scratch for qg_eval_grad_noalloc: a file-scope device array.  Every GPU that loads the library
// holds it from module load until the process exits.  Host code must not pass the symbol itself
// to a kernel (on the host it only names a stand-in); the device address comes from
// cudaGetSymbolAddress, looked up once per device.
// =============================================================================================

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up on first use per device).
int noalloc_scratch(qg_ctx *h, unsigned char **out) {
  int dev = -1;
  CUDA_TRY(h, cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(h, QG_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(h, QG_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<unsigned char *>(ptr);
    bounds_register(ptr, NOALLOC_SCRATCH_BYTES);
  }
  *out = g_noalloc_ptr[dev];
  return QG_OK;
}

// Carve every per-evaluation work buffer of `d` out of [base, base + cap); returns the bytes used
// (more than cap means the handle does not fit, and nothing is assigned past cap).
template <typename Real, typename Dc>
size_t carve_scratch(const qg_ctx *h, unsigned char *base, size_t cap, Dev<Real, Dc> &d) {
  const Plan &P = h->plan;
  long long sTM = 0, sTn = 0, sTZ = 0, sTK = 0, sTG = 0, sPM = 0, sPK = 0, sGI = 0, sTX = 0;
  for (int b = 0; b < h->n_inst; ++b) {
    const Inst &I = P.tab.I[b];
    sTM += (long long)I.T * I.M; sTn += (long long)I.T * I.n; sTZ += (long long)I.T * I.Z;
    sTK += (long long)I.T * I.K; sTG += (long long)I.T * I.G;
    sPM += (long long)I.n_kt * I.T * I.M; sPK += (long long)I.n_mg * I.T * I.K;
    sGI += (long long)I.T * (I.Gc + 1); sTX += (long long)I.T * I.X;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) -> unsigned char * {
    off = (off + 255) & ~size_t(255);
    unsigned char *p = (off + bytes <= cap) ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t R = sizeof(Real), D = sizeof(Dc);
  d.pf = (Real *)take(R * sTM); d.qf = (Real *)take(R * sTM); d.pt = (Real *)take(R * sTM);
  d.qt = (Real *)take(R * sTM); d.qm2 = (Real *)take(R * sTM); d.fre = (Real *)take(R * sTM);
  d.gF = (Real *)take(R * sTM); d.avf = (Real *)take(R * sTM); d.avo = (Real *)take(R * sTM);
  d.ad = (Real *)take(R * sTM); d.qside = take(sTM); d.f32 = (float *)take(4 * sTM);
  d.atx = (Real *)take(R * std::max(1LL, sTX));
  d.fk = (Real *)take(R * sTK); d.fk32 = (float *)take(4 * sTK); d.pold = (Real *)take(R * sTG);
  d.uold = (Real *)take(R * sTG);
  d.dP = (Real *)take(R * sTn); d.dQ = (Real *)take(R * sTn); d.dZ = (Real *)take(R * sTZ);
  d.pm = (Real *)take(R * sPM); d.pq = (Real *)take(R * sPM); d.pk = (Real *)take(R * sPK);
  {
    long long sPF = 0;
    for (int b = 0; b < h->n_inst; ++b) sPF += (long long)P.tab.I[b].n_kt * P.tab.I[b].T * P.tab.I[b].n_mt;
    d.pmf = take(std::max(1LL, sPF));
    long long sRM = 0;
    for (int b = 0; b < h->n_inst; ++b) sRM += (long long)P.tab.I[b].T * P.tab.I[b].n_mt * CT_BM;
    d.ctg_rmin = (float *)take(4 * std::max(1LL, sRM));
  }
  d.gip = (Dc *)take(D * sGI); d.objp = (Dc *)take(D * (size_t)d.n_obj_slots * N_TERMS);
  d.terms = (double *)take(sizeof(double) * N_TERMS * h->n_inst);
  d.ticket = (unsigned int *)take(sizeof(unsigned int));
  d.step = (long long *)take(sizeof(long long));
  d.trace_step0 = d.step;
  return off;
}

template <typename Real, typename Dc>
int eval_noalloc(qg_ctx *h, Dev<Real, Dc> d, const void *x, double *obj, void *g) {
  unsigned char *base = nullptr;
  int rc = noalloc_scratch(h, &base);
  if (rc) return rc;
  const size_t need = carve_scratch(h, base, NOALLOC_SCRATCH_BYTES, d);
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(h, QG_ERR_UNSUPPORTED, "qg_eval_grad_noalloc: this handle needs " + std::to_string(need) +
                                           " bytes of scratch; the static scratch holds " +
                                           std::to_string(NOALLOC_SCRATCH_BYTES));
  d.obj = obj;
  d.g = static_cast<Real *>(g);
  d.trace = nullptr;
  d.trace_len = 0;
  bounds_register(obj, sizeof(double) * h->n_inst);  // the caller's arrays (index-checked builds)
  bounds_register(g, sizeof(Real) * h->n_x);
  // the closing kernel reads and rewrites the step counter (the rest is fully written before it is read)
  CUDA_TRY(h, cudaMemsetAsync(d.step, 0, sizeof(long long), h->stream));
  cudaError_t e = launch_eval<Real, Dc>(d, h->plan, x, false, true, h->stream, nullptr);
  if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("evaluation launch: ") + cudaGetErrorString(e));
  return QG_OK;
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================

extern "C" {

void qg_default_options(qg_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->c_p = 1e4; o->c_q = 1e4; o->c_s = 1e3; o->c_rz = 1e3; o->rho = 1e3;
  o->eps = 1e-3; o->beta = 1.0; o->adam_eps = 1e-8;
  o->precision = QG_FP64; o->lodf_dtype = QG_LODF_F32; o->adam_paper_eps = 0;
}

int qg_create_batch(qg_ctx **out, int32_t n_inst, const qg_network *net, const qg_horizon *hor,
                    const qg_contingencies *ctg, const qg_options *opt) {
  NvtxRange range("qg_create (set-up)");
  g_create_error.clear();
  if (!out) return fail(nullptr, QG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_inst < 1 || !net || !hor || !ctg) return fail(nullptr, QG_ERR_INVALID_ARG, "bad batch arguments");
  if (n_inst > MAXB)
    return fail(nullptr, QG_ERR_UNSUPPORTED, "at most " + std::to_string(MAXB) + " instances per handle");
  qg_ctx *h = new qg_ctx();
  if (opt) h->opt = *opt;
  else qg_default_options(&h->opt);
  const qg_options &o = h->opt;
  auto reject = [&](int code, const std::string &m) {
    fail(h, code, m);
    delete h;
    return code;
  };
  if (o.precision != QG_FP64 && o.precision != QG_MIXED) return reject(QG_ERR_INVALID_ARG, "precision");
  if (o.lodf_dtype < 0 || o.lodf_dtype > 2) return reject(QG_ERR_INVALID_ARG, "lodf_dtype");
  if (o.dc_solver < QG_DC_AUTO || o.dc_solver > QG_DC_SPARSE) return reject(QG_ERR_INVALID_ARG, "dc_solver");
  if (!(o.ctg_frac >= 0.0) || !std::isfinite(o.ctg_frac)) return reject(QG_ERR_INVALID_ARG, "ctg_frac");
  if (o.ctg_bound < QG_CTG_BOUND_AUTO || o.ctg_bound > QG_CTG_BOUND_LAZY) return reject(QG_ERR_INVALID_ARG, "ctg_bound");
  if (o.dc_solver == QG_DC_SPARSE && n_inst > 1)
    return reject(QG_ERR_UNSUPPORTED, "the sparse DC solver takes one instance per handle");
  if (!(o.eps >= 0) || !(o.beta >= 0) || !(o.c_p >= 0) || !(o.c_q >= 0) || !(o.c_s >= 0) || !(o.c_rz >= 0) ||
      !(o.rho >= 0) || !(o.adam_eps >= 0) || !std::isfinite(o.eps + o.beta + o.c_p + o.c_q + o.c_s + o.c_rz + o.rho))
    return reject(QG_ERR_INVALID_ARG, "penalty parameters must be finite and >= 0");
  int rc = QG_OK;
  h->n_inst = n_inst;
  h->hi.resize(n_inst);
  for (int b = 0; b < n_inst; ++b) {
    rc = read_instance(h, net[b], hor[b], ctg[b], h->hi[b], b);
    if (rc) { delete h; return rc; }
  }
  h->hi[0].sparse = o.dc_solver == QG_DC_SPARSE || (o.dc_solver == QG_DC_AUTO && n_inst == 1 && h->hi[0].n > SPARSE_AUTO_N);
  h->screen = o.ctg_frac > 0.0 && o.ctg_frac < 1.0;
  for (auto &H : h->hi) {  // outages per evaluation; the first Ks until qg_ctg_select
    H.Ks = h->screen ? std::max(std::min(H.K, 1), (int)std::ceil(o.ctg_frac * H.K)) : H.K;
    H.sel.resize(H.Ks);
    for (int j = 0; j < H.Ks; ++j) H.sel[j] = j;
  }
  {  // FP64 network set-up per instance, in parallel over instances
    std::vector<int> rcs(n_inst, 0);
    std::vector<std::string> errs(n_inst);
    const unsigned nth = std::max(1u, std::min((unsigned)n_inst, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nth; ++w)
      pool.emplace_back([&, w]() {
        for (int b = (int)w; b < n_inst; b += (int)nth) {
          qg_ctx tmp;
          rcs[b] = build_dc(&tmp, h->hi[b], b);
          errs[b] = tmp.err;
        }
      });
    for (auto &t : pool) t.join();
    for (int b = 0; b < n_inst; ++b)
      if (rcs[b]) return reject(rcs[b], errs[b]);
  }
  std::vector<int> slot_map;
  build_plan(h, slot_map, h->knobs);
  if (h->plan.s1.n > MAXSPAN || h->plan.s2.n > MAXSPAN) return reject(QG_ERR_UNSUPPORTED, "too many block spans");
  // everything above is host-side validation and set-up; from here on the device is needed
  rc = check_device(h);
  if (rc) { delete h; return rc; }
  h->n_x = h->plan.n_x;
  const size_t rs = mixed(h) ? sizeof(float) : sizeof(double);
  if ((rc = dalloc(h, &h->d_obj, (size_t)n_inst)) || (rc = dalloc(h, &h->d_terms, (size_t)n_inst * N_TERMS)) ||
      (rc = dalloc(h, (char **)&h->d_g, rs * h->n_x)) || (rc = dalloc(h, (char **)&h->d_m, rs * h->n_x)) ||
      (rc = dalloc(h, (char **)&h->d_v, rs * h->n_x)) || (rc = dalloc(h, (char **)&h->d_xs, rs * h->n_x)) ||
      (rc = dalloc(h, &h->d_xd, (size_t)h->n_x)) || (rc = dalloc(h, &h->d_step, 1)) ||
      (rc = dalloc(h, &h->d_step0, 1)) || (rc = dalloc(h, &h->d_ticket, 1))) {
    free_all(h);
    delete h;
    return rc;
  }
  rc = mixed(h) ? build_device<float, df32>(h, h->d32, slot_map) : build_device<double, double>(h, h->d64, slot_map);
  if (!rc) {
    cudaError_t e = mixed(h) ? prepare_eval<float, df32>(h->plan.maxTB, h->screen, h->plan.ctg_lazy != 0)
                             : prepare_eval<double, double>(h->plan.maxTB, h->screen, h->plan.ctg_lazy != 0);
    if (e != cudaSuccess) rc = fail(h, QG_ERR_UNSUPPORTED, std::string("prepare_eval: ") + cudaGetErrorString(e));
  }
  if (rc) {
    free_all(h);
    delete h;
    return rc;
  }
  for (auto &I : h->hi) {  // the device holds the set-up products now
    I.ptdfg.clear(); I.ptdfg.shrink_to_fit();
    I.lodf.clear(); I.lodf.shrink_to_fit();
    I.cload.clear(); I.cload.shrink_to_fit();
  }
  *out = h;
  return QG_OK;
}

int qg_create(qg_ctx **out, const qg_network *net, const qg_horizon *hor, const qg_contingencies *ctg,
              const qg_options *opt) {
  return qg_create_batch(out, 1, net, hor, ctg, opt);
}

void qg_destroy(qg_ctx *h) {
  if (!h) return;
  free_all(h);
  delete h;
}

int64_t qg_num_vars(const qg_ctx *h) { return h ? h->n_x : 0; }

int qg_layout(const qg_ctx *h, int32_t inst, int64_t *first, int64_t *n_x, int64_t offsets[8]) {
  if (!h || inst < 0 || inst >= h->n_inst) return QG_ERR_INVALID_ARG;
  const Inst &I = h->plan.tab.I[inst];
  const int64_t Tn = (int64_t)I.T * I.n, TG = (int64_t)I.T * I.G, TX = (int64_t)I.T * I.X;
  if (first) *first = I.x0;
  if (n_x) *n_x = 2 * Tn + 3 * TG + 2 * TX + (I.uc ? TG : 0);
  if (offsets) {
    offsets[0] = 0; offsets[1] = Tn; offsets[2] = 2 * Tn; offsets[3] = 2 * Tn + TG; offsets[4] = 2 * Tn + 2 * TG;
    offsets[5] = 2 * Tn + 3 * TG; offsets[6] = 2 * Tn + 3 * TG + TX; offsets[7] = 2 * Tn + 3 * TG + 2 * TX;
  }
  return QG_OK;
}

int qg_set_stream(qg_ctx *h, void *stream) {
  if (!h) return QG_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  return QG_OK;
}

int qg_eval_grad(qg_ctx *h, const void *x, double *obj, void *g) {
  NvtxRange range("qg_eval_grad");
  if (!h || !x) return h ? fail(h, QG_ERR_INVALID_ARG, "x is NULL") : QG_ERR_INVALID_ARG;
  int rc = run_eval(h, x, false, 0, 0, 0, nullptr, 0);
  if (rc) return rc;
  const size_t rs = mixed(h) ? sizeof(float) : sizeof(double);
  if (obj) CUDA_TRY(h, cudaMemcpyAsync(obj, h->d_obj, sizeof(double) * h->n_inst, cudaMemcpyDeviceToDevice, h->stream));
  if (g) CUDA_TRY(h, cudaMemcpyAsync(g, h->d_g, rs * h->n_x, cudaMemcpyDeviceToDevice, h->stream));
  return QG_OK;
}

int qg_eval_grad_noalloc(qg_ctx *h, const void *x, double *obj, void *g) {
  if (!h || !x || !obj || !g)
    return h ? fail(h, QG_ERR_INVALID_ARG, "qg_eval_grad_noalloc needs x, obj and g") : QG_ERR_INVALID_ARG;
  if (h->plan.sp)
    return fail(h, QG_ERR_UNSUPPORTED, "qg_eval_grad_noalloc: handles on the sparse DC solver do not fit its scratch");
  if (h->screen)
    return fail(h, QG_ERR_UNSUPPORTED, "qg_eval_grad_noalloc: handles with contingency screening do not fit its scratch");
  return mixed(h) ? eval_noalloc<float, df32>(h, h->d32, x, obj, g) : eval_noalloc<double, double>(h, h->d64, x, obj, g);
}

}  // extern "C"

namespace {

// The work of qg_eval_grad_host on h->stream: copy x in, evaluate, copy the gradient and objective out.
// The device address through which a kernel reaches the page-locked host buffer p (NULL for NULL,
// for pageable memory, or when the buffer has no device mapping).
void *device_view(const void *p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int host_eval_work(qg_ctx *h, const double *x, double *obj, double *g) {
  const long long n = h->n_x;
  const int nb = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  // page-locked buffers that kernels can reach: read x and write g, obj from the kernels themselves
  // (no copy nodes); otherwise copies through the handle's staging array
  const double *dx = static_cast<const double *>(device_view(x));
  double *dobj = static_cast<double *>(device_view(obj)), *dg = static_cast<double *>(device_view(g));
  if (dx && (!obj || dobj) && (!g || dg)) {
    bounds_register(dx, sizeof(double) * n);  // index-checked builds: the caller's arrays
    if (mixed(h)) k_host_in<float><<<nb, 256, 0, h->stream>>>(dx, (float *)h->d_xs, n);
    else k_host_in<double><<<nb, 256, 0, h->stream>>>(dx, (double *)h->d_xs, n);
    CUDA_TRY(h, cudaGetLastError());
    int rc = run_eval(h, h->d_xs, false, 0, 0, 0, nullptr, 0);
    if (rc) return rc;
    if (mixed(h)) k_host_out<float><<<nb, 256, 0, h->stream>>>((const float *)h->d_g, dg, g ? n : 0, h->d_obj, dobj, h->n_inst);
    else k_host_out<double><<<nb, 256, 0, h->stream>>>((const double *)h->d_g, dg, g ? n : 0, h->d_obj, dobj, h->n_inst);
    CUDA_TRY(h, cudaGetLastError());
    return QG_OK;
  }
  if (mixed(h)) {
    CUDA_TRY(h, cudaMemcpyAsync(h->d_xd, x, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    k_d2f<<<nb, 256, 0, h->stream>>>(h->d_xd, (float *)h->d_xs, n);
  } else {
    CUDA_TRY(h, cudaMemcpyAsync(h->d_xs, x, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
  }
  int rc = run_eval(h, h->d_xs, false, 0, 0, 0, nullptr, 0);
  if (rc) return rc;
  if (g) {
    if (mixed(h)) {
      k_f2d<<<nb, 256, 0, h->stream>>>((const float *)h->d_g, h->d_xd, n);
      CUDA_TRY(h, cudaMemcpyAsync(g, h->d_xd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    } else {
      CUDA_TRY(h, cudaMemcpyAsync(g, h->d_g, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    }
  }
  if (obj) CUDA_TRY(h, cudaMemcpyAsync(obj, h->d_obj, sizeof(double) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
  return QG_OK;
}

bool pinned(const void *p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int qg_eval_grad_host(qg_ctx *h, const double *x, double *obj, double *g) {
  NvtxRange range("qg_eval_grad_host");
  if (!h || !x) return h ? fail(h, QG_ERR_INVALID_ARG, "x is NULL") : QG_ERR_INVALID_ARG;
  // pinned buffers (and no per-kernel timing): one cached graph of the copies and the evaluation,
  // re-captured when the buffers change (the same buffers as the cached graph's skip the check)
  const bool cached = h->hexec && h->h_x == x && h->h_obj == obj && h->h_g == g;
  const bool graph = !h->profiling && (cached || (pinned(x) && pinned(obj) && pinned(g)));
  if (graph) {
    if (!cached) {
      if (h->hexec) cudaGraphExecDestroy(h->hexec);
      h->hexec = nullptr;
      cudaStream_t cs;
      CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaStream_t saved = h->stream;
      h->stream = cs;
      cudaGraph_t gr;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      int rc = QG_OK;
      if (e == cudaSuccess) {
        rc = host_eval_work(h, x, obj, g);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
        if (!rc && e2 == cudaSuccess) {
          e = cudaGraphInstantiate(&h->hexec, gr, 0);
          cudaGraphDestroy(gr);
        } else if (!rc) {
          e = e2;
        }
      }
      h->stream = saved;
      cudaStreamDestroy(cs);
      if (rc) return rc;
      if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      h->h_x = x; h->h_obj = obj; h->h_g = g;
    }
    CUDA_TRY(h, cudaGraphLaunch(h->hexec, h->stream));
  } else {
    const int rc = host_eval_work(h, x, obj, g);
    if (rc) return rc;
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaGetLastError());
  // the objective is on the host now: a NaN or Inf (from x or from an overflow) is reported, with
  // every output written as computed
  if (obj)
    for (int b = 0; b < h->n_inst; ++b)
      if (!std::isfinite(obj[b]))
        return fail(h, QG_ERR_NONFINITE, "instance " + std::to_string(b) + ": the objective is not finite");
  return QG_OK;
}

int qg_adam_step(qg_ctx *h, void *x, void *m, void *v, double lr, double beta1, double beta2) {
  if (!h || !x || !m || !v) return h ? fail(h, QG_ERR_INVALID_ARG, "null pointer") : QG_ERR_INVALID_ARG;
  if (!(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1))
    return fail(h, QG_ERR_INVALID_ARG, "Adam parameters out of range");
  return run_adam(h, x, m, v, lr, beta1, beta2);
}

}  // extern "C"

namespace {

// qg_solve and qg_solve_schedule: replay the cached graph of one (evaluation + fused Adam)
// iteration `iters` times, capturing it first when the arguments differ from the cached ones.
int solve_graph(qg_ctx *h, void *x, int32_t iters, double lr, double beta1, double beta2, double *obj_trace,
                const double *sched, int len, bool restart) {
  if (!h || !x || iters < 0) return h ? fail(h, QG_ERR_INVALID_ARG, "bad solve arguments") : QG_ERR_INVALID_ARG;
  if (!(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1))
    return fail(h, QG_ERR_INVALID_ARG, "Adam parameters out of range");
  if (iters == 0) return QG_OK;
  // the trace and the schedule are indexed by (step - step at the origin of the run)
  if ((obj_trace || sched) && restart)
    CUDA_TRY(h, cudaMemcpyAsync(h->d_step0, h->d_step, sizeof(long long), cudaMemcpyDeviceToDevice, h->stream));
  if (!obj_trace && !sched) len = 0;
  if (obj_trace) bounds_register(obj_trace, sizeof(double) * (size_t)len * h->n_inst);  // index-checked builds
  if (sched) bounds_register(sched, sizeof(double) * 3 * (size_t)len);
  const bool same = h->gexec && h->g_x == x && h->g_lr == lr && h->g_b1 == beta1 && h->g_b2 == beta2 &&
                    h->g_trace == obj_trace && h->g_sched == sched && h->g_trace_len == len;
  if (!same) drop_graphs(h);
  // capture `n` iterations (evaluation + fused Adam) into one graph
  auto capture = [&](cudaGraphExec_t *out, int n) -> int {
    cudaStream_t cs;
    CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = h->stream;
    h->stream = cs;
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = QG_OK;
    if (e == cudaSuccess) {
      // without a trace the objective is summed once, after the last iteration of the graph
      const bool defer = obj_trace == nullptr && !h->profiling;
      for (int k = 0; k < n && !rc; ++k)
        rc = run_eval(h, x, true, lr, beta1, beta2, obj_trace, obj_trace ? len : 0, sched, sched ? len : 0,
                      defer ? k : 0, defer);
      if (!rc && defer) rc = run_finish(h, n, sched, sched ? len : 0);
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (!rc && e2 == cudaSuccess) {
        e = cudaGraphInstantiate(out, graph, 0);
        cudaGraphDestroy(graph);
      } else if (!rc) {
        e = e2;
      }
    }
    h->stream = saved;
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(h, QG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    return QG_OK;
  };
  if (!h->gexec) {
    int rc = capture(&h->gexec, 1);
    if (rc) return rc;
    h->g_x = x; h->g_lr = lr; h->g_b1 = beta1; h->g_b2 = beta2; h->g_trace = obj_trace; h->g_sched = sched;
    h->g_trace_len = len;
  }
  // long solves: SOLVE_UNROLL iterations per launch (no graph-launch gap between them); the timed
  // per-kernel mode keeps one iteration per launch
  const int n_u = h->profiling ? 0 : iters / SOLVE_UNROLL;
  if (n_u > 0 && !h->gexec_u) {
    int rc = capture(&h->gexec_u, SOLVE_UNROLL);
    if (rc) return rc;
  }
  for (int it = 0; it < n_u; ++it) CUDA_TRY(h, cudaGraphLaunch(h->gexec_u, h->stream));
  for (int it = n_u * SOLVE_UNROLL; it < iters; ++it) CUDA_TRY(h, cudaGraphLaunch(h->gexec, h->stream));
  return QG_OK;
}

// Reflected sigmoid of Eq. mag_scale.
double mag_scale(double t) {
  const double e = std::exp(4.0 * t);
  return e / (0.6 + e);
}

}  // namespace

extern "C" {

int qg_solve(qg_ctx *h, void *x, int32_t iters, double lr, double beta1, double beta2, double *obj_trace) {
  NvtxRange range("qg_solve");
  return solve_graph(h, x, iters, lr, beta1, beta2, obj_trace, nullptr, iters, true);
}

int qg_solve_schedule(qg_ctx *h, void *x, int32_t iters, const double *sched, int32_t sched_len, int32_t restart,
                      double beta1, double beta2, double *obj_trace) {
  NvtxRange range("qg_solve_schedule");
  if (!sched || sched_len < 1) return h ? fail(h, QG_ERR_INVALID_ARG, "empty schedule") : QG_ERR_INVALID_ARG;
  return solve_graph(h, x, iters, 0.0, beta1, beta2, obj_trace, sched, sched_len, restart != 0);
}

int qg_schedule(double *out, int32_t iters, double lr0, double lrf, double eps0, double epsf, double beta0,
                double beta1, double lag) {
  if (!out || iters < 1 || !(lr0 > 0) || !(lrf > 0) || !(eps0 > 0) || !(epsf > 0) || !std::isfinite(beta0) ||
      !std::isfinite(beta1) || !std::isfinite(lag))
    return QG_ERR_INVALID_ARG;
  for (int i = 0; i < iters; ++i) {
    const double t = iters > 1 ? 2.0 * i / (iters - 1) - 1.0 : -1.0;  // Eq. norm_t on the iteration fraction
    out[3 * i + 0] = lr0 * std::pow(10.0, mag_scale(t) * std::log10(lrf / lr0));          // Eq. step_size
    out[3 * i + 1] = eps0 * std::pow(10.0, mag_scale(t - lag) * std::log10(epsf / eps0));  // tightening
    out[3 * i + 2] = beta0 + (beta1 - beta0) * 0.5 * (t + 1.0);                               // homotopy
  }
  return QG_OK;
}

int qg_breakdown(qg_ctx *h, double *out) {
  if (!h || !out) return QG_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(out, h->d_terms, sizeof(double) * N_TERMS * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return QG_OK;
}

int qg_dc_flows(qg_ctx *h, float *out) {
  if (!h || !out) return QG_ERR_INVALID_ARG;
  long long n = 0;
  for (int b = 0; b < h->n_inst; ++b) n += (long long)h->plan.tab.I[b].T * h->plan.tab.I[b].M;
  const float *src = mixed(h) ? h->d32.f32 : h->d64.f32;
  CUDA_TRY(h, cudaMemcpyAsync(out, src, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return QG_OK;
}

int qg_get_step(qg_ctx *h, int64_t *step) {
  if (!h || !step) return QG_ERR_INVALID_ARG;
  long long s = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&s, h->d_step, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  *step = s;
  return QG_OK;
}

int qg_set_step(qg_ctx *h, int64_t step) {
  if (!h || step < 0) return QG_ERR_INVALID_ARG;
  long long s = step;
  if (step == 0) {  // a fresh start also clears the moments qg_solve keeps in the handle
    const size_t rs = mixed(h) ? sizeof(float) : sizeof(double);
    CUDA_TRY(h, cudaMemsetAsync(h->d_m, 0, rs * h->n_x, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->d_v, 0, rs * h->n_x, h->stream));
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->d_step, &s, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return QG_OK;
}

}  // extern "C"

namespace {

// Solver state blob (qg_get_state / qg_set_state): a fixed header, then the sections below, each
// starting on an 8-byte boundary.
constexpr uint32_t STATE_MAGIC = 0x31534751u;  // "QGS1" in little-endian byte order
constexpr uint32_t STATE_VERSION = 1;
constexpr int32_t STATE_SEL = 1, STATE_ROUND = 2;

struct StateHeader {
  uint32_t magic, version;
  int32_t precision, n_inst;
  int64_t n_x;
  int64_t step, step0;  // Adam step counter; its value at the start of the current scheduled run
  int32_t flags;        // STATE_SEL: selections follow the moments; STATE_ROUND: rounding state follows
  int32_t n_sel;        // selected outages over all instances
  int64_t n_pairs;      // (period, device) pairs of the rounding flags
};

size_t pad8(size_t b) { return (b + 7) & ~size_t(7); }

template <typename Real, typename Dc>
int round_alloc(qg_ctx *h, Dev<Real, Dc> &d);

// The header this handle would write now, and the blob's size.
size_t state_layout(const qg_ctx *h, StateHeader *hd) {
  StateHeader H{};
  H.magic = STATE_MAGIC;
  H.version = STATE_VERSION;
  H.precision = h->opt.precision;
  H.n_inst = h->n_inst;
  H.n_x = h->n_x;
  H.flags = (h->screen ? STATE_SEL : 0) | (h->d_fixed ? STATE_ROUND : 0);
  for (const HostInst &I : h->hi) H.n_sel += h->screen ? (int32_t)I.sel.size() : 0;
  H.n_pairs = h->d_fixed ? (int64_t)h->fixed.size() : 0;
  if (hd) *hd = H;
  const size_t rs = h->opt.precision == QG_MIXED ? sizeof(float) : sizeof(double);
  size_t n = pad8(sizeof(StateHeader)) + 2 * pad8(rs * h->n_x);
  if (H.flags & STATE_SEL) n += pad8(sizeof(int32_t) * H.n_sel);
  if (H.flags & STATE_ROUND) n += pad8((size_t)H.n_pairs) + 2 * pad8(rs * h->n_x);
  return n;
}

template <typename Real, typename Dc>
int set_state_dev(qg_ctx *h, Dev<Real, Dc> &d, const unsigned char *buf, int64_t size) {
  StateHeader H;
  std::memcpy(&H, buf, sizeof(H));
  if (H.magic != STATE_MAGIC || H.version != STATE_VERSION)
    return fail(h, QG_ERR_INVALID_ARG, "qg_set_state: not a state blob of this library version");
  StateHeader mine;
  state_layout(h, &mine);
  if (H.precision != mine.precision || H.n_inst != mine.n_inst || H.n_x != mine.n_x)
    return fail(h, QG_ERR_INVALID_ARG, "qg_set_state: the blob belongs to a handle of another precision or size");
  if ((H.flags & STATE_SEL) != (mine.flags & STATE_SEL) || ((H.flags & STATE_SEL) && H.n_sel != mine.n_sel))
    return fail(h, QG_ERR_INVALID_ARG, "qg_set_state: contingency screening differs from this handle's");
  if ((H.flags & STATE_ROUND) && H.n_pairs != (int64_t)d.n_pairs)
    return fail(h, QG_ERR_INVALID_ARG, "qg_set_state: rounding state of another device count");
  if (H.step < 0 || H.step0 < 0 || H.step0 > H.step) return fail(h, QG_ERR_INVALID_ARG, "qg_set_state: bad step counters");
  const size_t rs = sizeof(Real), nx = (size_t)h->n_x;
  size_t need = pad8(sizeof(StateHeader)) + 2 * pad8(rs * nx);
  if (H.flags & STATE_SEL) need += pad8(sizeof(int32_t) * H.n_sel);
  if (H.flags & STATE_ROUND) need += pad8((size_t)H.n_pairs) + 2 * pad8(rs * nx);
  if ((size_t)size < need) return fail(h, QG_ERR_INVALID_ARG, "qg_set_state: blob truncated");
  size_t o = pad8(sizeof(StateHeader));
  const unsigned char *m = buf + o;
  o += pad8(rs * nx);
  const unsigned char *v = buf + o;
  o += pad8(rs * nx);
  if (H.flags & STATE_SEL) {  // validate every selection before changing anything
    const int32_t *sel = reinterpret_cast<const int32_t *>(buf + o);
    long long j = 0;
    for (const HostInst &I : h->hi) {
      std::vector<char> seen(I.K, 0);
      for (int k = 0; k < I.Ks; ++k, ++j) {
        const int32_t id = sel[j];
        if (id < 0 || id >= I.K || seen[id]) return fail(h, QG_ERR_INVALID_ARG, "qg_set_state: bad outage selection");
        seen[id] = 1;
      }
    }
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->d_m, m, rs * nx, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_v, v, rs * nx, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_step, &H.step, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_step0, &H.step0, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // H lives on this stack frame
  if (H.flags & STATE_SEL) {
    const int32_t *sel = reinterpret_cast<const int32_t *>(buf + o);
    for (int b = 0; b < h->n_inst; ++b) {
      HostInst &I = h->hi[b];
      I.sel.assign(sel, sel + I.Ks);
      sel += I.Ks;
      const int rc = upload_selection(h, b);
      if (rc) return rc;
    }
    o += pad8(sizeof(int32_t) * H.n_sel);
  }
  if (H.flags & STATE_ROUND) {
    int rc = round_alloc(h, d);  // keeps this handle's own original box as the one to reset to
    if (rc) return rc;
    const unsigned char *fx = buf + o;
    o += pad8((size_t)H.n_pairs);
    h->fixed.assign(fx, fx + H.n_pairs);
    CUDA_TRY(h, cudaMemcpyAsync(h->d_fixed, h->fixed.data(), (size_t)H.n_pairs, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(const_cast<Real *>(d.lo), buf + o, rs * nx, cudaMemcpyHostToDevice, h->stream));
    o += pad8(rs * nx);
    CUDA_TRY(h, cudaMemcpyAsync(const_cast<Real *>(d.hi), buf + o, rs * nx, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  } else if (h->d_fixed) {
    const int rc = qg_round_reset(h);  // the blob predates rounding: no pair is fixed
    if (rc) return rc;
  }
  return QG_OK;
}

}  // namespace

extern "C" {

int64_t qg_state_size(qg_ctx *h) {
  if (!h) return QG_ERR_INVALID_ARG;
  return (int64_t)state_layout(h, nullptr);
}

int qg_get_state(qg_ctx *h, void *buf, int64_t size) {
  if (!h || !buf) return h ? fail(h, QG_ERR_INVALID_ARG, "qg_get_state: null buffer") : QG_ERR_INVALID_ARG;
  StateHeader H;
  const size_t need = state_layout(h, &H);
  if (size < 0 || (size_t)size < need)
    return fail(h, QG_ERR_INVALID_ARG, "qg_get_state: the buffer needs " + std::to_string(need) + " bytes");
  unsigned char *out = static_cast<unsigned char *>(buf);
  std::memset(out, 0, need);
  const size_t rs = mixed(h) ? sizeof(float) : sizeof(double), nx = (size_t)h->n_x;
  size_t o = pad8(sizeof(StateHeader));
  CUDA_TRY(h, cudaMemcpyAsync(out + o, h->d_m, rs * nx, cudaMemcpyDeviceToHost, h->stream));
  o += pad8(rs * nx);
  CUDA_TRY(h, cudaMemcpyAsync(out + o, h->d_v, rs * nx, cudaMemcpyDeviceToHost, h->stream));
  o += pad8(rs * nx);
  long long st[2] = {0, 0};
  CUDA_TRY(h, cudaMemcpyAsync(&st[0], h->d_step, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(&st[1], h->d_step0, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  if (H.flags & STATE_SEL) {
    int32_t *sel = reinterpret_cast<int32_t *>(out + o);
    for (const HostInst &I : h->hi) sel = std::copy(I.sel.begin(), I.sel.end(), sel);
    o += pad8(sizeof(int32_t) * H.n_sel);
  }
  if (H.flags & STATE_ROUND) {
    std::copy(h->fixed.begin(), h->fixed.end(), out + o);
    o += pad8((size_t)H.n_pairs);
    const void *lo = mixed(h) ? (const void *)h->d32.lo : (const void *)h->d64.lo;
    const void *hi = mixed(h) ? (const void *)h->d32.hi : (const void *)h->d64.hi;
    CUDA_TRY(h, cudaMemcpyAsync(out + o, lo, rs * nx, cudaMemcpyDeviceToHost, h->stream));
    o += pad8(rs * nx);
    CUDA_TRY(h, cudaMemcpyAsync(out + o, hi, rs * nx, cudaMemcpyDeviceToHost, h->stream));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  H.step = st[0];
  H.step0 = st[1];
  std::memcpy(out, &H, sizeof(H));
  return QG_OK;
}

int qg_set_state(qg_ctx *h, const void *buf, int64_t size) {
  if (!h || !buf) return h ? fail(h, QG_ERR_INVALID_ARG, "qg_set_state: null buffer") : QG_ERR_INVALID_ARG;
  if (size < (int64_t)sizeof(StateHeader)) return fail(h, QG_ERR_INVALID_ARG, "qg_set_state: blob truncated");
  const unsigned char *in = static_cast<const unsigned char *>(buf);
  return mixed(h) ? set_state_dev(h, h->d32, in, size) : set_state_dev(h, h->d64, in, size);
}

int qg_set_profiling(qg_ctx *h, int on) {
  if (!h) return QG_ERR_INVALID_ARG;
  if (on && !h->ev[0])
    for (auto &e : h->ev) CUDA_TRY(h, cudaEventCreate(&e));
  if ((on != 0) != h->profiling && h->gexec) {  // the cached graph must be re-captured
    drop_graphs(h);
  }
  h->profiling = on != 0;
  return QG_OK;
}

int qg_phase_times(qg_ctx *h, float *ms, int32_t cap) {
  if (!h || !ms || cap < 0) return QG_ERR_INVALID_ARG;
  if (!h->profiling) return fail(h, QG_ERR_INVALID_ARG, "profiling is off");
  CUDA_TRY(h, cudaEventSynchronize(h->ev[N_PHASES - 1]));
  int n = 0;
  for (int k = 0; k < N_PHASES && n < cap; ++k) {
    float v = 0.f;
    if (k == N_PHASES - 1 && cudaEventQuery(h->ev[N_PHASES]) != cudaSuccess) break;
    if (cudaEventElapsedTime(&v, h->ev[k], h->ev[k + 1]) != cudaSuccess) {
      if (k == N_PHASES - 1) break;  // no stand-alone Adam step followed the evaluation
      v = -1.f;
    }
    ms[n++] = v;
  }
  cudaGetLastError();
  return n;
}

const char *qg_last_error(const qg_ctx *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int qg_ctg_select(qg_ctx *h, int32_t inst, const int32_t *ids, int32_t n) {
  if (!h) return QG_ERR_INVALID_ARG;
  if (!h->screen) return fail(h, QG_ERR_UNSUPPORTED, "qg_ctg_select: the handle has no contingency screening");
  if (inst < 0 || inst >= h->n_inst || !ids) return fail(h, QG_ERR_INVALID_ARG, "qg_ctg_select: bad instance or ids");
  HostInst &H = h->hi[inst];
  if (n != H.Ks) return fail(h, QG_ERR_INVALID_ARG, "qg_ctg_select: n must equal the instance's Ks = " + std::to_string(H.Ks));
  std::vector<char> seen(H.K, 0);
  for (int j = 0; j < n; ++j) {
    if (ids[j] < 0 || ids[j] >= H.K || seen[ids[j]]) return fail(h, QG_ERR_INVALID_ARG, "qg_ctg_select: ids must be distinct in [0, K)");
    seen[ids[j]] = 1;
  }
  H.sel.assign(ids, ids + n);
  return upload_selection(h, inst);
}

int qg_ctg_scores(qg_ctx *h, double *z) {
  if (!h || !z) return QG_ERR_INVALID_ARG;
  if (!h->screen) return fail(h, QG_ERR_UNSUPPORTED, "qg_ctg_scores: the handle has no contingency screening");
  long long n = 0;
  for (int b = 0; b < h->n_inst; ++b) n += (long long)h->plan.tab.I[b].T * h->plan.tab.I[b].K;
  if (mixed(h)) {
    std::vector<float> tmp(n);
    CUDA_TRY(h, cudaMemcpyAsync(tmp.data(), h->d32.zs, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (long long i = 0; i < n; ++i) z[i] = tmp[i];
  } else {
    CUDA_TRY(h, cudaMemcpyAsync(z, h->d64.zs, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return QG_OK;
}

int32_t qg_launches_per_eval(const qg_ctx *h) {
  if (!h) return QG_ERR_INVALID_ARG;
  const Plan &P = h->plan;
  // no contingencies: no stage 2; the on-demand contingency path adds the clearance kernel before it
  const int s2 = P.s2.n_blocks > 0 ? 1 + (P.ctg_lazy ? 1 : 0) : 0;
  // + 1: the closing kernel (the mixed path's dense mode updates the devices in stage 4)
  if (!P.sp) return 3 + s2 + (P.s5.n_blocks > 0 ? 1 : 0) + 1;
  return 4 + s2 + 3 + (P.sp_tail_blocks > 0 ? 2 : 0) + (P.sp_bw_blocks > 0 ? 1 : 0) + (P.sp_bwa_blocks > 0 ? 1 : 0) + 1;
}

int32_t qg_ctg_path(const qg_ctx *h) {
  if (!h) return QG_ERR_INVALID_ARG;
  return h->plan.ctg_lazy ? 2 : h->plan.ctg_bound ? 1 : 0;
}

int qg_autotune(qg_ctx *h, const void *x, int32_t reps, int32_t cold, int32_t shape[2]) {
  NvtxRange range("qg_autotune");
  if (!h) return QG_ERR_INVALID_ARG;
  if (!x || reps < 1) return fail(h, QG_ERR_INVALID_ARG, "qg_autotune needs x and reps >= 1");
  int maxT = 0, max_nmt = 0;
  bool any_ctg = false;
  for (int b = 0; b < h->n_inst; ++b) {
    maxT = std::max(maxT, h->plan.tab.I[b].T);
    max_nmt = std::max(max_nmt, h->plan.tab.I[b].n_mt);
    any_ctg = any_ctg || h->plan.tab.I[b].K > 0;
  }
  Knobs best = h->knobs;
  if (any_ctg) {
    void *flush = nullptr;
    const size_t flush_bytes = (size_t)256 << 20;  // twice the L2
    if (cold && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, QG_ERR_CUDA, "qg_autotune: no room for the L2 flush buffer");
    }
    // candidates (the heuristic first); a candidate that repeats a shape already seen is skipped
    std::vector<Knobs> cand{Knobs{}};
    for (int ntc : {1, 2, 3, 4, 6, 8, 12, 16, 24, 48})
      for (int mg : {1, 2, 3, 4, 6, 9, 12, 16, 24, 32})
        if (ntc <= maxT && mg <= max_nmt) cand.push_back(Knobs{ntc, mg});
    std::vector<std::vector<int>> seen;
    std::vector<std::pair<double, size_t>> timed;  // (ms, candidate)
    int rc = QG_OK;
    auto time_one = [&](const Knobs &kn, double &ms) -> int {
      ms = -1.0;
      int r = replan(h, kn);
      if (r) return r;
      ms = time_evals(h, x, reps, flush, flush_bytes);
      return ms < 0 ? fail(h, QG_ERR_CUDA, "qg_autotune: timing an evaluation failed") : QG_OK;
    };
    for (size_t c = 0; c < cand.size() && !rc; ++c) {
      int r = replan(h, cand[c]);
      if (r == QG_ERR_UNSUPPORTED) continue;  // e.g. a period chunk whose shared memory does not fit
      if (r) { rc = r; break; }
      std::vector<int> sig;
      for (int b = 0; b < h->n_inst; ++b) {
        sig.push_back(h->plan.tab.I[b].ctg_tb);
        sig.push_back(h->plan.tab.I[b].ctg_mg);
      }
      if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
      seen.push_back(sig);
      double ms;
      rc = time_one(cand[c], ms);
      if (!rc) timed.emplace_back(ms, c);
    }
    // second round: the heuristic and the four fastest, each timed twice more, interleaved; each keeps
    // its best round; a shape replaces the heuristic only when it is faster by more than 2%
    if (!rc && !timed.empty()) {
      std::vector<std::pair<double, size_t>> top(timed.begin() + 1, timed.end());
      std::sort(top.begin(), top.end());
      if (top.size() > 4) top.resize(4);
      top.insert(top.begin(), timed[0]);
      for (int round = 0; round < 2 && !rc; ++round)
        for (auto &t : top) {
          double ms;
          rc = time_one(cand[t.second], ms);
          if (rc) break;
          t.first = std::min(t.first, ms);
        }
      if (!rc) {
        size_t pick = 0;
        for (size_t i = 1; i < top.size(); ++i)
          if (top[i].first < top[pick].first) pick = i;
        best = top[pick].first < 0.98 * top[0].first ? cand[top[pick].second] : cand[top[0].second];
      }
    }
    if (flush) cudaFree(flush);
    if (rc) {
      replan(h, Knobs{});
      return rc;
    }
  }
  int rc = replan(h, best);
  if (rc) return rc;
  if (shape) {
    shape[0] = h->plan.tab.I[0].ctg_tb;
    shape[1] = h->plan.tab.I[0].ctg_mg;
  }
  return QG_OK;
}

}  // extern "C"

namespace {

// Buffers of batch rounding, allocated on first use: fixed flags, distances, projections, the
// index list, and a copy of the original clip box (taken now, before any pair is fixed).
template <typename Real, typename Dc>
int round_alloc(qg_ctx *h, Dev<Real, Dc> &d) {
  if (h->d_fixed) return QG_OK;
  const long long sTG = d.n_pairs;
  int rc;
  if ((rc = dalloc(h, &h->d_fixed, (size_t)sTG)) || (rc = dalloc(h, &h->d_dist, (size_t)sTG)) ||
      (rc = dalloc(h, (Real **)&h->d_proj, (size_t)(4 * sTG))) || (rc = dalloc(h, &h->d_idx, (size_t)sTG)) ||
      (rc = dalloc(h, (Real **)&h->d_lo0, (size_t)h->n_x)) || (rc = dalloc(h, (Real **)&h->d_hi0, (size_t)h->n_x)))
    return rc;
  CUDA_TRY(h, cudaMemcpy(h->d_lo0, d.lo, sizeof(Real) * h->n_x, cudaMemcpyDeviceToDevice));
  CUDA_TRY(h, cudaMemcpy(h->d_hi0, d.hi, sizeof(Real) * h->n_x, cudaMemcpyDeviceToDevice));
  h->fixed.assign((size_t)sTG, 0);
  return QG_OK;
}

// One round of batch rounding on the device data of precision Real.
template <typename Real, typename Dc>
int round_batch_dev(qg_ctx *h, Dev<Real, Dc> &d, void *xv, double frac, int64_t *n_fixed, int64_t *n_bin) {
  Real *x = static_cast<Real *>(xv);
  const long long sTG = d.n_pairs;
  int rc;
  if ((rc = round_alloc(h, d))) return rc;
  for (int b = 0; b < h->n_inst; ++b) {
    const Inst &I = h->plan.tab.I[b];
    if (!I.uc) continue;
    CUDA_TRY(h, (launch_round_project<Real, Dc>(d, I, x, h->d_fixed, h->d_dist, (Real *)h->d_proj, h->stream)));
  }
  std::vector<double> dist((size_t)sTG);
  CUDA_TRY(h, cudaMemcpyAsync(dist.data(), h->d_dist, sizeof(double) * sTG, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  long long nf = 0, nb = 0;
  for (int b = 0; b < h->n_inst; ++b) {
    const Inst &I = h->plan.tab.I[b];
    if (!I.uc) continue;
    const long long TG = (long long)I.T * I.G;
    std::vector<int> freev;
    for (long long e = 0; e < TG; ++e)
      if (!h->fixed[I.tg0 + e]) freev.push_back((int)e);
    const long long take = std::min<long long>((long long)freev.size(), (long long)std::ceil(frac * freev.size()));
    // the unfixed pairs whose projection moved them least; ties by pair index
    std::stable_sort(freev.begin(), freev.end(),
                     [&](int a, int c) { return dist[I.tg0 + a] < dist[I.tg0 + c]; });
    std::vector<int> pick(freev.begin(), freev.begin() + take);
    std::sort(pick.begin(), pick.end());
    if (!pick.empty()) {
      CUDA_TRY(h, cudaMemcpyAsync(h->d_idx, pick.data(), sizeof(int) * pick.size(), cudaMemcpyHostToDevice, h->stream));
      CUDA_TRY(h, (launch_round_fix<Real, Dc>(d, I, x, const_cast<Real *>(d.lo), const_cast<Real *>(d.hi), h->d_idx,
                                              (int)pick.size(), h->d_fixed, (const Real *)h->d_proj, h->stream)));
      CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // the index list is reused by the next instance
    }
    for (int e : pick) h->fixed[I.tg0 + e] = 1;
    for (long long e = 0; e < TG; ++e) nf += h->fixed[I.tg0 + e];
    nb += TG;
  }
  if (n_fixed) *n_fixed = nf;
  if (n_bin) *n_bin = nb;
  return QG_OK;
}

}  // namespace

extern "C" {

int qg_round_batch(qg_ctx *h, void *x, double frac, int64_t *n_fixed, int64_t *n_binaries) {
  if (!h) return QG_ERR_INVALID_ARG;
  if (!x || !(frac > 0.0) || !(frac <= 1.0)) return fail(h, QG_ERR_INVALID_ARG, "qg_round_batch needs x and 0 < frac <= 1");
  return mixed(h) ? round_batch_dev(h, h->d32, x, frac, n_fixed, n_binaries)
                  : round_batch_dev(h, h->d64, x, frac, n_fixed, n_binaries);
}

int qg_round_reset(qg_ctx *h) {
  if (!h) return QG_ERR_INVALID_ARG;
  if (!h->d_fixed) return QG_OK;
  const size_t rs = mixed(h) ? sizeof(float) : sizeof(double);
  void *lo = mixed(h) ? (void *)h->d32.lo : (void *)h->d64.lo;
  void *hi = mixed(h) ? (void *)h->d32.hi : (void *)h->d64.hi;
  CUDA_TRY(h, cudaMemcpyAsync(lo, h->d_lo0, rs * h->n_x, cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(hi, h->d_hi0, rs * h->n_x, cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_fixed, 0, h->fixed.size(), h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  std::fill(h->fixed.begin(), h->fixed.end(), 0);
  return QG_OK;
}

int qg_tile_shape(const qg_ctx *h, int32_t inst, int32_t shape[2]) {
  if (!h || inst < 0 || inst >= h->n_inst || !shape) return QG_ERR_INVALID_ARG;
  shape[0] = h->plan.tab.I[inst].ctg_tb;
  shape[1] = h->plan.tab.I[inst].ctg_mg;
  return QG_OK;
}

int qg_bounds_report(int64_t *line, uint64_t *addr) {
  long long l = 0;
  unsigned long long a = 0;
  const int r = bounds_report(&l, &a);
  if (r < 0) return QG_ERR_UNSUPPORTED;
  if (line) *line = l;
  if (addr) *addr = a;
  return r;
}

int qg_version(void) { return 302; }

}  // extern "C"
